"""The batched form against the FP64 oracle, case by case.

Ten uneven cases in one batch: Taylor-Green boxes and cavities, DUGKS and
BKG, sides 32 to 96, uniform and tanh-stretched meshes, bounce-back and
diffuse walls with a moving lid, a flat plate with inflow, outflow and
symmetry segments.  Every case's f_tilde after 60 steps (graphs of 20 steps)
is compared element by element with the oracle's: FP64 to relative 1e-12,
FP32-deviation storage to 1e-6 of max |f_tilde|."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

STEPS = 60


@pytest.fixture(scope="module")
def dv():
    from paper_1511_00242_gb300 import build
    build.build()
    import paper_1511_00242_gb300 as dv
    return dv


def _cases():
    out = []
    for k, (n, scheme) in enumerate([(32, "dugks"), (64, "bkg"), (96, "dugks"), (40, "bkg")]):
        case, _ = W.taylor_green_box(n, u0=0.03, scheme=scheme, dt_over_tau=4.0 + k)
        out.append(case)
    out.append(W.cavity(48, Re=400, scheme="dugks")[0])
    out.append(W.cavity(56, Re=200, scheme="bkg", stretch_beta=1.5)[0])
    out.append(W.cavity(33, Re=100, scheme="dugks", kind="diffuse", stretch_beta=1.2)[0])
    out.append(W.cavity(70, Re=800, scheme="bkg", kind="diffuse")[0])
    out.append(W.flat_plate(nx_up=10, nx_plate=30, ny=36, scheme="dugks", Re_L=2e3)[0])
    out.append(W.cavity_four_lids(62, 35, scheme="bkg"))
    return out


@pytest.fixture(scope="module")
def reference():
    """Initial states and the oracle's f_tilde after STEPS steps."""
    res = []
    for k, case in enumerate(_cases()):
        fields, _ = W.random_state(case, 100 + k)
        res.append((case, fields, O.step(case, O.init_equilibrium(case, *fields), STEPS)))
    return res


@pytest.mark.parametrize("precision", ["f64", "f32_dev"])
def test_batch_against_oracle(dv, reference, precision):
    b = dv.Batch([c for c, _, _ in reference], precision=precision)
    try:
        b.set_launch(strip_rows=16, warps_per_block=4)
        for k, (_, fields, _) in enumerate(reference):
            b.init_equilibrium(k, *fields)
        b.step(STEPS, graph_chunk=20)
        for k, (case, _, o) in enumerate(reference):
            assert b.case_status(k) == 0, case["name"]
            g = b.get_f(k)
            if precision == "f64":
                err = float(np.max(np.abs(g - o) / np.abs(o)))
                assert err < 1e-12, (case["name"], err)
            else:
                err = float(np.max(np.abs(g - o)) / np.max(np.abs(o)))
                assert err < 1e-6, (case["name"], err)
    finally:
        b.close()
