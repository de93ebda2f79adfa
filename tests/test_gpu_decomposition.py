"""The decomposed step on one GPU: a mesh split into 2-D blocks, each block
its own solver of the extended block (owned cells plus the halo ring), the
halo ring refreshed every step through the library's line pack / unpack
kernels on device buffers, in-process (the transport of the multi-GPU path
is point-to-point messages of the same buffers; its host logic is tested
with gloo ranks on CPU).  Against the FP64 oracle on the whole mesh: FP64 to
relative 1e-12, FP32-deviation storage to 1e-6 of max |f_tilde|; the owned
cells' FP64 sums against the oracle's; and the line copies themselves."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dv():
    from paper_1511_00242_gb300 import build
    build.build()
    import paper_1511_00242_gb300 as dv
    return dv


def _cases():
    cav, cf = W.cavity(150, Re=300, scheme="dugks", stretch_beta=1.3)
    box = W.cavity_four_lids(131, 70, scheme="bkg", kind="diffuse")
    plate, _ = W.flat_plate(nx_up=30, nx_plate=100, ny=66, scheme="dugks", Re_L=3e3)
    tg, _ = W.taylor_green_box(128, scheme="bkg")
    return [cav, box, plate, tg]


@pytest.mark.parametrize("k", range(4))
@pytest.mark.parametrize("PX,PY", [(2, 1), (2, 2), (3, 2)])
def test_decomposed_step_matches_oracle(dv, k, PX, PY):
    from paper_1511_00242_gb300 import decomp
    case = _cases()[k]
    fields, _ = W.random_state(case, 40 + k)
    steps = 20
    o = O.step(case, O.init_equilibrium(case, *fields), steps)
    for precision in ("f64", "f32_dev"):
        g, sums = decomp.run_local(case, PX, PY, fields, steps, precision)
        if precision == "f64":
            assert float(np.max(np.abs(g - o) / np.abs(o))) < 1e-12
            np.testing.assert_allclose(sums, O.conserved(case, o), rtol=1e-12, atol=1e-14)
        else:
            assert float(np.max(np.abs(g - o)) / np.max(np.abs(o))) < 1e-6


@pytest.mark.parametrize("precision", ["f64", "f32_dev", "bf16_dev"])
def test_line_copies_round_trip(dv, precision):
    torch = pytest.importorskip("torch")
    case, fields = W.cavity(70, Re=200, scheme="dugks")
    (r, u, v), _ = W.random_state(case, 3)
    with dv.Solver(case, precision=precision) as s:
        s.init_equilibrium(r, u, v)
        f = s.get_f()
        es = s.device_state()[3]
        dt = {8: torch.float64, 4: torch.float32, 2: torch.float16}[es]
        col = torch.empty((9, 30), dtype=dt, device="cuda")
        s.pack_line(0, 5, 10, 40, col.data_ptr())     # column 5, rows 10..39
        row = torch.empty((9, 70), dtype=dt, device="cuda")
        s.pack_line(1, 69, 0, 70, row.data_ptr())     # the last row
        s.unpack_line(1, 0, 0, 70, row.data_ptr())    # into the first row
        s.unpack_line(0, 60, 10, 40, col.data_ptr())  # into column 60
        g = s.get_f()
        want = f.copy()
        want[:, 0, :] = f[:, 69, :]
        want[:, 10:40, 60] = f[:, 10:40, 5]
        np.testing.assert_array_equal(g, want)
        for bad in ((0, 70, 0, 10), (1, 0, 5, 71), (2, 0, 0, 1), (0, 1, 4, 4)):
            with pytest.raises(dv.DvbeError) as e:
                s.pack_line(*bad, col.data_ptr())
            assert e.value.status == dv.DVBE_ERR_INVALID_ARG
        w = s.conserved_window(3, 4, 50, 60)
        sub = dict(case, nx=50, ny=60, xf=case["xf"][3:54], yf=case["yf"][4:65], bc=W.periodic_bc())
        np.testing.assert_allclose(w, O.conserved(sub, np.ascontiguousarray(g[:, 4:64, 3:53])),
                                   rtol=1e-13, atol=1e-15)
