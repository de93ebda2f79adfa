"""Laminar flat-plate boundary layer on a 512 x 256 stretched mesh (Sec 3.3
set-up: U = 0.1, L = 1, Re_L = 1e5, y cells growing geometrically from
dy_min = L / 5000), FP32 arithmetic with FP32-deviation storage, DUGKS
against BKG at CFL 0.1, 0.5, 0.9 and 0.95.  After 2.5 flow-through times the
u profiles at x = 0.2 L and 0.6 L are compared with the Blasius solution
(max |u / U - f'| over eta < 5).  DUGKS follows Blasius at every CFL number;
BKG's error grows with the time step (its numerical dissipation is
proportional to dt, Sec 2.4) or it diverges near CFL 1."""
import math

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dv():
    from paper_1511_00242_gb300 import build
    build.build()
    import paper_1511_00242_gb300 as dv
    return dv


def _profile_error(case, u, X):
    from oracle import blasius
    xc, yc = W.centres(case["xf"]), W.centres(case["yf"])
    i = int(np.searchsorted(xc, X)) - 1
    a = (X - xc[i]) / (xc[i + 1] - xc[i])
    col = (1 - a) * u[:, i] + a * u[:, i + 1]
    ub, _ = blasius.profiles(yc, X, case["U"], case["nu"])
    inside = yc < 5.0 * math.sqrt(case["nu"] * X / case["U"])
    return float(np.max(np.abs(col[inside] / case["U"] - ub[inside])))


def _run(dv, scheme, cfl):
    case, fields = W.flat_plate(nx_up=170, nx_plate=342, ny=256, cfl=cfl, scheme=scheme)
    steps = int(round(2.5 * 1.5 / case["U"] / case["dt"]))
    with dv.Solver(case, precision="f32_dev") as s:
        s.autotune(5)
        s.set_launch(graph_chunk=500)
        s.init_equilibrium(*fields)
        try:
            s.step(steps)
        except dv.DvbeError as e:
            if e.status == dv.DVBE_ERR_DIVERGED:
                return None, steps
            raise
        _, u, _ = s.moments()
    if not np.all(np.isfinite(u)):
        return None, steps
    return (_profile_error(case, u, 0.2), _profile_error(case, u, 0.6)), steps


def test_plate_512x256_cfl_sweep(dv):
    out = {}
    for scheme in ("dugks", "bkg"):
        for cfl in (0.1, 0.5, 0.9, 0.95):
            err, steps = _run(dv, scheme, cfl)
            out[(scheme, cfl)] = err
            msg = "diverged" if err is None else f"x=0.2L {err[0]:.4f}, x=0.6L {err[1]:.4f}"
            print(f"plate 512x256 {scheme} CFL {cfl} ({steps} steps): max |u/U - f'| {msg}")
    for cfl in (0.1, 0.5, 0.9, 0.95):
        assert out[("dugks", cfl)] is not None and max(out[("dugks", cfl)]) < 0.05, (cfl, out)
    b01 = out[("bkg", 0.1)]
    assert b01 is not None
    for cfl in (0.5, 0.9, 0.95):
        b = out[("bkg", cfl)]
        assert b is None or max(b) > max(b01), (cfl, out)
