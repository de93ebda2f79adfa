"""Seeded random configurations against the oracle: mesh widths around the
strip edges of both lane layouts (30 columns per strip with one column per
lane in FP64, 60 with two in FP32), random heights, uniform or randomly
stretched spacing, random boundary kinds and segments on each side, random
launch shapes, both schemes and the upwind collision-free face, and for half
of the configurations a velocity model with RT drawn log-uniformly from
[0.1, 3] (lattice speed c = sqrt(3 RT) != 1; wall and free-stream speeds
scaled by c).  FP64 to relative 1e-12 and FP32-deviation storage to 1e-6 of
max |f_tilde| after 20 steps."""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

NCONF = 40
WIDTHS = [2, 3, 29, 30, 31, 32, 58, 59, 60, 61, 62, 89, 90, 91, 119, 120, 121, 122]


@pytest.fixture(scope="module")
def dv():
    from paper_1511_00242_gb300 import build
    build.build()
    import paper_1511_00242_gb300 as dv
    return dv


def _faces(rng, n, length):
    if rng.random() < 0.5:
        return W.uniform_faces(n, 0.0, length)
    w = rng.uniform(0.5, 1.5, n)
    return np.concatenate([[0.0], np.cumsum(w)]) * (length / w.sum())


def _side(rng, length, tangential_speed):
    """Segments of one non-periodic side: one kind, or two kinds split at a
    random point along it."""
    kinds = ["wall", "diffuse", "inflow", "outflow", "symmetry"]

    def seg(kind, s0, s1):
        if kind in ("wall", "diffuse"):
            return (kind, s0, s1, 1.0, tangential_speed if rng.random() < 0.5 else 0.0, 0.0)
        if kind == "inflow":
            return ("inflow", s0, s1, 1.0 + 0.01 * rng.random(), 0.03 * rng.random(), 0.0)
        return (kind, s0, s1, 1.0, 0.0, 0.0)

    if rng.random() < 0.7:
        return [seg(str(rng.choice(kinds)), -W.INF, W.INF)]
    cut = float(rng.uniform(0.3, 0.7) * length)
    a, b = rng.choice(kinds, 2, replace=False)
    return [seg(str(a), -W.INF, cut), seg(str(b), cut, W.INF)]


def _config(k):
    rng = np.random.default_rng(1000 + k)
    nx = int(rng.choice(WIDTHS)) if rng.random() < 0.8 else int(rng.integers(2, 131))
    ny = int(rng.integers(2, 41))
    per_x, per_y = bool(rng.random() < 0.4), bool(rng.random() < 0.4)
    xf, yf = _faces(rng, nx, nx / 16.0), _faces(rng, ny, ny / 16.0)
    per = [("periodic", -W.INF, W.INF, 0.0, 0.0, 0.0)]
    bc = [per if per_x else _side(rng, yf[-1], 0.0), per if per_x else _side(rng, yf[-1], 0.0),
          per if per_y else _side(rng, xf[-1], 0.0), per if per_y else _side(rng, xf[-1], 0.04)]
    scheme = str(rng.choice(["dugks", "bkg", "cfree_upwind"], p=[0.45, 0.45, 0.1]))
    rng_rt = np.random.default_rng(5000 + k)
    rt = W.RT_LATTICE if rng_rt.random() < 0.5 else float(10 ** rng_rt.uniform(-1, np.log10(3)))
    c = np.sqrt(3 * rt)
    bc = [[(kind, s0, s1, rho, ux * c, uy * c) for (kind, s0, s1, rho, ux, uy) in side] for side in bc]
    case = dict(nx=nx, ny=ny, xf=xf, yf=yf, RT=rt, tau=float(rng.uniform(0.002, 0.05)) / c,
                dt=W.cfl_dt(xf, yf, float(rng.uniform(0.2, 0.8)), rt), scheme=scheme, bc=bc)
    launch = dict(strip_rows=int(rng.choice([1, 2, 3, 5, 8, 16, 33])),
                  warps_per_block=int(rng.choice([1, 2, 4, 8])), blocks=int(rng.choice([0, 0, 3])))
    return case, launch, int(rng.integers(1 << 30))


@pytest.mark.parametrize("k", range(NCONF))
def test_random_configuration(dv, k):
    case, launch, seed = _config(k)
    fields, delta = W.random_state(case, seed, amp_neq=1e-3)
    o = O.step(case, O.init_equilibrium(case, *fields) + delta, 20)
    for precision in ("f64", "f32_dev"):
        with dv.Solver(case, precision=precision) as s:
            s.set_launch(**launch)
            s.init_equilibrium(*fields)
            s.init_f(s.get_f() + delta)
            s.step(20)
            g = s.get_f()
        if precision == "f64":
            err = float(np.max(np.abs(g - o) / np.abs(o)))
            assert err < 1e-12, (case["nx"], case["ny"], case["scheme"], launch, err)
        else:
            err = float(np.max(np.abs(g - o)) / np.max(np.abs(o)))
            assert err < 1e-6, (case["nx"], case["ny"], case["scheme"], launch, err)
