"""The two-kernel step: strips that touch no boundary run in a kernel compiled
without boundary code, the ring of strips around them in a second kernel cut
into shorter pieces.  Parity with the FP64 oracle on meshes that have an
inner rectangle and ragged edges on every side, for strip heights whose ring
pieces are shorter than the strip (32, 16, 12: pieces of 8, 8, 6 rows) or as
tall (5), with periodic sides and with walls, FP64 to 1e-12 and FP32
deviations to 1e-6 of max |f_tilde|; and the launch count of a step."""
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


def _per():
    return [("periodic", -W.INF, W.INF, 0.0, 0.0, 0.0)]


def _case(nx, ny, scheme, walls, stretched):
    xf = W.tanh_faces(nx, 0.0, nx / 32.0, 0.8) if stretched else W.uniform_faces(nx, 0.0, nx / 32.0)
    yf = W.uniform_faces(ny, 0.0, ny / 32.0)
    if walls:
        bc = [[W.wall(0.0, 0.02)], [W.wall(kind="diffuse")], [W.wall()], [W.wall(0.05, 0.0)]]
    else:
        bc = [_per(), _per(), _per(), _per()]
    return dict(nx=nx, ny=ny, xf=xf, yf=yf, RT=W.RT_LATTICE, tau=0.01, dt=W.cfl_dt(xf, yf, 0.5),
                scheme=scheme, bc=bc)


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
@pytest.mark.parametrize("H", [32, 16, 12, 5])
@pytest.mark.parametrize("walls", [False, True])
def test_inner_and_ring_kernels(dv, scheme, H, walls):
    # FP32 strips hold 60 columns, FP64 strips 30: 187 columns give inner
    # strips in both layouts and a ragged last strip; 3H + 7 rows give an
    # inner band of strips and a ragged top piece
    nx, ny = 187, 3 * H + 7
    case = _case(nx, ny, scheme, walls, stretched=walls)
    fields, delta = W.random_state(case, H + 7 * walls, amp_neq=1e-3)
    o = O.step(case, O.init_equilibrium(case, *fields) + delta, 12)
    for precision in ("f64", "f32_dev"):
        with dv.Solver(case, precision=precision) as s:
            s.set_launch(strip_rows=H, warps_per_block=2)
            s.init_equilibrium(*fields)
            s.init_f(s.get_f() + delta)
            l0 = s.launch_count()
            s.step(12)
            # inner kernel and ring kernel per step; a mesh periodic in x keeps
            # halo columns (FP64 at any width, pairs of FP32 columns at even
            # widths) and then every strip is inner
            halo = not walls and (precision == "f64" or nx % 2 == 0)
            assert s.launch_count() - l0 == (12 if halo else 24)
            g = s.get_f()
        if precision == "f64":
            assert float(np.max(np.abs(g - o) / np.abs(o))) < 1e-12
        else:
            assert float(np.max(np.abs(g - o)) / np.max(np.abs(o))) < 1e-6


@pytest.mark.parametrize("blocks", [0, 7])
def test_persistent_inner_grid(dv, blocks):
    """A fixed grid smaller than the inner work (warps loop over strips)."""
    case = _case(250, 70, "dugks", walls=True, stretched=True)
    fields, delta = W.random_state(case, 3, amp_neq=1e-3)
    o = O.step(case, O.init_equilibrium(case, *fields) + delta, 10)
    with dv.Solver(case, precision="f64") as s:
        s.set_launch(strip_rows=8, warps_per_block=4, blocks=blocks)
        s.init_equilibrium(*fields)
        s.init_f(s.get_f() + delta)
        s.step(10)
        assert float(np.max(np.abs(s.get_f() - o) / np.abs(o))) < 1e-12


def test_small_mesh_runs_one_kernel(dv):
    """No inner strip: one kernel per step over every strip."""
    case = _case(61, 9, "bkg", walls=True, stretched=False)
    with dv.Solver(case, precision="f32_dev") as s:
        s.set_launch(strip_rows=4)
        s.init_equilibrium(*W.random_state(case, 1)[0])
        l0 = s.launch_count()
        s.step(5)
        assert s.launch_count() - l0 == 5
