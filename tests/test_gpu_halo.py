"""Rows with halo columns on meshes periodic in x: the step writes copies of
the columns at each end of a row next to the other end, so the strips at the
two ends read their wrap neighbours as cells and run in the kernel without
boundary code.  Parity with the FP64 oracle (FP64 to 1e-12, FP32 storage to
1e-6 of max |f_tilde|) on doubly periodic meshes (one kernel per step), on
meshes periodic in x with walls (the halo strips and the wall rows), at the
narrowest halo width and just below it, at odd widths (FP64); the halo
refreshed after host writes (init, unpack_line); and the device view of the
state, which addresses column 0."""
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


PER = [("periodic", -W.INF, W.INF, 0.0, 0.0, 0.0)]


def _case(nx, ny, scheme, walls):
    xf = W.uniform_faces(nx, 0.0, nx / 32.0)
    yf = W.tanh_faces(ny, 0.0, ny / 32.0, 0.8) if walls else W.uniform_faces(ny, 0.0, ny / 32.0)
    bc = [PER, PER, [W.wall(0.01, 0.0, kind="diffuse")], [W.wall(0.05, 0.0)]] if walls else [PER] * 4
    return dict(nx=nx, ny=ny, xf=xf, yf=yf, RT=W.RT_LATTICE, tau=0.01, dt=W.cfl_dt(xf, yf, 0.5),
                scheme=scheme, bc=bc)


def _check(g, o, precision):
    if precision == "f64":
        assert float(np.max(np.abs(g - o) / np.abs(o))) < 1e-12
    else:
        assert float(np.max(np.abs(g - o)) / np.max(np.abs(o))) < 1e-6


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
@pytest.mark.parametrize("nx,ny,walls,precisions", [
    (186, 41, False, ("f64", "f32_dev", "f32")),  # ragged last strip (6 / 6 columns)
    (186, 55, True, ("f64", "f32_dev")),          # halo strips plus the wall rows
    (61, 23, False, ("f64",)),                    # odd width: FP64 keeps the halo
    (8, 12, False, ("f32_dev", "f64")),           # narrowest halo (2 x 4 FP32 columns)
    (6, 12, False, ("f32_dev",)),                 # below it: plain rows and wrap copies
])
def test_halo_rows_match_oracle(dv, scheme, nx, ny, walls, precisions):
    case = _case(nx, ny, scheme, walls)
    fields, delta = W.random_state(case, nx + ny, amp_neq=1e-3)
    o = O.step(case, O.init_equilibrium(case, *fields) + delta, 14)
    for precision in precisions:
        with dv.Solver(case, precision=precision) as s:
            s.set_launch(strip_rows=8, warps_per_block=2)
            s.init_equilibrium(*fields)
            s.init_f(s.get_f() + delta)
            l0 = s.launch_count()
            s.step(14)
            if not walls and nx >= 8 and (precision == "f64" or nx % 2 == 0):
                assert s.launch_count() - l0 == 14  # every strip inner: one kernel per step
            _check(s.get_f(), o, precision)


@pytest.mark.parametrize("precision", ["f64", "f32_dev"])
def test_halo_follows_host_writes(dv, precision):
    """unpack_line into the first and the last column, then steps: the halo
    copies must carry the new values across the wrap."""
    torch = pytest.importorskip("torch")
    case = _case(124, 30, "dugks", walls=False)
    fields, delta = W.random_state(case, 5, amp_neq=1e-3)
    with dv.Solver(case, precision=precision) as s:
        s.init_equilibrium(*fields)
        s.init_f(s.get_f() + delta)
        f = s.get_f()
        dt = {8: torch.float64, 4: torch.float32, 2: torch.float16}[s.device_state()[3]]
        buf = torch.empty((9, case["ny"]), dtype=dt, device="cuda")
        s.pack_line(0, 60, 0, case["ny"], buf.data_ptr())   # column 60 into columns 0 and nx-1
        s.unpack_line(0, 0, 0, case["ny"], buf.data_ptr())
        s.unpack_line(0, case["nx"] - 1, 0, case["ny"], buf.data_ptr())
        f[:, :, 0] = f[:, :, 60]
        f[:, :, -1] = f[:, :, 60]
        np.testing.assert_array_equal(s.get_f(), f)
        s.step(9)
        g = s.get_f()
    _check(g, O.step(case, f, 9), precision)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_device_view_addresses_column_zero(dv, precision):
    """The allocation-free sums read the state through dvbe_device_state's
    pointer and pitch, on a halo layout as on plain rows."""
    torch = pytest.importorskip("torch")
    case = _case(126, 40, "bkg", walls=True)
    (r, u, v), _ = W.random_state(case, 8)
    with dv.Solver(case, precision=precision) as s:
        s.init_equilibrium(r, u, v)
        s.step(5)
        ref = s.conserved()
        ptr, pitch, plane, _ = s.device_state()
        assert pitch >= case["nx"] + 4 and plane == pitch * case["ny"]
        dx = torch.tensor(np.diff(case["xf"]), dtype=torch.float64, device="cuda")
        dy = torch.tensor(np.diff(case["yf"]), dtype=torch.float64, device="cuda")
        out = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
        dv.dvbe_conserved_noalloc(ptr, precision, case["nx"], case["ny"], pitch, dx.data_ptr(),
                                  dy.data_ptr(), case["RT"], 1.0, 0.0, out.data_ptr())
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-13, atol=1e-15 * abs(ref[0]))
