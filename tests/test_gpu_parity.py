"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

FP64 bar: relative max error on f_tilde <= 1e-12 after 100 steps (the
arithmetic differs from the oracle only in the order of rounding).  Sizes
span several strips (30 columns in FP64, 60 in FP32) and several row strips
with ragged tails.
Lower precisions are held to bounds derived from their storage rounding
(see test_precision_modes_error_bounds)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


@pytest.fixture(scope="module")
def dv():
    from paper_1511_00242_gb300 import build
    build.build()
    import paper_1511_00242_gb300 as dv
    return dv


def _per():
    return [("periodic", -W.INF, W.INF, 0.0, 0.0, 0.0)]


def periodic_case(nx, ny, scheme, xf=None, yf=None, tau=0.02, cfl=0.5):
    xf = W.uniform_faces(nx, 0.0, nx / 32.0) if xf is None else xf
    yf = W.uniform_faces(ny, 0.0, ny / 32.0) if yf is None else yf
    return dict(nx=nx, ny=ny, xf=xf, yf=yf, RT=W.RT_LATTICE, tau=tau, dt=W.cfl_dt(xf, yf, cfl),
                scheme=scheme, bc=[_per(), _per(), _per(), _per()])


def gpu_state(dv, s, fields, delta=None):
    """Library-side initial state: its own equilibrium, plus a perturbation."""
    s.init_equilibrium(*fields)
    if delta is not None:
        s.init_f(s.get_f() + delta)


def oracle_state(case, fields, delta=None):
    f = O.init_equilibrium(case, *fields)
    return f if delta is None else f + delta


def rel_err(a, b):
    return float(np.max(np.abs(a - b) / np.abs(b)))


def run_pair(dv, case, steps, seed=0, amp_neq=1e-3, fields=None, launch=None, precision="f64",
             **kw):
    if fields is None:
        fields, delta = W.random_state(case, seed, amp_neq=amp_neq)
    else:
        delta = None
    with dv.Solver(case, precision=precision, **kw) as s:
        if launch:
            s.set_launch(**launch)
        gpu_state(dv, s, fields, delta)
        s.step(steps)
        g = s.get_f()
    o = O.step(case, oracle_state(case, fields, delta), steps)
    return g, o


# ------------------------------------------------------------------ FP64 parity

@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_taylor_green_32(dv, scheme):
    """Taylor-Green 32^2 on [0, 2pi]^2, nu = 0.05, CFL 0.5, 150 steps."""
    case, fields = W.taylor_green_box(32, scheme=scheme)
    g, o = run_pair(dv, case, 150, fields=fields)
    assert rel_err(g, o) < TOL64


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
@pytest.mark.parametrize("launch", [dict(strip_rows=1, warps_per_block=1),
                                    dict(strip_rows=3, warps_per_block=4),
                                    dict(strip_rows=7, warps_per_block=8, blocks=3),
                                    dict(strip_rows=64, warps_per_block=2)])
def test_ragged_periodic(dv, scheme, launch):
    """Random state on a periodic 67 x 23 mesh (three strips, ragged), any launch shape."""
    case = periodic_case(67, 23, scheme)
    g, o = run_pair(dv, case, 100, seed=1, launch=launch)
    assert rel_err(g, o) < TOL64


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
@pytest.mark.parametrize("nx", [2, 29, 30, 31, 60, 61])
def test_strip_edges(dv, scheme, nx):
    """Mesh widths at and around the 30-column strip boundary, periodic in x,
    walls in y."""
    ny = 9
    xf, yf = W.uniform_faces(nx, 0, nx / 16.0), W.uniform_faces(ny, 0, ny / 16.0)
    case = dict(nx=nx, ny=ny, xf=xf, yf=yf, RT=W.RT_LATTICE, tau=0.01, dt=W.cfl_dt(xf, yf, 0.5),
                scheme=scheme, bc=[_per(), _per(), [W.wall()], [W.wall(0.05, 0.0)]])
    g, o = run_pair(dv, case, 100, seed=2, launch=dict(strip_rows=4))
    assert rel_err(g, o) < TOL64


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_random_stretched_periodic(dv, scheme):
    rng = np.random.default_rng(3)
    xf = np.concatenate([[0], np.cumsum(rng.uniform(0.5, 1.5, 45))]) / 45
    yf = np.concatenate([[0], np.cumsum(rng.uniform(0.5, 1.5, 38))]) / 38
    case = periodic_case(45, 38, scheme, xf=xf, yf=yf, tau=0.005)
    g, o = run_pair(dv, case, 100, seed=4)
    assert rel_err(g, o) < TOL64


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
@pytest.mark.parametrize("kind", ["wall", "diffuse"])
@pytest.mark.parametrize("beta", [None, 1.5])
def test_cavity(dv, scheme, kind, beta):
    """Lid-driven cavity 40^2, uniform and tanh-stretched, both wall kinds."""
    case, fields = W.cavity(40, Re=400, scheme=scheme, stretch_beta=beta, kind=kind)
    g, o = run_pair(dv, case, 100, fields=fields, launch=dict(strip_rows=16))
    assert rel_err(g, o) < TOL64


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
@pytest.mark.parametrize("kind", ["wall", "diffuse"])
def test_four_lid_box_corners(dv, scheme, kind):
    """All four walls moving (every corner ghost in use), tanh mesh: FP64
    parity, and the 180-degree rotation symmetry of the problem kept to
    rounding."""
    case = W.cavity_four_lids(75, 43, scheme=scheme, kind=kind)
    fields = W.rotation_symmetric_state(case, 4)
    g, o = run_pair(dv, case, 100, fields=fields, launch=dict(strip_rows=8))
    assert rel_err(g, o) < TOL64
    with dv.Solver(case) as s:
        s.set_launch(strip_rows=8)
        s.init_equilibrium(*fields)
        s.step(100)
        r, u, v = s.moments()
    R = lambda a: a[::-1, ::-1]
    assert np.max(np.abs(r - R(r))) < 1e-13 and np.max(np.abs(u + R(u))) < 1e-13


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_flat_plate(dv, scheme):
    """Inflow (W, N), outflow (E), symmetry + wall segments (S), stretched both ways."""
    case, fields = W.flat_plate(nx_up=12, nx_plate=40, ny=26, scheme=scheme)
    g, o = run_pair(dv, case, 100, fields=fields, launch=dict(strip_rows=8))
    assert rel_err(g, o) < TOL64


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_walls_on_x_sides_periodic_y(dv, scheme):
    """Walls on W/E with periodic S/N: x-ghosts of wrapped rows, moving walls."""
    nx, ny = 35, 21
    xf, yf = W.tanh_faces(nx, 0, 1, 1.0), W.uniform_faces(ny, 0, 0.6)
    case = dict(nx=nx, ny=ny, xf=xf, yf=yf, RT=W.RT_LATTICE, tau=0.01, dt=W.cfl_dt(xf, yf, 0.5),
                scheme=scheme, bc=[[W.wall(0, 0.03)], [("symmetry", -W.INF, W.INF, 1, 0, 0)],
                                   _per(), _per()])
    g, o = run_pair(dv, case, 100, seed=5, launch=dict(strip_rows=5))
    assert rel_err(g, o) < TOL64


def test_bkg_fd_form(dv):
    """BKG in finite-difference form (Eqs. bkgfd, central_schemes) against the
    oracle's finite-difference step and the finite-volume form."""
    case = periodic_case(64, 40, "bkg", tau=0.003)
    fields, delta = W.random_state(case, 6, amp_neq=1e-3)
    with dv.Solver(case, bkg_fd=True) as s:
        s.set_launch(strip_rows=8)
        gpu_state(dv, s, fields, delta)
        s.step(100)
        g = s.get_f()
    o = O.step_bkg_fd(case, oracle_state(case, fields, delta), 100)
    assert rel_err(g, o) < TOL64


def test_chapman_enskog_init(dv):
    for scheme in ("dugks", "bkg"):
        case, fields, d, _ = W.taylor_green_paper(24, scheme)
        with dv.Solver(case) as s:
            s.init_chapman_enskog(*fields, d)
            g = s.get_f()
        o = O.init_chapman_enskog(case, *fields, d)
        assert rel_err(g, o) < 1e-14


def test_diagnostics(dv):
    case, fields = W.cavity(33, Re=200, stretch_beta=1.2)
    fields, delta = W.random_state(case, 7, amp_neq=1e-3)
    with dv.Solver(case) as s:
        gpu_state(dv, s, fields, delta)
        s.step(20)
        g = s.get_f()
        r, u, v = s.moments()
        c = s.conserved()
        ua, va = np.sin(np.arange(33 * 33)).reshape(33, 33), np.cos(np.arange(33 * 33)).reshape(33, 33)
        eu = s.l2_error_u(ua, va)
        assert s.residual() == math.inf
        s.step(5)
        r2 = s.residual()
        u2 = s.moments()
    ro, uo, vo = O.moments(case, g)
    np.testing.assert_allclose(r, ro, rtol=1e-14)
    np.testing.assert_allclose(u, uo, rtol=1e-12, atol=1e-16)
    np.testing.assert_allclose(c, O.conserved(case, g), rtol=1e-13, atol=1e-15)
    assert eu == pytest.approx(O.l2_error_u(case, g, ua, va), rel=1e-13)
    num = np.sqrt(np.sum((u2[1] - u) ** 2 + (u2[2] - v) ** 2))
    den = np.sqrt(np.sum(u2[1] ** 2 + u2[2] ** 2))
    assert r2 == pytest.approx(num / den, rel=1e-10)


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_graph_replay_is_bitwise_identical(dv, scheme):
    case = periodic_case(70, 50, scheme)
    fields, delta = W.random_state(case, 8, amp_neq=1e-3)
    out = []
    for chunk in (0, 10):
        with dv.Solver(case, precision="f32") as s:
            s.set_launch(strip_rows=16, graph_chunk=chunk)
            gpu_state(dv, s, fields, delta)
            s.step(37)
            assert s.step_count() == 37
            out.append(s.get_f())
    np.testing.assert_array_equal(out[0], out[1])


def test_divergence_is_reported(dv):
    """A NaN planted in the host state makes the step report divergence and
    leaves the solver usable."""
    case = periodic_case(40, 30, "dugks")
    with dv.Solver(case) as s:
        f = s.get_f()
        f[3, 10, 10] = np.nan
        s.init_f(f)
        with pytest.raises(dv.DvbeError) as e:
            s.step(3)
        assert e.value.status == dv.DVBE_ERR_DIVERGED
        s.init_equilibrium(np.ones((30, 40)), np.zeros((30, 40)), np.zeros((30, 40)))
        s.step(3)


def test_torch_allocator_and_stream(dv):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("CUDA is not available")
    stream = torch.cuda.Stream()
    dv.use_torch_allocator(True)
    try:
        case, fields = W.taylor_green_box(48)
        before = torch.cuda.memory_allocated()
        with dv.Solver(case, precision="f32", stream=stream.cuda_stream) as s:
            assert torch.cuda.memory_allocated() > before
            s.init_equilibrium(*fields)
            s.step(10)
            g = s.get_f()
        o = O.step(case, O.init_equilibrium(case, *fields), 10)
        assert np.max(np.abs(g - o)) < 1e-6
    finally:
        dv.use_torch_allocator(False)


# ------------------------------------------------------------------ precision modes

@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_set_density_outflow(dv, scheme):
    """Outflow at a set density (east side of the flat plate; both sides of a
    channel with fluid at another density) against the oracle, FP64 and
    FP32-deviation storage."""
    case, fields = W.flat_plate(nx_up=12, nx_plate=40, ny=26, scheme=scheme, outflow="outflow_neq")
    g, o = run_pair(dv, case, 60, fields=fields, launch=dict(strip_rows=8))
    assert rel_err(g, o) < TOL64
    xf, yf = W.uniform_faces(70, 0.0, 1.0), W.uniform_faces(9, 0.0, 9 / 70)
    side = [("outflow_neq", -W.INF, W.INF, 1.0, 0.0, 0.0)]
    chan = dict(nx=70, ny=9, xf=xf, yf=yf, RT=W.RT_LATTICE, tau=0.01, dt=W.cfl_dt(xf, yf, 0.5),
                scheme=scheme, bc=[side, side, _per(), _per()])
    fields = (np.full((9, 70), 1.02), np.full((9, 70), 0.02), np.zeros((9, 70)))
    for precision, bound in (("f64", TOL64), ("f32_dev", 1e-6)):
        g, o = run_pair(dv, chan, 40, fields=fields, precision=precision, launch=dict(strip_rows=4))
        err = rel_err(g, o) if precision == "f64" else float(np.max(np.abs(g - o)) / np.max(np.abs(o)))
        assert err < bound, (precision, err)


# ------------------------------------------- collision-free faces (Sec 2.4)

CFREE = ["cfree_upwind", "cfree_central"]


@pytest.mark.parametrize("scheme", CFREE)
def test_collision_free_faces_periodic(dv, scheme):
    """Eqs. cfd2 / cfd1: random state on a ragged periodic 67 x 23 mesh and on a
    random stretched mesh, against the oracle."""
    g, o = run_pair(dv, periodic_case(67, 23, scheme), 50, seed=11, launch=dict(strip_rows=7))
    assert rel_err(g, o) < TOL64
    rng = np.random.default_rng(12)
    xf = np.concatenate([[0], np.cumsum(rng.uniform(0.5, 1.5, 45))]) / 45
    yf = np.concatenate([[0], np.cumsum(rng.uniform(0.5, 1.5, 38))]) / 38
    g, o = run_pair(dv, periodic_case(45, 38, scheme, xf=xf, yf=yf, tau=0.005), 50, seed=13)
    assert rel_err(g, o) < TOL64


@pytest.mark.parametrize("scheme", CFREE)
@pytest.mark.parametrize("kind", ["wall", "diffuse"])
def test_collision_free_faces_walls(dv, scheme, kind):
    """Walls, the moving lid and the free-stream boundaries with collision-free
    faces: stretched cavity and flat plate against the oracle."""
    case, fields = W.cavity(40, Re=400, scheme=scheme, stretch_beta=1.5, kind=kind)
    g, o = run_pair(dv, case, 50, fields=fields, launch=dict(strip_rows=16))
    assert rel_err(g, o) < TOL64
    case, fields = W.flat_plate(nx_up=12, nx_plate=40, ny=26, scheme=scheme)
    g, o = run_pair(dv, case, 50, fields=fields, launch=dict(strip_rows=8))
    assert rel_err(g, o) < TOL64


@pytest.mark.parametrize("scheme", CFREE)
def test_collision_free_faces_fp32(dv, scheme):
    """FP32 arithmetic with FP32-deviation storage, same bound as the other
    schemes (storage rounding of 2^-24 |delta| per step, 50 steps)."""
    case, fields = W.taylor_green_box(64, u0=0.05, scheme=scheme)
    g, o = run_pair(dv, case, 50, fields=fields, precision="f32_dev")
    assert np.max(np.abs(g - o)) / np.max(np.abs(o)) < 1e-6


def test_batch_rejects_collision_free_faces(dv):
    case, _ = W.taylor_green_box(32, scheme="cfree_upwind")
    with pytest.raises(dv.DvbeError) as e:
        dv.Batch([case], precision="f32")
    assert e.value.status == dv.DVBE_ERR_UNSUPPORTED


# ------------------------------------------------------------------ paired layout

@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
@pytest.mark.parametrize("nx", [2, 59, 60, 61, 120, 121])
def test_strip_edges_paired_fp32(dv, scheme, nx):
    """FP32 arithmetic holds two columns per lane and 60 output columns per
    strip: mesh widths at and around those edges, periodic in x and walls in
    y, then walls on all sides; FP32-deviation storage against the oracle."""
    ny = 9
    xf, yf = W.uniform_faces(nx, 0, nx / 16.0), W.uniform_faces(ny, 0, ny / 16.0)
    for bcx in (_per(), [W.wall()]):
        case = dict(nx=nx, ny=ny, xf=xf, yf=yf, RT=W.RT_LATTICE, tau=0.01,
                    dt=W.cfl_dt(xf, yf, 0.5), scheme=scheme,
                    bc=[bcx, bcx, [W.wall()], [W.wall(0.05, 0.0)]])
        g, o = run_pair(dv, case, 40, seed=2, precision="f32_dev", launch=dict(strip_rows=4))
        assert np.max(np.abs(g - o)) / np.max(np.abs(o)) < 1e-6


@pytest.mark.parametrize("precision,bound", [("f32", 1e-5), ("f32_dev", 1e-6),
                                             ("f16_dev", 3e-3), ("bf16_dev", 3e-2)])
@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_precision_modes_error_bounds(dv, precision, bound, scheme):
    """FP32 arithmetic with FP32 / FP32-deviation / FP16 / BF16 deviation
    storage against the FP64 oracle after 100 steps, max error relative to
    max |f_tilde|.  Bounds from storage rounding accumulated over 100 steps:
    FP32 2^-24 |f| per step (1e-5), FP32 deviations 2^-24 |delta| (1e-6),
    FP16 2^-11 |delta| (3e-3), BF16 2^-8 |delta| (3e-2), |delta| ~ 3% of |f|."""
    case, fields = W.taylor_green_box(64, u0=0.05, scheme=scheme)
    g, o = run_pair(dv, case, 100, fields=fields, precision=precision)
    err = np.max(np.abs(g - o)) / np.max(np.abs(o))
    assert err < bound, err


# ------------------------------------------------------------------ batched form

@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_batch_matches_single_solver(dv, precision):
    """The batched persistent launch gives the same bits as each case's own
    solver with the same strip height."""
    cases = []
    for k, (case, fields) in enumerate(W.batched_cases(10, seed=1511, side_max=96)):
        cases.append((case, fields))
    b = dv.Batch([c for c, _ in cases], precision=precision)
    try:
        b.set_launch(strip_rows=16, warps_per_block=4)
        for k, (c, f) in enumerate(cases):
            b.init_equilibrium(k, *f)
        b.step(40, graph_chunk=10)
        for k, (c, f) in enumerate(cases):
            assert b.case_status(k) == 0
            with dv.Solver(c, precision=precision) as s:
                s.set_launch(strip_rows=16)
                s.init_equilibrium(*f)
                s.step(40)
                np.testing.assert_array_equal(b.get_f(k), s.get_f())
    finally:
        b.close()


def test_batch_divergent_case_is_isolated(dv):
    ok, _ = W.taylor_green_box(40)
    ok2, _ = W.cavity(40, Re=100)
    b = dv.Batch([ok, ok2, ok], precision="f32")
    try:
        b.init_equilibrium(0, *W.taylor_green_box(40)[1])
        b.init_equilibrium(1, *W.cavity(40, Re=100)[1])
        nan = np.full((40, 40), np.nan)
        b.init_equilibrium(2, nan, nan, nan)
        b.step(10)
        assert b.case_status(0) == 0 and b.case_status(1) == 0
        assert b.case_status(2) == dv.DVBE_ERR_DIVERGED
        with dv.Solver(ok, precision="f32") as s:
            s.set_launch(strip_rows=32)
            s.init_equilibrium(*W.taylor_green_box(40)[1])
            s.step(10)
            b.set_launch(strip_rows=32)
            np.testing.assert_allclose(b.get_f(0), s.get_f(), rtol=0, atol=0)
    finally:
        b.close()


# ------------------------------------------------------------------ degenerate cases

@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_collisionless_limit(dv, scheme):
    """tau -> infinity (Omega -> 0): pure Lax-Wendroff advection."""
    case = periodic_case(40, 33, scheme, tau=1e30)
    g, o = run_pair(dv, case, 50, seed=12, amp_neq=1e-2)
    assert rel_err(g, o) < TOL64


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_large_dt_over_tau(dv, scheme):
    """dt/tau = 100 (the paper's largest Taylor-Green ratio), FP64 parity."""
    case = periodic_case(50, 41, scheme)
    case["tau"] = case["dt"] / 100.0
    g, o = run_pair(dv, case, 100, seed=13, amp_neq=1e-4)
    assert rel_err(g, o) < TOL64


def test_zero_steps_and_counts(dv):
    case, fields = W.taylor_green_box(32)
    with dv.Solver(case) as s:
        s.init_equilibrium(*fields)
        f0 = s.get_f()
        l0 = s.launch_count()
        s.step(0)
        assert s.launch_count() == l0 and s.step_count() == 0
        np.testing.assert_array_equal(s.get_f(), f0)


def test_cfl_above_one_blows_up(dv):
    """With the CFL check overridden (CFL 1.6), the scheme is unstable, as
    the paper reports for CFL > 1; the divergence flag reports it."""
    case, fields = W.taylor_green_box(64, u0=0.05, cfl=1.6)
    with dv.Solver(case, precision="f32", allow_cfl_ge_1=True) as s:
        s.init_equilibrium(*fields)
        with pytest.raises(dv.DvbeError) as e:
            for _ in range(200):
                s.step(50)
        assert e.value.status == dv.DVBE_ERR_DIVERGED
