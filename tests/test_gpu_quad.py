"""Curvilinear (quadrilateral-cell) meshes on the GPU: the multi-pass FP64
step of dvbe_mesh_create_quad meshes against the oracle's quad step
(Sec 2.2 finite volumes on cells of any shape).

Parity: relative 1e-12 after 30 steps on randomly distorted, wavy periodic
and sheared meshes with every kind of side (moving and diffuse walls, free
stream, zero-gradient and set-density outflow, symmetry, periodic), DUGKS,
BKG and the collision-free faces, linear and upwind-cell reconstructions;
the FP64 mass / momentum sums with the cells' own volumes; FP32 storage and
arithmetic to 1e-5 of max |f_tilde| on the same meshes; a tensor mesh
given as vertices against the tensor multi-pass step; and the rejections
(deviation storage modes, batches, slanted symmetry sides, periodic sides
that are not translates)."""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

RT = W.RT_LATTICE
INF = 1e300


@pytest.fixture(scope="module")
def dv():
    from paper_1511_00242_gb300 import build
    build.build()
    import paper_1511_00242_gb300 as dv
    return dv


def qcase(X, Y, scheme, tau, bc, recon="linear", cfl=0.45):
    ny, nx = X.shape[0] - 1, X.shape[1] - 1
    c = dict(nx=nx, ny=ny, X=X, Y=Y, RT=RT, tau=tau, dt=1.0, scheme=scheme, recon=recon, bc=bc)
    c["dt"] = O.quad_dt_from_cfl(c, cfl)
    return c


def seg(kind, rho=1.0, ux=0.0, uy=0.0):
    return [(kind, -INF, INF, rho, ux, uy)]


def _meshes():
    """(name, X, Y, bc) with the sides each mesh allows."""
    out = []
    X, Y = W.quad_random_interior(41, 33, 11, amp=0.3)
    out.append(("random cavity, moving lid", X, Y,
                [seg("wall"), seg("wall"), seg("wall"), seg("wall", ux=0.05)]))
    out.append(("random cavity, diffuse walls", X, Y,
                [seg("diffuse"), seg("diffuse", uy=0.03), seg("diffuse"), seg("diffuse", ux=0.05)]))
    X2, Y2 = W.quad_random_interior(37, 29, 12, amp=0.3, L=(2.0, 1.0))
    out.append(("random channel: free stream, outflows, symmetry", X2, Y2,
                [seg("inflow", 1.0, 0.05, 0.0), seg("outflow_neq", 1.0), seg("symmetry"), seg("outflow")]))
    Xw, Yw = W.quad_wavy_periodic(40, L=2 * math.pi, amp=0.05)
    out.append(("wavy periodic box", Xw, Yw, W.periodic_bc()))
    cou, _ = W.couette(24, 30, U=0.05, nu=0.02, scheme="dugks", kind="wall")
    q = W.quad_sheared(cou, 0.6)
    out.append(("sheared Couette", q["X"], q["Y"], cou["bc"]))
    return out


MESHES = _meshes()
SCHEMES = [("dugks", "linear"), ("dugks", "upwind_cell"), ("bkg", "linear"), ("bkg", "upwind_cell"),
           ("cfree_upwind", "linear"), ("cfree_central", "linear")]


def _random_f(case, seed):
    rng = np.random.default_rng(seed)
    ny, nx = case["ny"], case["nx"]
    r = 1 + 0.01 * rng.standard_normal((ny, nx))
    u, v = 0.02 * rng.standard_normal((2, ny, nx))
    return O.quad_init_equilibrium(case, r, u, v) + 1e-3 * rng.standard_normal((9, ny, nx)) / 9


@pytest.mark.parametrize("k", range(len(MESHES)))
@pytest.mark.parametrize("scheme,recon", SCHEMES)
def test_quad_step_matches_the_oracle(dv, k, scheme, recon):
    name, X, Y, bc = MESHES[k]
    case = qcase(X, Y, scheme, 0.02, bc, recon=recon)
    f0 = _random_f(case, 100 + k)
    o = O.quad_step(case, f0, 30)
    with dv.Solver(case, precision="f64") as s:
        s.init_f(f0)
        l0 = s.launch_count()
        s.step(30)
        assert s.launch_count() - l0 == 30 * 6
        g = s.get_f()
        sums = s.conserved()
    assert float(np.max(np.abs(g - o) / np.abs(o))) < 1e-12, name
    np.testing.assert_allclose(sums, O.quad_conserved(case, o), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_tensor_mesh_as_vertices_matches_the_tensor_step(dv, scheme):
    case, _ = W.cavity(45, Re=200, scheme=scheme, stretch_beta=1.3)
    (r, u, v), d = W.random_state(case, 3, amp_neq=1e-3)
    with dv.Solver(case, precision="f64", path="multipass") as s:
        s.init_equilibrium(r, u, v)
        f0 = s.get_f() + d
        s.init_f(f0)
        s.step(25)
        ref = s.get_f()
    with dv.Solver(W.quad_from_faces(case), precision="f64") as s:
        s.init_f(f0)
        s.step(25)
        g = s.get_f()
    assert float(np.max(np.abs(g - ref) / np.abs(ref))) < 1e-13


@pytest.mark.parametrize("k", range(len(MESHES)))
@pytest.mark.parametrize("scheme,recon", [("dugks", "linear"), ("dugks", "upwind_cell"),
                                          ("bkg", "linear"), ("cfree_upwind", "linear")])
def test_quad_step_fp32_matches_the_oracle(dv, k, scheme, recon):
    """FP32 storage and arithmetic on the same meshes: 30 steps of FP32
    rounding, within 1e-5 of max |f_tilde| of the FP64 oracle; the FP64 sums
    of the FP32 state within 1e-6."""
    name, X, Y, bc = MESHES[k]
    case = qcase(X, Y, scheme, 0.02, bc, recon=recon)
    f0 = _random_f(case, 200 + k)
    o = O.quad_step(case, f0, 30)
    with dv.Solver(case, precision="f32") as s:
        s.init_f(f0)
        s.step(30)
        g = s.get_f()
        sums = s.conserved()
    err = float(np.max(np.abs(g - o)) / np.max(np.abs(o)))
    assert err < 1e-5, (name, err)
    np.testing.assert_allclose(sums, O.quad_conserved(case, o), rtol=1e-6, atol=1e-6 * abs(sums[0]))


def test_quad_mesh_rejections(dv):
    name, X, Y, bc = MESHES[0]
    case = qcase(X, Y, "dugks", 0.02, bc)
    for prec in ("f32_dev", "f16_dev", "bf16_dev"):
        with pytest.raises(dv.DvbeError) as e:
            dv.Solver(case, precision=prec)
        assert e.value.status == dv.DVBE_ERR_UNSUPPORTED
    with pytest.raises(dv.DvbeError) as e:
        dv.Batch([case], precision="f64")
    assert e.value.status == dv.DVBE_ERR_UNSUPPORTED
    cou, _ = W.couette(12, 10, scheme="dugks", kind="wall")
    sym = seg("symmetry")
    sheared = W.quad_sheared(dict(cou, bc=[sym, sym, cou["bc"][2], cou["bc"][3]]), 0.5)
    with pytest.raises(dv.DvbeError) as e:  # symmetry on slanted sides
        dv.Solver(sheared, precision="f64")
    assert e.value.status == dv.DVBE_ERR_INVALID_ARG
    Xb = np.array(MESHES[3][1])
    Xb[:, -1] += np.linspace(0, 0.1, Xb.shape[0])  # E side no longer a translate of W
    with pytest.raises(dv.DvbeError) as e:
        dv.Solver(dict(qcase(Xb, MESHES[3][2], "bkg", 0.02, W.periodic_bc())), precision="f64")
    assert e.value.status == dv.DVBE_ERR_INVALID_ARG


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_taylor_green_decay_on_a_wavy_mesh(dv, scheme, precision):
    """The Taylor-Green vortex on the wavy periodic 64^2 mesh decays at
    nu = tau RT (Sec 3.1, Eq. nu_tau) to 1%, fitted between t = 2 and 6 as on
    the tensor mesh, and its velocity stays within 1% of the analytic field,
    in FP64 and in FP32 storage and arithmetic."""
    case, (r, u, v) = W.taylor_green_quad(64, amp=0.05, cfl=0.5, dt_over_tau=0.5, scheme=scheme)
    X, Y = case["X"], case["Y"]
    x = 0.25 * (X[:-1, :-1] + X[:-1, 1:] + X[1:, 1:] + X[1:, :-1])
    y = 0.25 * (Y[:-1, :-1] + Y[:-1, 1:] + Y[1:, 1:] + Y[1:, :-1])
    ua0, va0 = -case["u0"] * np.cos(x) * np.sin(y), case["u0"] * np.sin(x) * np.cos(y)
    amps, times = [], []
    with dv.Solver(case, precision=precision) as s:
        s.set_launch(graph_chunk=200)
        s.init_equilibrium(r, u, v)
        done = 0
        for t in (2.0, 6.0):
            n = int(round(t / case["dt"]))
            s.step(n - done)
            done = n
            _, uu, vv = s.moments()
            amps.append((np.sum(uu * ua0) + np.sum(vv * va0)) / (np.sum(ua0 ** 2) + np.sum(va0 ** 2)))
            times.append(n * case["dt"])
    nu_fit = math.log(amps[0] / amps[1]) / (2 * (times[1] - times[0]))
    print(f"wavy quad 64^2 {scheme} {precision}: nu_fit / nu - 1 = {nu_fit / case['nu'] - 1:.4f}")
    assert abs(nu_fit / case["nu"] - 1) < 0.01
    d = math.exp(-2 * case["nu"] * times[1])
    err = np.sqrt(np.sum((uu - ua0 * d) ** 2 + (vv - va0 * d) ** 2) / np.sum((ua0 * d) ** 2 + (va0 * d) ** 2))
    assert err < 0.01, err
