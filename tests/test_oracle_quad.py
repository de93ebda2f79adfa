"""Pins of the oracle's curvilinear (general quadrilateral) mesh step.

The paper states the FV form for general cells V_k with faces of any
orientation (Sec 2.2) but writes the reconstruction only on uniform meshes
(Sec 2.4), so the quad step is a reading: the normal slope from the two
cells of a face, the tangential slope from their gradients, ghost cells
mirrored across the boundary face (parity unpinned by the paper).  What the
mathematics fixes, and these tests check:

  - on a tensor mesh given as vertices the step is the tensor oracle's, and
    so is it with the index directions turned (i along +y, j along -x);
  - data that depend on y alone, on a mesh sheared along x, step exactly as
    on the unsheared mesh (the face slopes split along the face normal);
  - a uniform equilibrium stays put on any closed mesh (the face normals
    times areas of a cell sum to zero: free-stream preservation);
  - with collisions off, linear data advect exactly: one step moves every
    cell value by -dt xi . grad f (cells two or more from the boundary);
  - mass and momentum are conserved on a doubly periodic distorted mesh,
    mass in a closed distorted cavity with walls;
  - collisionless advection of a smooth wave on a smoothly distorted mesh
    converges at second order.
A set of planted mistakes, each caught by at least one of these pins, closes
the file.
"""
import math
import pathlib
import shutil
import subprocess

import numpy as np
import pytest

import oracle as O
import workloads as W

RT = W.RT_LATTICE
INF = 1e300
PER = W.periodic_bc()


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


def qcase(X, Y, scheme, tau, recon="linear", bc=PER, cfl=0.4):
    ny, nx = X.shape[0] - 1, X.shape[1] - 1
    c = dict(nx=nx, ny=ny, X=X, Y=Y, RT=RT, tau=tau, dt=1.0, scheme=scheme, recon=recon, bc=bc)
    c["dt"] = O.quad_dt_from_cfl(c, cfl)
    return c


def _tensor_cases():
    """Tensor problems with every kind of side, stretched and uniform."""
    cav, _ = W.cavity(14, Re=100, scheme="dugks", stretch_beta=1.3)
    box = W.cavity_four_lids(13, 9, scheme="bkg", kind="diffuse")
    plate, _ = W.flat_plate(nx_up=5, nx_plate=11, ny=12, scheme="dugks", Re_L=2e3)
    tg = dict(W.taylor_green_box(12, scheme="bkg")[0])
    tg["xf"] = W.tanh_faces(12, 0.0, 2 * math.pi, 0.8)
    tg["dt"] = W.cfl_dt(tg["xf"], tg["yf"], 0.5)
    fs = W.free_stream_channel(14, scheme="dugks")
    return {"cavity": cav, "four_lids": box, "plate": plate, "tg_stretched": tg, "free_stream": fs}


TENSOR = _tensor_cases()
SCHEME_RECON = [("dugks", "linear"), ("dugks", "upwind_cell"), ("bkg", "linear"),
                ("bkg", "upwind_cell"), ("cfree_upwind", "linear"), ("cfree_central", "linear")]


def _state(case, seed):
    (r, u, v), d = W.random_state(case, seed, amp_neq=1e-3)
    return O.init_equilibrium(case, r, u, v) + d


@pytest.mark.parametrize("name", sorted(TENSOR))
@pytest.mark.parametrize("scheme,recon", SCHEME_RECON)
def test_quad_step_reduces_to_the_tensor_oracle(name, scheme, recon):
    case = dict(TENSOR[name], scheme=scheme, recon=recon)
    f0 = _state(case, 5)
    assert rel(O.quad_step(W.quad_from_faces(case), f0, 5), O.step(case, f0, 5)) < 1e-13


def _single_segment_cases():
    cav, _ = W.cavity(12, Re=100, scheme="dugks", stretch_beta=1.2)
    sym = dict(cav, bc=[[W.wall()], [("outflow", -INF, INF, 1.0, 0.0, 0.0)],
                        [("symmetry", -INF, INF, 1.0, 0.0, 0.0)], [W.wall(ux=0.05)]])
    return [cav, sym, W.cavity_four_lids(11, 9, scheme="bkg"),
            W.cavity_four_lids(11, 9, scheme="dugks", kind="diffuse")]


@pytest.mark.parametrize("k", range(4))
@pytest.mark.parametrize("recon", ["linear", "upwind_cell"])
def test_turned_index_directions_give_the_same_step(k, recon):
    """The mesh of a tensor problem with quad index i along +y and j along
    -x: x-faces of the quad are horizontal, its y-faces vertical."""
    case = dict(_single_segment_cases()[k], recon=recon)
    f0 = _state(case, 6)
    q, to_quad, from_quad = W.quad_reindexed(case)
    assert rel(from_quad(O.quad_step(q, to_quad(f0), 6)), O.step(case, f0, 6)) < 1e-13


@pytest.mark.parametrize("kind", ["wall", "diffuse"])
@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
@pytest.mark.parametrize("recon", ["linear", "upwind_cell"])
def test_sheared_mesh_steps_y_only_data_as_the_tensor_mesh(kind, scheme, recon):
    c, _ = W.couette(8, 20, U=0.05, nu=0.02, scheme=scheme, kind=kind)
    c = dict(c, recon=recon)
    ny, nx = c["ny"], c["nx"]
    rng = np.random.default_rng(4)

    def prof(amp):
        return np.repeat(amp * rng.standard_normal((ny, 1)), nx, axis=1)
    f0 = O.init_equilibrium(c, 1 + prof(0.01), prof(0.02), prof(0.01))
    f0 = f0 + np.repeat(1e-3 * rng.standard_normal((9, ny, 1)), nx, axis=2)
    ref = O.step(c, f0, 8)
    for s in (0.4, -1.1):
        assert rel(O.quad_step(W.quad_sheared(c, s), f0, 8), ref) < 1e-14


@pytest.mark.parametrize("scheme", ["dugks", "bkg", "cfree_upwind", "cfree_central"])
def test_uniform_flow_is_kept_on_a_distorted_periodic_mesh(scheme):
    X, Y = W.quad_wavy_periodic(16, L=1.0, amp=0.06)
    c = qcase(X, Y, scheme, 0.02)
    f0 = O.quad_init_equilibrium(c, np.full((16, 16), 1.01), np.full((16, 16), 0.03),
                                 np.full((16, 16), -0.02))
    assert np.max(np.abs(O.quad_step(c, f0, 20) - f0)) < 2e-15


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
@pytest.mark.parametrize("recon", ["linear", "upwind_cell"])
def test_free_stream_sides_keep_a_uniform_flow_on_a_random_mesh(scheme, recon):
    X, Y = W.quad_random_interior(14, 11, 3, amp=0.3)
    inf = [("inflow", -INF, INF, 1.01, 0.03, -0.02)]
    c = qcase(X, Y, scheme, 0.02, recon=recon, bc=[inf] * 4)
    f0 = O.quad_init_equilibrium(c, np.full((11, 14), 1.01), np.full((11, 14), 0.03),
                                 np.full((11, 14), -0.02))
    assert np.max(np.abs(O.quad_step(c, f0, 20) - f0)) < 2e-15


@pytest.mark.parametrize("scheme,recon", SCHEME_RECON)
def test_linear_fields_advect_exactly_on_a_random_quad_mesh(scheme, recon):
    X, Y = W.quad_random_interior(12, 12, 9, amp=0.3)
    out = [("outflow", -INF, INF, 1.0, 0.0, 0.0)]
    c = qcase(X, Y, scheme, 1e300, recon=recon, bc=[out] * 4)
    xi, w, _ = O.d2q9(RT)
    xc, yc, _ = O.quad_geometry(c)
    gx, gy = 0.7e-2, 1.3e-2
    f0 = np.array([w[a] * (1 + gx * xc + gy * yc) for a in range(9)])
    f1 = O.quad_step(c, f0, 1)
    dt = c["dt"]
    ex = np.array([w[a] * (1 + gx * (xc - xi[a, 0] * dt) + gy * (yc - xi[a, 1] * dt)) for a in range(9)])
    inner = (slice(None), slice(2, 10), slice(2, 10))
    assert np.max(np.abs(f1[inner] - ex[inner])) < 2e-16


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
@pytest.mark.parametrize("recon", ["linear", "upwind_cell"])
def test_conservation_on_a_distorted_periodic_mesh(scheme, recon):
    X, Y = W.quad_wavy_periodic(16, L=1.0, amp=0.06)
    c = qcase(X, Y, scheme, 0.01, recon=recon)
    rng = np.random.default_rng(3)
    r = 1 + 0.01 * rng.standard_normal((16, 16))
    u, v = 0.02 * rng.standard_normal((2, 16, 16))
    f0 = O.quad_init_equilibrium(c, r, u, v) + 1e-3 * rng.standard_normal((9, 16, 16))
    c0, c1 = O.quad_conserved(c, f0), O.quad_conserved(c, O.quad_step(c, f0, 40))
    assert np.max(np.abs(c1 - c0)) < 1e-14 * c0[0]


@pytest.mark.parametrize("kind", ["wall", "diffuse"])
@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_closed_distorted_cavity_conserves_mass(kind, scheme):
    X, Y = W.quad_random_interior(12, 10, 5, amp=0.3)
    c = qcase(X, Y, scheme, 0.01, bc=[[(kind, -INF, INF, 1.0, 0.0, 0.0)]] * 4)
    rng = np.random.default_rng(3)
    r = 1 + 0.01 * rng.standard_normal((10, 12))
    u, v = 0.02 * rng.standard_normal((2, 10, 12))
    f0 = O.quad_init_equilibrium(c, r, u, v)
    c0, c1 = O.quad_conserved(c, f0), O.quad_conserved(c, O.quad_step(c, f0, 40))
    assert abs(c1[0] - c0[0]) < 1e-14 * c0[0]


def _wave_errors(recon, sizes=(32, 64)):
    xi, w, _ = O.d2q9(RT)
    errs = []
    for n in sizes:
        X, Y = W.quad_wavy_periodic(n, L=1.0, amp=0.04)
        c = qcase(X, Y, "dugks", 1e30, recon=recon)
        xc, yc, _ = O.quad_geometry(c)
        steps = int(round(0.25 / c["dt"]))
        T = steps * c["dt"]
        f0 = np.array([w[a] * (1 + 0.01 * np.sin(2 * np.pi * (xc + 2 * yc))) for a in range(9)])
        ex = np.array([w[a] * (1 + 0.01 * np.sin(2 * np.pi * ((xc - xi[a, 0] * T) + 2 * (yc - xi[a, 1] * T))))
                       for a in range(9)])
        errs.append(float(np.sqrt(np.mean((O.quad_step(c, f0, steps) - ex) ** 2))))
    return errs


@pytest.mark.parametrize("recon", ["linear", "upwind_cell"])
def test_collisionless_advection_on_a_wavy_mesh_is_second_order(recon):
    e = _wave_errors(recon)
    lo, hi = (3.5, 4.5) if recon == "linear" else (3.5, 6.0)
    assert lo < e[0] / e[1] < hi, e


def test_quad_problem_checks():
    X, Y = W.quad_random_interior(6, 5, 1, amp=0.2)
    wl = [W.wall()]
    c = qcase(X, Y, "dugks", 0.01, bc=[wl] * 4)
    O.quad_geometry(c)
    Xb = X.copy()
    Xb[2, 3] = Xb[2, 1] - 0.05  # folds a cell over
    with pytest.raises(O.OracleError):
        O.quad_geometry(dict(c, X=Xb))
    sym = [("symmetry", -INF, INF, 1.0, 0.0, 0.0)]
    cs = W.quad_sheared(dict(W.cavity(6, Re=100)[0], bc=[sym, sym, wl, wl]), 0.3)
    with pytest.raises(O.OracleError):  # symmetry on a slanted side
        O.quad_geometry(cs)
    O.quad_geometry(dict(cs, bc=[wl, wl, sym, sym]))  # horizontal sides may be symmetric
    with pytest.raises(O.OracleError):  # periodic on one side only
        O.quad_geometry(dict(c, bc=[PER[0], wl, wl, wl]))


# ---------------------------------------------------------------- mutations

QMUTATIONS = {
    # face value without the offset of the face midpoint from the centre line
    "offset_term": ("const double pb = (1.0 - th) * Pa[L] + th * Pa[R] + gbx * ox + gby * oy;",
                    "const double pb = (1.0 - th) * Pa[L] + th * Pa[R];"),
    # face-gradient correction along d instead of the face normal
    "corr_along_d": ("const double gfx = gbx + corr * nx_, gfy = gby + corr * ny_;",
                     "const double gfx = gbx + corr * dx / (dx * dx + dy * dy) * dn,"
                     " gfy = gby + corr * dy / (dx * dx + dy * dy) * dn;"),
    # transposed inverse Jacobian of the cell gradient
    "grad_transposed": ("*gx = (pi * yj_ - yi_ * pj) / det;", "*gx = (pi * yj_ - xj_ * pj) / det;"),
    # the y-face normal turned the other way
    "yface_normal": ("g->ynx[f] = -ty / len;\n      g->yny[f] = tx / len;",
                     "g->ynx[f] = ty / len;\n      g->yny[f] = -tx / len;"),
    # face area taken as one
    "face_area": ("g->xA[f] = len;", "g->xA[f] = 1.0;"),
    # ghost centre continued along the mesh line instead of mirrored
    "ghost_centre": ("mirror(g->cx[QIDX(g, i1, j)], g->cy[QIDX(g, i1, j)], g->xbx[f], g->xby[f], g->xnx[f], g->xny[f],\n"
                     "               &g->cx[QIDX(g, ig, j)], &g->cy[QIDX(g, ig, j)]);",
                     "g->cx[QIDX(g, ig, j)] = 2.0 * g->cx[QIDX(g, i1, j)] - g->cx[QIDX(g, side ? nx - 2 : 1, j)];\n"
                     "        g->cy[QIDX(g, ig, j)] = 2.0 * g->cy[QIDX(g, i1, j)] - g->cy[QIDX(g, side ? nx - 2 : 1, j)];"),
    # wall extrapolation along the mesh line instead of the wall normal
    "ext_along_line": ("return ((g->cx[cg] - g->cx[c1]) * nx_ + (g->cy[cg] - g->cy[c1]) * ny_) / (dx * nx_ + dy * ny_);",
                       "return ((g->cx[cg] - g->cx[c1]) * dx + (g->cy[cg] - g->cy[c1]) * dy) / (dx * dx + dy * dy);"),
    # periodic image of the centres shifted the wrong way
    "periodic_image": ("g->cx[QIDX(g, -l, j)] = g->cx[QIDX(g, nx - l, j)] - g->Px[0];",
                       "g->cx[QIDX(g, -l, j)] = g->cx[QIDX(g, nx - l, j)] + g->Px[0];"),
    # upwind-cell value from the downwind cell
    "upwind_side": ("const int iC = xn > 0.0 ? iL : iR, jC = xn > 0.0 ? jL : jR;",
                    "const int iC = xn > 0.0 ? iR : iL, jC = xn > 0.0 ? jR : jL;"),
}

QTARGETED = {"corr_along_d": "shear", "offset_term": "linear_exact", "grad_transposed": "linear_exact",
             "periodic_image": "order"}


def _qmutant(tmp_path, name):
    here = pathlib.Path(O.__file__).parent
    src = (here / "dvbe_oracle.c").read_text()
    old, new = QMUTATIONS[name]
    assert src.count(old) == 1, name
    d = tmp_path / name
    d.mkdir()
    shutil.copy(here / "dvbe_oracle.h", d)
    (d / "dvbe_oracle.c").write_text(src.replace(old, new))
    so = d / "lib.so"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", str(so), str(d / "dvbe_oracle.c"), "-lm"])
    return str(so)


def _qpins_with(so_path):
    saved = O._lib
    O._lib = None
    real_build = O.build
    O.build = lambda force=False: so_path
    failed = []
    try:
        O.lib()
        checks = {
            "reduce_cavity": lambda: test_quad_step_reduces_to_the_tensor_oracle("cavity", "dugks", "linear"),
            "reduce_tg": lambda: test_quad_step_reduces_to_the_tensor_oracle("tg_stretched", "bkg", "linear"),
            "reduce_upwind": lambda: test_quad_step_reduces_to_the_tensor_oracle("tg_stretched", "dugks",
                                                                                 "upwind_cell"),
            "turned": lambda: test_turned_index_directions_give_the_same_step(1, "linear"),
            "shear": lambda: test_sheared_mesh_steps_y_only_data_as_the_tensor_mesh("wall", "dugks", "linear"),
            "uniform": lambda: test_uniform_flow_is_kept_on_a_distorted_periodic_mesh("dugks"),
            "linear_exact": lambda: test_linear_fields_advect_exactly_on_a_random_quad_mesh("dugks", "linear"),
            "order": lambda: test_collisionless_advection_on_a_wavy_mesh_is_second_order("linear"),
        }
        for k, fn in checks.items():
            try:
                fn()
            except (AssertionError, O.OracleError):
                failed.append(k)
    finally:
        O.build = real_build
        O._lib = saved
    return failed


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(QMUTATIONS))
def test_planted_quad_mistakes_are_caught(tmp_path, name):
    failed = _qpins_with(_qmutant(tmp_path, name))
    assert failed, f"mutation {name} passed every pin"
    if name in QTARGETED:
        assert QTARGETED[name] in failed, (name, failed)


@pytest.mark.parametrize("RTv", [0.2, 0.7])
def test_quad_step_reduces_to_the_tensor_oracle_at_other_RT(RTv):
    """The same reduction with the lattice speed c = sqrt(3 RT) away from 1:
    walls with a moving lid, a free stream and a symmetry side."""
    for name in ("cavity", "plate"):
        case = dict(TENSOR[name], RT=RTv, recon="linear")
        case["dt"] = W.cfl_dt(case["xf"], case["yf"], 0.5, RT=RTv)
        f0 = _state(case, 8)
        assert rel(O.quad_step(W.quad_from_faces(case), f0, 5), O.step(case, f0, 5)) < 1e-13, name
