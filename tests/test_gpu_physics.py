"""Physics runs on the GPU path, held to what the paper and the mathematics
fix: Table tab:tv_Nerr (Sec 3.1), steady-state cavities driven by the FP64
residual, the error of the reduced-precision storage modes against the FP64
path and against the analytic decay, and the flat-plate boundary layer
against the Blasius solution (Sec 3.3).  Results are printed for the record.
"""
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


def _golden():
    import pathlib
    rows = {}
    for line in (pathlib.Path(__file__).parent / "golden" / "table1_tv_nerr.txt").read_text().splitlines():
        if line.strip() and not line.startswith("#"):
            s, n, e = line.split()
            rows[(s, int(n))] = float(e)
    return rows


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_table1_on_gpu(dv, scheme):
    """Table tab:tv_Nerr at N = 16 .. 128 with the FP64 GPU path: E_u(t_c)
    against the printed values (the CPU oracle matches N = 16, 32 to 5e-4),
    second-order convergence, and DUGKS below BKG."""
    gold = _golden()
    errs = {}
    for n in (16, 32, 64, 128):
        case, fields, d, tc = W.taylor_green_paper(n, scheme)
        steps = int(round(tc / case["dt"]))
        with dv.Solver(case, precision="f64") as s:
            s.set_launch(strip_rows=4, warps_per_block=4, graph_chunk=1000)
            s.init_chapman_enskog(*fields, d)
            s.step(steps)
            ua, va = W.taylor_green_paper_analytic(case, steps * case["dt"])
            errs[n] = s.l2_error_u(ua, va)
        print(f"table1 {scheme} N={n} E_u={errs[n]:.5e} paper={gold[(scheme, n)]:.4e} "
              f"ratio={errs[n] / gold[(scheme, n)]:.4f}")
    for n in (16, 32):
        assert abs(errs[n] / gold[(scheme, n)] - 1) < 5e-4
    for n in (64, 128):
        assert abs(errs[n] / gold[(scheme, n)] - 1) < 0.1
    for a, b in ((16, 32), (32, 64), (64, 128)):
        assert 1.8 < math.log2(errs[a] / errs[b]) < 2.3


def test_time_step_sweep_n64(dv):
    """Sec 3.1, Fig. tv_dtErr: N = 64, tau fixed, dt/tau = 10 .. 50.  The error
    at t_c grows almost linearly with dt once the time error dominates, the
    DUGKS error stays below BKG's at every dt, and both schemes blow up at
    dt/tau = 100, where the CFL number (dt |xi|_max / dx = 1.57) exceeds 1."""
    errs = {}
    for scheme in ("dugks", "bkg"):
        for ratio in (10.0, 20.0, 50.0):
            case, fields, d, tc = W.taylor_green_paper(64, scheme, dt_over_tau=ratio)
            steps = int(round(tc / case["dt"]))
            with dv.Solver(case, precision="f64") as s:
                s.set_launch(strip_rows=16, warps_per_block=2, graph_chunk=1000)
                s.init_chapman_enskog(*fields, d)
                s.step(steps)
                errs[(scheme, ratio)] = s.l2_error_u(*W.taylor_green_paper_analytic(case, steps * case["dt"]))
            print(f"dt sweep {scheme} dt/tau={ratio:g}: E_u(t_c)={errs[(scheme, ratio)]:.4e}")
    for scheme in ("dugks", "bkg"):
        e = [errs[(scheme, r)] for r in (10.0, 20.0, 50.0)]
        assert all(a < b for a, b in zip(e, e[1:]))
        slope = math.log(e[2] / e[1]) / math.log(50.0 / 20.0)
        assert 0.7 < slope < 1.3, slope
    for ratio in (10.0, 20.0, 50.0):
        assert errs[("dugks", ratio)] < errs[("bkg", ratio)]
    for scheme in ("dugks", "bkg"):
        case, fields, d, tc = W.taylor_green_paper(64, scheme, dt_over_tau=100.0)
        cfl = case["dt"] * math.sqrt(6.0 * case["RT"]) / (1.0 / 64)
        assert cfl > 1.0
        with dv.Solver(case, precision="f64", allow_cfl_ge_1=True) as s:
            s.init_chapman_enskog(*fields, d)
            with pytest.raises(dv.DvbeError) as e:
                s.step(int(round(tc / case["dt"])))
            assert e.value.status == dv.DVBE_ERR_DIVERGED


def _decay_viscosity(case, u, v, t):
    """nu from the Taylor-Green amplitude: u = A(t) (mode shape), A = e^{-8 pi^2 nu t} A(0)."""
    us, vs = W.taylor_green_paper_analytic(case, 0.0)
    A = (np.sum(u * us) + np.sum(v * vs)) / (np.sum(us * us) + np.sum(vs * vs))
    return -math.log(A) / (8.0 * math.pi ** 2 * t)


def test_collision_free_faces_numerical_viscosity(dv):
    """Sec 2.4: dropping the collision integral from the face distribution
    (the upwind face of Eq. cfd2) adds a numerical viscosity proportional to
    dt.  Taylor-Green, paper set-up, N = 64, tau fixed, run to t_c / 4: the
    excess nu_eff / nu - 1 of the upwind collision-free face grows in
    proportion to dt/tau, while DUGKS stays within a few percent of nu.  The
    central face of Eq. cfd1 is reported."""
    ex = {}
    for scheme in ("cfree_upwind", "dugks", "cfree_central"):
        for ratio in (2.0, 4.0, 8.0):
            case, fields, d, tc = W.taylor_green_paper(64, scheme, dt_over_tau=ratio)
            steps = int(round(0.25 * tc / case["dt"]))
            with dv.Solver(case, precision="f64") as s:
                s.set_launch(strip_rows=16, warps_per_block=2, graph_chunk=2000)
                s.init_chapman_enskog(*fields, d)
                try:
                    s.step(steps)
                    _, u, v = s.moments()
                    ex[(scheme, ratio)] = _decay_viscosity(case, u, v, steps * case["dt"]) / case["nu"] - 1
                except dv.DvbeError:
                    ex[(scheme, ratio)] = float("nan")
            print(f"numerical viscosity {scheme} dt/tau={ratio:g}: nu_eff/nu - 1 = {ex[(scheme, ratio)]:.4f}")
    up = [ex[("cfree_upwind", r)] for r in (2.0, 4.0, 8.0)]
    assert up[0] > 0.4
    assert 1.6 < up[1] / up[0] < 2.4 and 3.2 < up[2] / up[0] < 4.8
    assert all(abs(ex[("dugks", r)]) < 0.05 for r in (2.0, 4.0, 8.0))


def test_dugks_more_accurate_than_bkg_at_n32(dv):
    """Sec 3.1: DUGKS errors below BKG's on the same mesh."""
    out = {}
    for scheme in ("dugks", "bkg"):
        case, fields, d, tc = W.taylor_green_paper(32, scheme)
        steps = int(round(tc / case["dt"]))
        with dv.Solver(case) as s:
            s.set_launch(strip_rows=4, graph_chunk=1000)
            s.init_chapman_enskog(*fields, d)
            s.step(steps)
            out[scheme] = s.l2_error_u(*W.taylor_green_paper_analytic(case, steps * case["dt"]))
    assert out["dugks"] < out["bkg"]


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_cavity_reaches_steady_state(dv, scheme):
    """Lid-driven cavity Re = 400 on 128^2 (FP64): the FP64 velocity residual
    between checks 1000 steps apart falls below 1e-7; mass is conserved up to
    FP64 rounding accumulated over the run (each step adds O(eps) per cell,
    about 1e-14 of the total, random-walking to ~1e-11 over 2.6e5 steps)."""
    case, fields = W.cavity(128, Re=400, scheme=scheme)
    with dv.Solver(case, precision="f64") as s:
        s.set_launch(strip_rows=8, graph_chunk=100)
        s.init_equilibrium(*fields)
        m0 = s.conserved()[0]
        s.residual()
        r, steps = math.inf, 0
        while r >= 1e-7 and steps < 400_000:
            s.step(1000)
            steps += 1000
            r = s.residual()
        m1 = s.conserved()[0]
        _, u, v = s.moments()
    print(f"cavity {scheme} Re400 128^2: R={r:.2e} after {steps} steps, mass drift {abs(m1 - m0) / m0:.1e}")
    assert r < 1e-7
    assert abs(m1 - m0) < 1e-10 * m0
    # primary vortex: u changes sign along the vertical centre line
    uc = u[:, 64]
    assert uc[-1] > 0 and uc.min() < -0.02


def _centerlines(u, v):
    """u on the vertical centre line and v on the horizontal one (cell-centre
    averages of the two columns / rows next to x = 0.5 / y = 0.5)."""
    n = u.shape[0]
    return 0.5 * (u[:, n // 2 - 1] + u[:, n // 2]), 0.5 * (v[n // 2 - 1, :] + v[n // 2, :])


def _coarsen(a):
    """Values of a 2n mesh at the n mesh's cell centres along a line (pairs averaged)."""
    return 0.5 * (a[0::2] + a[1::2])


def test_bkg_cfl_sweep_cavity_re5000(dv):
    """Sec 3.2, Fig. cavity_cfl: lid-driven cavity at Re = 5000 on 128^2.  The
    BKG centre-line errors decrease with the CFL number, and even at CFL 0.1
    they stay above those of DUGKS on the same mesh.  The paper measures
    against Ghia's data, which are not available here; the reference is DUGKS
    on 256^2.  All runs go to t = 100 L/U, FP32 deviation storage."""
    T = 1000.0

    def run(n, scheme, cfl):
        case, fields = W.cavity(n, Re=5000, cfl=cfl, scheme=scheme)
        with dv.Solver(case, precision="f32_dev") as s:
            s.set_launch(strip_rows=16, graph_chunk=1000)
            s.init_equilibrium(*fields)
            s.step(int(round(T / case["dt"])))
            s.residual()
            s.step(1000)
            r = s.residual()
            _, u, v = s.moments()
        return _centerlines(u, v), r

    (ur, vr), rr = run(256, "dugks", 0.5)
    ref = (_coarsen(ur), _coarsen(vr))

    def err(lines):
        return float(np.sqrt((np.sum((lines[0] - ref[0]) ** 2) + np.sum((lines[1] - ref[1]) ** 2))
                             / (np.sum(ref[0] ** 2) + np.sum(ref[1] ** 2))))

    errs = {}
    for cfl in (0.1, 0.3, 0.5, 0.7):
        lines, r = run(128, "bkg", cfl)
        errs[("bkg", cfl)] = err(lines)
        print(f"cavity Re5000 128^2 BKG CFL {cfl}: centre-line error vs DUGKS 256^2 = "
              f"{errs[('bkg', cfl)]:.3e} (residual {r:.1e})")
    lines, r = run(128, "dugks", 0.5)
    errs[("dugks", 0.5)] = err(lines)
    print(f"cavity Re5000 128^2 DUGKS CFL 0.5: {errs[('dugks', 0.5)]:.3e} (residual {r:.1e}; "
          f"reference residual {rr:.1e})")
    e = [errs[("bkg", c)] for c in (0.1, 0.3, 0.5, 0.7)]
    assert all(a < b for a, b in zip(e, e[1:]))
    assert errs[("dugks", 0.5)] < errs[("bkg", 0.1)]


def test_precision_modes_against_fp64_and_analytic(dv):
    """Taylor-Green 256^2, dt/tau = 10, to 10% decay (21k steps): error of
    each storage mode against the FP64 path (E_p) and of the FP64 path against
    the analytic solution (E_d).

    * FP32 deviation storage must keep E_p < 0.1 E_d (the accuracy bar for
      every reduced-precision result).
    * Absolute FP32 storage computes on deviations too, but stores f_tilde
      itself: each step rounds it by 2^-24 of f, about 2e-6 of the
      velocity-carrying part at u0 = 0.01.  That random-walks to ~3e-4 of u
      over the run, a few E_d: it is held to E_p < 10 E_d and reported.
    * The 16-bit modes cannot resolve the ~1e-7 per-step change of f here.
      They stagnate and are only reported."""
    case, fields = W.taylor_green_box(256, u0=0.01, cfl=0.5, dt_over_tau=10.0)
    steps = int(round(-math.log(0.9) / (2 * case["nu"]) / case["dt"]))
    ua, va = W.taylor_green_box_analytic(case, steps * case["dt"])
    res = {}
    for prec in ("f64", "f32", "f32_dev", "f16_dev", "bf16_dev"):
        with dv.Solver(case, precision=prec) as s:
            s.set_launch(strip_rows=8, graph_chunk=200)
            s.init_equilibrium(*fields)
            s.step(steps)
            res[prec] = s.moments()
    ed = np.sqrt(np.sum((res["f64"][1] - ua) ** 2 + (res["f64"][2] - va) ** 2) / np.sum(ua ** 2 + va ** 2))
    ratios = {}
    for prec in ("f32", "f32_dev", "f16_dev", "bf16_dev"):
        ep = np.sqrt(np.sum((res[prec][1] - res["f64"][1]) ** 2 + (res[prec][2] - res["f64"][2]) ** 2)
                     / np.sum(res["f64"][1] ** 2 + res["f64"][2] ** 2))
        ratios[prec] = ep / ed
        print(f"precision {prec}: E_p={ep:.3e} E_d={ed:.3e} E_p/E_d={ep / ed:.3e} ({steps} steps)")
        assert np.isfinite(ep)
    assert ratios["f32_dev"] < 0.1
    assert ratios["f32"] < 10.0
    assert ratios["f32_dev"] < ratios["f32"]


def test_flat_plate_against_blasius(dv):
    """Sec 3.3: laminar flat-plate boundary layer, Re_L = 1e5, stretched
    mesh.  At steady state the DUGKS u/U profile at x = 0.6 L follows
    Blasius (f' of the similarity solution) within 3% of U."""
    from oracle import blasius
    case, fields = W.flat_plate(nx_up=40, nx_plate=160, ny=96, dy_min=2e-4, dx_min=1e-3, scheme="dugks")
    U, nu = case["U"], case["nu"]
    with dv.Solver(case, precision="f32") as s:
        s.set_launch(strip_rows=4, graph_chunk=200)
        s.init_equilibrium(*fields)
        T = 2.5 * 1.5 / U  # 2.5 flow-through times of the domain
        s.step(int(T / case["dt"]))
        _, u, v = s.moments()
    xc, yc = W.centres(case["xf"]), W.centres(case["yf"])
    ix = int(np.argmin(np.abs(xc - 0.6)))
    ub, _ = blasius.profiles(yc, xc[ix], U, nu)
    inside = yc < 5.0 * math.sqrt(nu * xc[ix] / U) * 1.0
    err = np.max(np.abs(u[inside, ix] / U - ub[inside]))
    print(f"flat plate DUGKS x={xc[ix]:.3f}: max |u/U - f'| = {err:.3e} over {inside.sum()} cells")
    assert err < 0.03


def _plate_profile_error(case, u, X):
    """max |u/U - f'(eta)| for eta < 5 at x = X (linear interpolation between
    the two cell columns around X) against the Blasius solution."""
    from oracle import blasius
    xc, yc = W.centres(case["xf"]), W.centres(case["yf"])
    i = int(np.searchsorted(xc, X)) - 1
    a = (X - xc[i]) / (xc[i + 1] - xc[i])
    col = (1 - a) * u[:, i] + a * u[:, i + 1]
    U, nu = case["U"], case["nu"]
    ub, _ = blasius.profiles(yc, X, U, nu)
    inside = yc < 5.0 * math.sqrt(nu * X / U)
    return float(np.max(np.abs(col[inside] / U - ub[inside]))), int(inside.sum())


def test_flat_plate_paper_setup(dv):
    """Sec 3.3 with the paper's own mesh (U0 = 0.1, L = 94.76, Re = 1e5, y ratio
    1.1, 120 x 80 plate cells): u profiles at x = 6.4381 and 21.5082 against
    Blasius at t = 1000 (45 x / U at the second station), FP32 deviation
    storage; the error is max |u/U - f'| over both stations.  As the paper
    reports, DUGKS captures the layer on the three meshes (dy_min = 0.1,
    0.05, 0.02) while BKG stays further off on each,
    and a smaller BKG time step helps (CFL 0.5 -> 0.1 -> 0.02, dy_min = 0.1),
    at CFL 0.1 without reaching DUGKS.  Unlike the paper's report for CFL
    0.01, BKG at CFL 0.02 comes within DUGKS's error (0.036 against 0.076 for
    DUGKS at CFL 0.5 on this mesh), as its error scales with dt; that is
    reported, not asserted.  (With zero-gradient
    outflow, acoustic waves reflected at the top outflow corner grow at small
    dt/tau: BKG at CFL 0.03 and 0.02 (dt/tau 7.5 and 5) and DUGKS at CFL 0.02
    diverge before t = 1000, in FP64 as in FP32.  The CFL 0.02 BKG run
    therefore uses the set-density outflow, which stays bounded.)"""
    X = (6.4381, 21.5082)

    def run(dy, scheme, cfl, outflow="outflow"):
        case, fields = W.flat_plate_paper(dy, cfl=cfl, scheme=scheme, outflow=outflow)
        with dv.Solver(case, precision="f32_dev") as s:
            s.set_launch(strip_rows=8, graph_chunk=2000)
            s.init_equilibrium(*fields)
            s.step(int(round(1000.0 / case["dt"])))
            _, u, v = s.moments()
        assert np.max(np.hypot(u, v)) < 1.5 * case["U"]  # bounded: no growing reflections
        errs = [_plate_profile_error(case, u, x) for x in X]
        print(f"flat plate (paper) {scheme} dy_min={dy} CFL={cfl} {case['nx']}x{case['ny']}: "
              + ", ".join(f"x={x}: max|u/U-f'|={e:.3e} ({n} cells in eta<5)" for x, (e, n) in zip(X, errs)))
        return max(e for e, _ in errs)

    err = {}
    for dy in (0.1, 0.05, 0.02):
        for scheme in ("dugks", "bkg"):
            err[(scheme, dy, 0.5)] = run(dy, scheme, 0.5)
    err[("bkg", 0.1, 0.1)] = run(0.1, "bkg", 0.1)
    # the set-density outflow keeps the CFL 0.02 run bounded (see above)
    err[("bkg", 0.1, 0.02)] = run(0.1, "bkg", 0.02, outflow="outflow_neq")
    # DUGKS: within 3% of U where the layer holds 6 or more cells at the first
    # station, within 10% on the coarsest mesh (3 cells across eta < 5 there)
    assert err[("dugks", 0.05, 0.5)] < 0.03 and err[("dugks", 0.02, 0.5)] < 0.03
    assert err[("dugks", 0.1, 0.5)] < 0.1
    for dy in (0.1, 0.05, 0.02):
        assert err[("bkg", dy, 0.5)] > err[("dugks", dy, 0.5)]
    assert err[("bkg", 0.1, 0.1)] < err[("bkg", 0.1, 0.5)]
    assert err[("bkg", 0.1, 0.1)] > err[("dugks", 0.1, 0.5)]
    assert err[("bkg", 0.1, 0.02)] < err[("bkg", 0.1, 0.1)]
