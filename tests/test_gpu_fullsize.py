"""Parity at full size, in the launch configuration bench.py times.

The oracle cannot run a 4096^2 mesh in reasonable time, but one cell's update
depends only on its 3 x 3 neighbourhood.  So for sampled cells the oracle
steps a 5 x 5 periodic window cut from the GPU's own input state around the
cell; the window's centre is then exactly the oracle's value for that cell.
Samples include strip and row-strip boundaries and the domain edges (where
the periodic wrap of the window is the periodic wrap of the mesh).
"""
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


def window_expect(case, f, cells, periodic=True):
    """Oracle value after one step for each (i, j) in cells, from the 5 x 5
    window of f around it (periodic window; the centre only sees its 3 x 3
    neighbourhood)."""
    ny, nx = f.shape[1:]
    xf, yf = np.asarray(case["xf"]), np.asarray(case["yf"])
    out = []
    per = [("periodic", -W.INF, W.INF, 0.0, 0.0, 0.0)]
    for i, j in cells:
        ix = [(i + d) % nx for d in range(-2, 3)]
        iy = [(j + d) % ny for d in range(-2, 3)]
        fw = f[:, iy][:, :, ix]
        # local face coordinates of the window (mesh spacing carried over)
        dx = np.array([xf[k + 1] - xf[k] for k in ix])
        dy = np.array([yf[k + 1] - yf[k] for k in iy])
        wcase = dict(case, nx=5, ny=5, xf=np.concatenate([[0.0], np.cumsum(dx)]),
                     yf=np.concatenate([[0.0], np.cumsum(dy)]), bc=[per, per, per, per])
        out.append(O.step(wcase, fw, 1)[:, 2, 2])
    return np.array(out)


def sample_cells(nx, ny, H, n_random=48, seed=0, margin=0):
    rng = np.random.default_rng(seed)
    cells = set()
    for i in (margin, 29 + margin, 30, 31, 59, 60, nx // 2, nx - 1 - margin):
        for j in (margin, H - 1, H, H + 1, ny // 2, ny - 1 - margin):
            cells.add((i, j))
    for _ in range(n_random):
        cells.add((int(rng.integers(margin, nx - margin)), int(rng.integers(margin, ny - margin))))
    return sorted(cells)


def one_step_sampled(dv, case, fields, precision, launch, cells):
    """Developed state f0 (3 steps from fields), one more step; returns f0,
    the stepped values at cells (or the whole array if cells is empty) and
    the launch shape used ("autotune": what bench.py's autotuner picks)."""
    with dv.Solver(case, precision=precision) as s:
        s.init_equilibrium(*fields)
        if launch == "autotune":
            s.autotune(3)
        else:
            s.set_launch(**launch)
        s.step(3)
        f0 = s.get_f()
        s.step(1)
        f1 = s.get_f()
        used = s.get_launch()
    if not cells:
        return f0, f1, used
    return f0, np.array([f1[:, j, i] for i, j in cells]), used


@pytest.mark.parametrize("precision", ["f32", "f32_dev"])
@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_taylor_green_4096_fp32_bench_launch(dv, scheme, precision):
    """The bench workload (4096^2, FP32 arithmetic; FP32 deviation storage is
    the timed one) in the launch shape its autotuner picks, on the rows with
    halo columns the periodic mesh gets; FP32 against FP64 from the same
    input: one step's rounding, relative 2e-6 of f_tilde.  The sampled cells
    include the strip seams, the narrow last strip and both wrap columns."""
    case, fields = W.taylor_green_box(4096, u0=0.01, cfl=0.5, scheme=scheme, dt_over_tau=10.0)
    f0, got, used = one_step_sampled(dv, case, fields, precision, "autotune", [])
    cells = sample_cells(4096, 4096, used["strip_rows"])
    got = np.array([got[:, j, i] for i, j in cells])
    exp = window_expect(case, f0, cells)
    err = np.max(np.abs(got - exp) / np.abs(exp))
    assert err < 2e-6, err


def test_taylor_green_4096_fp64(dv):
    """FP64 parity at full size: relative 1e-13 after one step."""
    case, fields = W.taylor_green_box(4096, u0=0.01, cfl=0.5, scheme="dugks", dt_over_tau=10.0)
    cells = sample_cells(4096, 4096, 32, n_random=24)
    f0, got, used = one_step_sampled(dv, case, fields, "f64", dict(strip_rows=32, warps_per_block=2),
                                     cells)
    exp = window_expect(case, f0, cells)
    assert np.max(np.abs(got - exp) / np.abs(exp)) < 1e-13


@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_cavity_2048_interior(dv, scheme):
    """Cavity 2048^2, Re 5000, FP32: sampled interior cells (the window must
    not cross the walls), relative 2e-6."""
    case, fields = W.cavity(2048, Re=5000, scheme=scheme)
    (r, u, v), _ = W.random_state(case, 3, amp_u=0.05)
    cells = sample_cells(2048, 2048, 32, margin=2)
    f0, got, used = one_step_sampled(dv, case, (r, u, v), "f32", dict(strip_rows=32, warps_per_block=2),
                                     cells)
    exp = window_expect(case, f0, cells)
    assert np.max(np.abs(got - exp) / np.abs(exp)) < 2e-6


def test_batched_512_cases_sampled(dv):
    """The batched workload at full size (512 cases from seed 1511, FP32): a
    sample of cases against their own single solvers, bitwise, after 4 steps
    in graph chunks of 2."""
    cases = W.batched_cases(512, seed=1511)
    b = dv.Batch([c for c, _ in cases], precision="f32")
    try:
        b.set_launch(strip_rows=32, warps_per_block=4)
        for k, (c, f) in enumerate(cases):
            b.init_equilibrium(k, *f)
        b.step(4, graph_chunk=2)
        for k in (0, 1, 100, 255, 256, 257, 400, 511):
            c, f = cases[k]
            assert b.case_status(k) == 0
            with dv.Solver(c, precision="f32") as s:
                s.set_launch(strip_rows=32)
                s.init_equilibrium(*f)
                s.step(4)
                np.testing.assert_array_equal(b.get_f(k), s.get_f())
    finally:
        b.close()
