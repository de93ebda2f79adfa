"""Failure detection and restart of the step kernel.

Each warp stages rows of f_tilde through asynchronous copies completed on
mbarriers, and every wait on them is bounded.  With the bound set to zero
polls, a warp whose next row copy has not landed when first tested gives
up: it stops fetching, waits (bounded) for the copies it has in flight and
leaves, and the step returns DVBE_ERR_TIMEOUT.  The copies are of the
solver's own buffer and always land, so nothing is left pending on the GPU;
afterwards the default bound is restored, the state re-initialised, and the
same solver must again match the oracle.  Also: a run stopped after k steps,
read back with get_f and restarted in a new solver from init_f continues
bit for bit as the uninterrupted run."""
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


def _timeout_seen(step_once, tries=20):
    for _ in range(tries):
        st = step_once()
        if st != 0:
            return st
    return 0


@pytest.mark.parametrize("precision", ["f64", "f32_dev"])
def test_wait_limit_times_out_then_recovers(dv, precision):
    case, fields = W.cavity(200, Re=400, scheme="dugks")
    with dv.Solver(case, precision=precision) as s:
        s.set_launch(strip_rows=16, warps_per_block=2)
        s.init_equilibrium(*fields)
        s.set_wait_limit(0)

        def once():
            lib = dv.lib()
            st = lib.dvbe_step(s.h, 1)
            return st

        st = _timeout_seen(once)
        assert st == dv.DVBE_ERR_TIMEOUT, st
        assert "wait" in dv.dvbe_last_error()
        # the context is usable: restore the bound, restart, compare
        s.set_wait_limit(None)
        s.init_equilibrium(*fields)
        s.step(30)
        g = s.get_f()
    o = O.step(case, O.init_equilibrium(case, *fields), 30)
    if precision == "f64":
        assert float(np.max(np.abs(g - o) / np.abs(o))) < 1e-12
    else:
        assert float(np.max(np.abs(g - o)) / np.max(np.abs(o))) < 1e-6


def test_batch_wait_limit_times_out_then_recovers(dv):
    cases = [W.cavity(150, Re=300, scheme="dugks")[0], W.taylor_green_box(130, scheme="bkg")[0]]
    fields = [W.cavity(150)[1], W.taylor_green_box(130)[1]]
    b = dv.Batch(cases, precision="f32_dev")
    try:
        b.set_launch(strip_rows=16, warps_per_block=2)
        for k in range(2):
            b.init_equilibrium(k, *fields[k])
        b.set_wait_limit(0)
        seen = False
        for _ in range(20):
            b.step(1)
            if any(b.case_status(k) == dv.DVBE_ERR_TIMEOUT for k in range(2)):
                seen = True
                break
        assert seen
        b.set_wait_limit(None)
        for k in range(2):
            b.init_equilibrium(k, *fields[k])
        b.step(20)
        for k in range(2):
            assert b.case_status(k) == 0
            o = O.step(cases[k], O.init_equilibrium(cases[k], *fields[k]), 20)
            g = b.get_f(k)
            assert float(np.max(np.abs(g - o)) / np.max(np.abs(o))) < 1e-6
    finally:
        b.close()


def test_negative_wait_limit_is_rejected(dv):
    case, fields = W.taylor_green_box(32)
    with dv.Solver(case) as s:
        with pytest.raises(dv.DvbeError) as e:
            s.set_wait_limit(-1)
        assert e.value.status == dv.DVBE_ERR_INVALID_ARG


def _run_whole_and_mid(dv, case, fields, precision, k, m):
    with dv.Solver(case, precision=precision) as s:
        s.init_equilibrium(*fields)
        s.step(k + m)
        whole = s.get_f()
    s = dv.Solver(case, precision=precision)
    s.init_equilibrium(*fields)
    s.step(k)
    return whole, s


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_restart_from_get_f_is_bitwise(dv, precision, scheme):
    """get_f after k steps, init_f into a new solver, m more steps: the same
    bits as k + m steps in one solver.  For FP64 and absolute FP32 storage
    the float64 host copy holds the stored values exactly."""
    case, fields = W.cavity(150, Re=500, scheme=scheme, stretch_beta=1.2)
    k, m = 37, 41
    whole, s = _run_whole_and_mid(dv, case, fields, precision, k, m)
    with s:
        mid = s.get_f()
    with dv.Solver(case, precision=precision) as s:
        s.init_f(mid)
        s.step(m)
        np.testing.assert_array_equal(s.get_f(), whole)


@pytest.mark.parametrize("precision", ["f64", "f32_dev", "f16_dev", "bf16_dev"])
@pytest.mark.parametrize("scheme", ["dugks", "bkg"])
def test_restart_from_saved_state_is_bitwise(dv, precision, scheme):
    """save_state after k steps, load_state into a new solver, m more steps:
    the same bits and step count as k + m steps in one solver, in every
    storage mode (deviation modes included, whose float64 host copies may
    round a tiny deviation away)."""
    case, fields = W.cavity(150, Re=500, scheme=scheme, stretch_beta=1.2)
    k, m = 37, 41
    whole, s = _run_whole_and_mid(dv, case, fields, precision, k, m)
    with s:
        state, step = s.save_state()
    assert step == k
    with dv.Solver(case, precision=precision) as s:
        s.load_state(state, step)
        s.step(m)
        assert s.step_count() == k + m
        np.testing.assert_array_equal(s.get_f(), whole)
    with dv.Solver(case, precision=precision) as s:
        with pytest.raises(dv.DvbeError) as e:
            s.load_state(state[:-8], step)
        assert e.value.status == dv.DVBE_ERR_INVALID_ARG
