"""Stability map by batched bisection (Sec 3.2, Fig. cavity_stab): the largest
stable dt/tau at a given CFL number for the lid-driven cavity, for both
schemes.  The paper reports that BKG becomes unstable at moderate dt/tau
even below CFL 1 while DUGKS is nearly unaffected by the CFL number; this
test checks the first of these at CFL 0.9 on the 32^2 cavity, and that the
bisection brackets are consistent with every trial."""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dv():
    from paper_1511_00242_gb300 import build
    build.build()
    import paper_1511_00242_gb300 as dv
    return dv


def test_cavity_stability_map_32(dv):
    from paper_1511_00242_gb300.stability import bisect_max_ratio
    points = [("dugks", 32, 0.5), ("dugks", 32, 0.9), ("bkg", 32, 0.5), ("bkg", 32, 0.9)]
    res = bisect_max_ratio(W.cavity_at_ratio, points, lo=0.5, hi=1e4, iters=8, t_end=50.0)
    by = {}
    for r in res:
        print(f"stability {r['point']}: max stable dt/tau in [{r['lo']:.4g}, {r['hi']}]"
              + (" (stable at the upper end)" if r["stable_at_upper_end"] else ""))
        lo = r["lo"]
        hi = r["hi"] if r["hi"] is not None else float("inf")
        for ratio, ok in r["trials"]:
            # every stable trial is at or below lo, every unstable one at or above hi
            assert (ratio <= lo) if ok else (ratio >= hi)
        by[r["point"]] = (lo, hi)
    # DUGKS stays stable above the dt/tau at which BKG fails (CFL 0.9)
    assert by[("dugks", 32, 0.9)][0] >= by[("bkg", 32, 0.9)][1]
