"""Stability map: the largest stable dt/tau against the CFL number (Sec 3.2,
Fig. cavity_stab), by bisection over batches of cases.

Every bisection iteration builds one batch that holds all points of the map
at their current trial dt/tau.  The batch is stepped by the batched kernels
for a fixed number of steps, and each case is then classified by the flag the
kernel raised for it (rho <= 0, non-finite or overflowing), plus a bound on
the velocity read back through the batch moments.  A stable
trial raises the point's lower bracket, an unstable one lowers its upper
bracket; the search runs in log(dt/tau).  The final bracket [lo, hi] is the
error range of the map.  All stepping runs in the library's kernels; this
module only schedules the iterations and keeps the brackets.
"""
from __future__ import annotations

import json
import math

import numpy as np


def bisect_max_ratio(make_case, points, lo=0.5, hi=1e4, iters=10, steps=None, t_end=None,
                     u_bound=None, precision="f32", graph_chunk=50):
    """Largest stable dt/tau for each point.

    make_case(point, ratio) -> (case, (rho, ux, uy)) builds the case of one
    point at dt/tau = ratio; the case dict may carry "U" (velocity scale).
    Each iteration steps `steps` steps, or enough to reach the time `t_end` in the
    case with the smallest dt.  A case is unstable if its flag is raised or
    max |u| exceeds u_bound (default 2 U).  Returns a list of dicts with the
    bracket per point; a point whose upper end never failed reports hi.
    """
    from paper_1511_00242_gb300 import Batch

    n = len(points)
    los = np.full(n, float(lo))
    his = np.full(n, float(hi))
    stable_at_hi = np.zeros(n, dtype=bool)
    history = [[] for _ in range(n)]
    # iteration 0 tries the upper end itself, so that points stable there report it
    for it in range(iters + 1):
        trial = his.copy() if it == 0 else np.sqrt(los * his)
        built = [make_case(p, float(r)) for p, r in zip(points, trial)]
        cases = [c for c, _ in built]
        nsteps = steps
        if nsteps is None:
            nsteps = int(math.ceil(t_end / min(c["dt"] for c in cases)))
        b = Batch(cases, precision=precision, allow_cfl_ge_1=True)
        try:
            for k, (_, f) in enumerate(built):
                b.init_equilibrium(k, *f)
            b.step(nsteps, graph_chunk=graph_chunk)
            for k, c in enumerate(cases):
                ok = b.case_status(k) == 0
                if ok:
                    _, u, v = b.moments(k)
                    umax = float(np.max(np.hypot(u, v)))
                    bound = u_bound if u_bound is not None else 2.0 * c.get("U", 0.1)
                    ok = math.isfinite(umax) and umax <= bound
                history[k].append((float(trial[k]), bool(ok)))
                if it == 0:
                    stable_at_hi[k] = ok
                elif ok:
                    los[k] = trial[k]
                else:
                    his[k] = trial[k]
        finally:
            b.close()
        if it == 0 and stable_at_hi.all():
            break
    out = []
    for k, p in enumerate(points):
        if stable_at_hi[k]:
            out.append(dict(point=p, lo=float(hi), hi=None, stable_at_upper_end=True,
                            trials=history[k]))
        else:
            out.append(dict(point=p, lo=float(los[k]), hi=float(his[k]), stable_at_upper_end=False,
                            trials=history[k]))
    return out
