#!/usr/bin/env python
"""Throughput of the fused D2Q9 finite-volume step (MLUPS and HBM roofline).

Headline workload: Taylor-Green vortex on a periodic 4096 x 4096 mesh
(u0 = 0.01, CFL 0.5, dt/tau = 10), DUGKS, FP32 arithmetic with f_tilde stored
as FP32 deviations from w rho0.  The line states that storage's error
against the FP64 path, relative to the discretisation error, on the 256^2 and
512^2 forms of the same decay, with the trend extrapolated to the timed mesh.
One step = one time step of the whole mesh (all 9 directions of every cell):
on this doubly periodic mesh one launch of the step kernel.  The two f_tilde
buffers (604 MB each) are far larger than the 129 MB L2, so no flush is
needed between steps.

Prints one JSON line.  `--impl reference` times the FP64 CPU oracle instead
(the plain program the CUDA path is checked against) on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

BYTES_PER_CELL = {"f64": 144, "f32": 72, "f32_dev": 72, "f16_dev": 36, "bf16_dev": 36}
METRIC = "D2Q9 DUGKS/BKG MLUPS and % HBM roofline, FP32/BF16 vs FP64 at stated L2 error"
DTYPE = {"f64": "f64", "f32": "f32", "f32_dev": "f32", "f16_dev": "f32 (f16 storage)",
         "bf16_dev": "f32 (bf16 storage)"}


def args_():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=600)
    p.add_argument("--warmup", type=int, default=10)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=4096, help="mesh side")
    p.add_argument("--scheme", default="dugks", choices=["dugks", "bkg"])
    p.add_argument("--precision", default="f32_dev", choices=list(BYTES_PER_CELL))
    p.add_argument("--no-extras", action="store_true", help="skip the secondary measurements")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--stability-map", action="store_true",
                   help="print the cavity stability map (max stable dt/tau against CFL) and exit")
    p.add_argument("--launch", default=None,
                   help="strip_rows,warps_per_block,blocks for the headline solver (skips its autotune)")
    p.add_argument("--accuracy-sizes", default="256,512",
                   help="mesh sides of the accuracy check of the headline mode (1024 adds ~4 min of FP64)")
    p.add_argument("--batch-steps", type=int, default=2000)
    return p.parse_args()


def workload(n, scheme):
    case, fields = W.taylor_green_box(n, u0=0.01, cfl=0.5, scheme=scheme, dt_over_tau=10.0)
    return case, fields


def workload_config(a):
    """The `config` object both arms print for the same workload."""
    return {"workload": f"taylor-green {a.n}x{a.n} periodic, u0=0.01, CFL 0.5, "
                        f"dt/tau=10, {a.scheme.upper()}, {a.precision} storage",
            "scheme": a.scheme, "precision": a.precision, "cells": a.n * a.n}


def step_kernels(scheme, precision):
    """Name of the kernels of one fused step: the inner strips and the edge
    strips, launched concurrently on two streams."""
    return f"k_step_inner + k_step_edge<{scheme}, {precision}>"


def measured_traffic(scheme, precision, cells):
    """DRAM bytes per step of this scheme's step kernels from the committed
    ncu captures (profiles/traffic.json), scaled to this mesh; None if no
    capture is of these kernels or the kernel source has changed since."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            recs = json.load(f)
    except Exception:
        return None
    for t in recs if isinstance(recs, list) else [recs]:
        if t.get("kernel") != step_kernels(scheme, precision):
            continue
        try:
            with open(os.path.join(ROOT, t["source"]), "rb") as f:
                sha = hashlib.sha256(f.read()).hexdigest()
        except Exception:
            return None
        return t["dram_bytes_per_cell"] * cells if sha.startswith(t["sha256_prefix"]) else None
    return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            m = json.load(f)
        return float(m["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                       "-lms", "100", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out, _ = self.p.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k]
                          and "Not" not in r[5 + k]})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def max_over_ranks(t, world, device):
    """Slowest rank's time: each rank runs its own replica of the workload
    (no collective on the data path), so the whole job takes the max."""
    if world == 1:
        return t
    import torch
    import torch.distributed as dist
    tt = torch.tensor([t], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_mlups(world, cells, steps, t):
    """Whole-job throughput: the cell updates of all ranks over the slowest rank's time."""
    return world * cells * steps / t / 1e6


def time_steps(dv, s, stream, torch, K):
    """K steps on the solver's stream bracketed by CUDA events on that stream."""
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = s.launch_count()
    e0.record(stream)
    s.step_async(K)
    e1.record(stream)
    e1.synchronize()
    s.sync()
    return e0.elapsed_time(e1) / 1e3, s.launch_count() - l0


def batched_vs_loop(dv, torch, steps=2000, chunk=50, ncases=512, precision="f32_dev"):
    """The batched workload: 512 cases from seed 1511 (half Taylor-Green, half
    cavities, sides 32..512, both schemes), FP32 arithmetic with FP32-deviation
    storage, `steps` steps in CUDA graphs of `chunk` steps.  The batched form
    is one persistent launch per scheme per step over all cases, its launch
    shape from the batch autotuner; the per-case loop steps each case with its
    own solver, each with its own autotuned launch shape and the same graphs.
    Cases that diverge in the batched run are excluded from both sides and
    listed by index.  The accuracy line is the first Taylor-Green case of the
    batch: its error against the FP64 path over the same steps, against the
    FP64 path's own error against the analytic decay."""
    cases = W.batched_cases(ncases, seed=1511)
    cells = np.array([c["nx"] * c["ny"] for c, _ in cases], dtype=np.float64)
    b = dv.Batch([c for c, _ in cases], precision=precision)
    for k, (c, f) in enumerate(cases):
        b.init_equilibrium(k, *f)
    tuned = b.autotune(10)
    b.step(chunk, graph_chunk=chunk)  # graph capture
    for k, (c, f) in enumerate(cases):
        b.init_equilibrium(k, *f)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    b.step(steps, graph_chunk=chunk)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    ok = np.array([b.case_status(k) == 0 for k in range(ncases)])
    itg = next(k for k, (c, _) in enumerate(cases) if "taylor" in c["name"] and ok[k])
    _, ub, vb = b.moments(itg)
    b.close()
    solvers, shapes = [], {}
    for k, (c, f) in enumerate(cases):
        s = dv.Solver(c, precision=precision)
        s.init_equilibrium(*f)
        s.autotune(10)
        s.set_launch(graph_chunk=chunk)
        l = s.get_launch()
        shapes[(l["strip_rows"], l["warps_per_block"], l["blocks"] > 0)] = \
            shapes.get((l["strip_rows"], l["warps_per_block"], l["blocks"] > 0), 0) + 1
        s.step_async(chunk)  # graph capture
        solvers.append(s)
    for s, (c, f) in zip(solvers, cases):
        s.init_equilibrium(*f)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k, s in enumerate(solvers):
        if ok[k]:
            s.step_async(steps)
    for s in solvers:
        s.status()
    tl = time.perf_counter() - t0
    for s in solvers:
        s.close()
    # accuracy of the sampled Taylor-Green case
    c, f = cases[itg]
    with dv.Solver(c, precision="f64") as s:
        s.set_launch(graph_chunk=chunk)
        s.init_equilibrium(*f)
        s.step(steps)
        _, u64, v64 = s.moments()
    ua, va = W.taylor_green_box_analytic(c, steps * c["dt"])
    ed = float(np.sqrt(np.sum((u64 - ua) ** 2 + (v64 - va) ** 2) / np.sum(ua ** 2 + va ** 2)))
    ep = float(np.sqrt(np.sum((ub - u64) ** 2 + (vb - v64) ** 2) / np.sum(u64 ** 2 + v64 ** 2)))
    work = float(np.sum(cells[ok])) * steps
    return {"cases": ncases, "precision": precision, "steps": steps, "graph_chunk": chunk,
            "diverged": [int(k) for k in np.nonzero(~ok)[0]],
            "cells_total": int(cells.sum()), "batched_MLUPS": work / tb / 1e6,
            "per_case_loop_MLUPS": work / tl / 1e6, "speedup": tl / tb,
            "batched_autotune_ms_per_step": tuned,
            "per_case_launch_shapes": {f"{h}x{w}{' persistent' if p else ''}": n
                                       for (h, w, p), n in sorted(shapes.items())},
            "accuracy_sampled_case": {"case": c["name"] + f" ({c['scheme']}, Re {c['Re']:.0f}, CFL {c['cfl']:.2f})",
                                      "E_vs_fp64": ep, "E_fp64_vs_analytic": ed, "ratio": ep / ed,
                                      "bar": 0.1}}


_FP64_REF = {}


def accuracy_at(dv, scheme, precision, n):
    """Error of `precision` against the FP64 path (E_p) and of the FP64 path
    against the analytic decay (E_d): Taylor-Green n^2, dt/tau = 10, run to
    10% decay of the velocity; relative L2 norms of the velocity field.  The
    FP64 run of a scheme and size is made once and reused."""
    case, fields = W.taylor_green_box(n, u0=0.01, cfl=0.5, scheme=scheme, dt_over_tau=10.0)
    steps = int(round(-math.log(0.9) / (2 * case["nu"]) / case["dt"]))
    ua, va = W.taylor_green_box_analytic(case, steps * case["dt"])

    def run(prec):
        with dv.Solver(case, precision=prec) as s:
            s.set_launch(strip_rows=16 if n <= 512 else 32, graph_chunk=200)
            s.init_equilibrium(*fields)
            s.step(steps)
            return s.moments()

    if (scheme, n) not in _FP64_REF:
        _FP64_REF[(scheme, n)] = run("f64")
    _, u64, v64 = _FP64_REF[(scheme, n)]
    _, up, vp = run(precision)
    ed = float(np.sqrt(np.sum((u64 - ua) ** 2 + (v64 - va) ** 2) / np.sum(ua ** 2 + va ** 2)))
    ep = float(np.sqrt(np.sum((up - u64) ** 2 + (vp - v64) ** 2) / np.sum(u64 ** 2 + v64 ** 2)))
    return {"n": n, "steps": steps, "E_vs_fp64": ep, "E_fp64_vs_analytic": ed, "ratio": ep / ed}


def accuracy(dv, scheme, precision, sizes=(256,), target_n=4096):
    """accuracy_at over `sizes`; with two or more sizes the trend of the ratio
    E_p / E_d is fitted as a power of n over the last two and extrapolated to
    the timed mesh (E_d falls as n^-2 while storage rounding accumulates over
    steps that grow as n^2)."""
    pts = [accuracy_at(dv, scheme, precision, n) for n in sizes]
    first = pts[0]
    out = {"case": f"taylor-green n^2, dt/tau=10, to 10% decay, {scheme.upper()}",
           "E_vs_fp64": first["E_vs_fp64"], "E_fp64_vs_analytic": first["E_fp64_vs_analytic"],
           "ratio": first["ratio"], "n": first["n"], "bar": 0.1}
    if len(pts) >= 2:
        a, b = pts[-2], pts[-1]
        p = math.log(b["ratio"] / a["ratio"]) / math.log(b["n"] / a["n"]) if a["ratio"] > 0 and b["ratio"] > 0 else None
        out["trend"] = {"points": pts, "exponent": p,
                        f"ratio_at_{target_n}_extrapolated":
                            (b["ratio"] * (target_n / b["n"]) ** p) if p is not None else None}
    return out


def case_throughput(dv, stream, torch, case, fields, precision, steps, peak, path="fused"):
    """MLUPS and HBM fraction of one workload.  The launch shape is the best
    of the autotuner's choice and a few common shapes, each timed over
    `steps` steps: on meshes with a ring kernel beside the inner one the
    autotuner's short timings are noisy."""
    s = dv.Solver(case, precision=precision, stream=stream.cuda_stream, path=path)
    try:
        s.init_equilibrium(*fields)
        s.autotune(30)
        best = None
        if path == "fused" and "X" not in case:  # the quad mesh runs the multi-pass step
            shapes = [s.get_launch()] + [dict(strip_rows=h, warps_per_block=w, blocks=0)
                                         for h, w in ((16, 4), (24, 2), (36, 2), (52, 2))]
            for shape in shapes:
                s.set_launch(**{k: shape[k] for k in ("strip_rows", "warps_per_block", "blocks")})
                s.step(5)
                tt, _ = time_steps(dv, s, stream, torch, steps)
                if best is None or tt < best[0]:
                    best = (tt, s.get_launch())
            s.set_launch(**{k: best[1][k] for k in ("strip_rows", "warps_per_block", "blocks")})
        s.step(5)
        t, _ = time_steps(dv, s, stream, torch, steps)
        cells = case["nx"] * case["ny"]
        ach = BYTES_PER_CELL[precision] * cells / (t / steps) / 1e9
        return {"MLUPS": cells * steps / t / 1e6, "hbm_GBs": ach, "hbm_frac": ach / peak,
                "launch": s.get_launch(), "cells": cells,
                "buffers_MB": BYTES_PER_CELL[precision] // 2 * cells / 1e6}
    finally:
        s.close()


def stability_map(meshes=(32, 64), cfls=(0.1, 0.3, 0.5, 0.7, 0.9, 1.0, 1.05), iters=10, t_end=100.0):
    """Largest stable dt/tau of the lid-driven cavity (impulsive start, lid
    U = 0.1 c) against the CFL number, both schemes, one JSON line per point:
    the bisection bracket [lo, hi] after `iters` iterations over [0.5, 1e4],
    each trial run to t = t_end (L / U = 10)."""
    from paper_1511_00242_gb300.stability import bisect_max_ratio
    points = [(s, n, c) for s in ("dugks", "bkg") for n in meshes for c in cfls]
    t0 = time.perf_counter()
    res = bisect_max_ratio(W.cavity_at_ratio, points, lo=0.5, hi=1e4, iters=iters, t_end=t_end)
    for r in res:
        r.pop("trials")
        scheme, n, cfl = r.pop("point")
        print(json.dumps(dict(scheme=scheme, mesh=n, cfl=cfl, **r)), flush=True)
    print(json.dumps({"stability_map_seconds": time.perf_counter() - t0}), flush=True)


def _oracle_sample(scheme, n, budget_s):
    """One host thread stepping the FP64 oracle on an n x n sample of the
    Taylor-Green workload until ~budget_s seconds are spent: (cell updates, s)."""
    import oracle as O
    case, fields = workload(n, scheme)
    f = O.init_equilibrium(case, *fields)
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < budget_s:
        f = O.step(case, f, 1)
        steps += 1
    return n * n * steps, time.perf_counter() - t0


def cpu_baseline(scheme, budget_s=12.0, n=512):
    """The FP64 oracle as it stands, on 512 x 512 samples of the same
    Taylor-Green workload: one process per host core, each stepping its own
    sample for ~budget_s seconds (processes started with spawn, as the GPU is
    already in use), and one thread alone for reference."""
    import multiprocessing as mp
    cells1, t1 = _oracle_sample(scheme, n, budget_s)
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.starmap(_oracle_sample, [(scheme, n, budget_s)] * cores)
    total = sum(c for c, _ in res) / max(t for _, t in res) / 1e6
    return {"value": total, "unit": "MLUPS", "cores": cores, "kind": "oracle",
            "sample": f"{scheme.upper()} Taylor-Green {n}x{n}, FP64 C oracle, {cores} processes "
                      f"(one per core) for ~{budget_s:g} s each",
            "single_thread": {"value": cells1 / t1 / 1e6, "unit": "MLUPS", "cores": 1}}


_REF = {}


def _ref_init(scheme, n):
    """Worker set-up of the reference arm: this process's own oracle sample."""
    import oracle as O
    case, fields = workload(n, scheme)
    _REF["case"] = case
    _REF["f"] = O.init_equilibrium(case, *fields)


def _ref_step(_):
    """One oracle step of this process's sample; returns its cell updates."""
    import oracle as O
    _REF["f"] = O.step(_REF["case"], _REF["f"], 1)
    return _REF["case"]["nx"] * _REF["case"]["ny"]


def run_reference(a):
    """Reference arm: the FP64 CPU oracle on the host cores, rank 0 only.  One
    spawned process per core holds its own 256^2 sample of the workload; a
    step is one oracle step of every process's sample."""
    import multiprocessing as mp
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = 256
    cores = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(cores, initializer=_ref_init, initargs=(a.scheme, n)) as pool:
        for _ in range(a.warmup):
            pool.map(_ref_step, range(cores), chunksize=1)
        t0 = time.perf_counter()
        cells = 0
        for _ in range(a.steps):
            cells += sum(pool.map(_ref_step, range(cores), chunksize=1))
        dt = time.perf_counter() - t0
    v = cells / dt / 1e6
    line = {"metric": METRIC, "value": v, "unit": "MLUPS", "impl": "reference", "n_gpus": a.gpus,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(workload_config(a),
                           sample=f"each step: one FP64 oracle step of a {n}x{n} sample of the workload "
                                  f"in each of {cores} processes"),
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": f"{a.scheme.upper()} Taylor-Green {n}x{n} per process and step, "
                                       f"{cores} processes (one per core)"},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    a = args_()
    if a.impl == "reference":
        run_reference(a)
        return
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import paper_1511_00242_gb300 as dv
    from paper_1511_00242_gb300 import build
    build.build()
    if a.stability_map:
        stability_map()
        return

    stream = torch.cuda.Stream()
    case, fields = workload(a.n, a.scheme)
    cells = a.n * a.n
    s = dv.Solver(case, precision=a.precision, stream=stream.cuda_stream)
    s.init_equilibrium(*fields)
    tuned_ms = None
    if a.launch:
        h, w, b = (int(x) for x in a.launch.split(","))
        s.set_launch(strip_rows=h, warps_per_block=w, blocks=b)
    elif not a.no_autotune:
        tuned_ms = s.autotune(10)
    launch = s.get_launch()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # clocks are sampled from the start of the warm-up, which runs for at
    # least half a second, to the end of the timed steps, so that a short
    # timed region still has samples under the same load
    clocks = Clocks(local)
    clocks.start()
    t_w = time.perf_counter()
    s.step(a.warmup)
    while time.perf_counter() - t_w < 0.5:
        s.step(50)
    barrier()
    t_w = time.perf_counter() - t_w
    t, launches = time_steps(dv, s, stream, torch, a.steps)
    barrier()
    ck = clocks.stop()
    if ck is not None:
        ck["window"] = f"warm-up ({t_w:.2f} s, same steps) and the {a.steps} timed steps"
    t = max_over_ranks(t, world, "cuda")
    value = job_mlups(world, cells, a.steps, t)
    per_launch = t / a.steps
    peak, peak_kind = peaks()
    achieved = BYTES_PER_CELL[a.precision] * cells / per_launch / 1e9

    # end to end through the C ABI with host buffers: pinned f_tilde in, K
    # steps, moments out
    f0 = s.get_f()
    pin = torch.empty(f0.shape, dtype=torch.float64, pin_memory=True).numpy()
    pin[...] = f0
    outs = [torch.empty((a.n, a.n), dtype=torch.float64, pin_memory=True).numpy() for _ in range(3)]
    barrier()
    t0 = time.perf_counter()
    s.init_f(pin)
    s.step(a.steps)
    r, u, v = s.moments()
    barrier()
    te = max_over_ranks(time.perf_counter() - t0, world, "cuda")
    outs[0][...] = r
    e2e = {"value": job_mlups(world, cells, a.steps, te), "unit": "MLUPS",
           "h2d_bytes_per_step": pin.nbytes / a.steps, "d2h_bytes_per_step": 3 * cells * 8 / a.steps,
           "note": "init_f from pinned host f_tilde (float64), the steps, get_moments to host"}

    extras = {}
    if not a.no_extras and rank == 0:
        # BKG and the other storage modes on the same workload, shorter runs
        for scheme, prec in (("bkg", "f32_dev"), ("dugks", "f32"), ("bkg", "f32"),
                             ("dugks", "f16_dev"), ("bkg", "f16_dev"), ("dugks", "bf16_dev"),
                             ("dugks", "f64")):
            if scheme == a.scheme and prec == a.precision:
                continue
            c2, fl2 = workload(a.n, scheme)
            s2 = dv.Solver(c2, precision=prec, stream=stream.cuda_stream)
            s2.init_equilibrium(*fl2)
            if not a.no_autotune:
                s2.autotune(3 if prec == "f64" else 10)
            s2.step(3)
            k2 = 60 if prec != "f64" else 20
            t2, _ = time_steps(dv, s2, stream, torch, k2)
            pl = t2 / k2
            ach = BYTES_PER_CELL[prec] * cells / pl / 1e9
            extras[f"{scheme}_{prec}"] = {"MLUPS": cells * k2 / t2 / 1e6, "hbm_GBs": ach,
                                          "hbm_frac": ach / peak, "launch": s2.get_launch()}
            s2.close()
            del s2
            if prec != "f64":
                a2 = accuracy(dv, scheme, prec)
                extras[f"{scheme}_{prec}"]["accuracy_ratio"] = a2["ratio"]
        # the other workloads of the paper's tests at their stated sizes (Sec 3.2, 3.3)
        for scheme in ("dugks", "bkg"):
            c3, fl3 = W.cavity(2048, Re=5000, cfl=0.5, scheme=scheme)
            extras[f"cavity_2048_re5000_{scheme}_f32_dev"] = case_throughput(
                dv, stream, torch, c3, fl3, "f32_dev", 60, peak)
            c4, fl4 = W.flat_plate(nx_up=170, nx_plate=342, ny=256, scheme=scheme)
            extras[f"plate_512x256_{scheme}_f32_dev"] = dict(case_throughput(
                dv, stream, torch, c4, fl4, "f32_dev", 400, peak),
                note="4.7 MB buffers, resident in L2: not HBM-bound")
        # curvilinear meshes: the multi-pass FP64 step on a wavy 1024^2 mesh,
        # beside the same step on the uniform tensor mesh and the fused FP64 step
        cq, flq = W.taylor_green_quad(1024, scheme="dugks")
        extras["quad_wavy_1024_dugks_f64_multipass"] = dict(case_throughput(
            dv, stream, torch, cq, flq, "f64", 40, peak),
            note="six kernels per step with face arrays; hbm_frac against the 144 B/cell minimum")
        extras["quad_wavy_1024_dugks_f32_multipass"] = dict(case_throughput(
            dv, stream, torch, cq, flq, "f32", 40, peak),
            note="FP32 storage and arithmetic; hbm_frac against the 72 B/cell minimum")
        ct, flt = workload(1024, "dugks")
        extras["tensor_1024_dugks_f64_multipass"] = case_throughput(
            dv, stream, torch, ct, flt, "f64", 40, peak, path="multipass")
        extras["tensor_1024_dugks_f64_fused"] = case_throughput(dv, stream, torch, ct, flt, "f64", 40, peak)
        extras["batched_vs_per_case_loop"] = batched_vs_loop(dv, torch, steps=a.batch_steps)
    s.close()
    sizes = tuple(int(x) for x in a.accuracy_sizes.split(",") if x)
    acc = (accuracy(dv, a.scheme, a.precision, sizes=sizes, target_n=a.n)
           if rank == 0 and a.precision != "f64" and sizes else None)

    fbytes = BYTES_PER_CELL[a.precision] // 2 * cells
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": t / a.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[a.precision], "data": "synthetic",
            "config": dict(workload_config(a), **{
                       "l2": (f"inputs larger than L2 (two {fbytes / 1e6:.0f} MB f_tilde buffers), no flush"
                              if fbytes > 129e6 else
                              f"f_tilde buffers of {fbytes / 1e6:.0f} MB fit in L2: not a bench configuration"),
                       "parallelism": f"replicas x{world}", "launch": launch,
                       "autotune_ms_per_step": tuned_ms}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": measured_traffic(a.scheme, a.precision, cells),
                         "peak_kind": peak_kind,
                         "bytes_per_cell": BYTES_PER_CELL[a.precision],
                         "kernel": step_kernels(a.scheme, a.precision)},
            "accuracy": acc,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": ck,
            "extras": extras,
        }
        if not a.no_cpu:
            line["cpu_baseline"] = cpu_baseline(a.scheme)
        other = "bkg" if a.scheme == "dugks" else "dugks"
        if f"{other}_{a.precision}" in extras:
            # cost of a DUGKS step over a BKG step, here and in the paper (context only)
            mlups = {a.scheme: value / world, other: extras[f"{other}_{a.precision}"]["MLUPS"]}
            ratio = {"gpu": mlups["bkg"] / mlups["dugks"],
                     "gpu_case": f"{a.n}^2 Taylor-Green, {a.precision} storage, one GB300",
                     "paper": 1.88, "paper_case": "64^2 Taylor-Green, CPU code on an Intel Xeon "
                                                  "E5-2670v3 at 2.6 GHz (Sec 3.1)"}
            if not a.no_cpu:
                c_d, t_d = _oracle_sample("dugks", 256, 4.0)
                c_b, t_b = _oracle_sample("bkg", 256, 4.0)
                ratio["oracle_1_thread"] = (c_b / t_b) / (c_d / t_d)
            line["dugks_bkg_cost_ratio"] = ratio
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
