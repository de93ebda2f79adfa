"""Build libdvbe.so in-tree with nvcc for sm_103a.

Each translation unit is compiled to an object in parallel, then linked into
paper_1511_00242_gb300/libdvbe.so.  No cmake, one -gencode, about a minute.
"""
from __future__ import annotations

import concurrent.futures
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libdvbe.so")
SOURCES = ["step_f64.cu", "step_f32.cu", "step_f16.cu", "aux_kernels.cu", "dvbe_capi.cu", "batch.cu",
           "noalloc.cu", "tune_cache.cu", "multipass.cu", "quad_mesh.cu"]
HEADERS = ["internal.h", "capi_common.h", "step_kernel.cuh"]

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
              "-I" + os.path.join(ROOT, "include"), "-I" + CSRC]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdvbe")


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


KNOBS = ("DVBE_DUGKS_MINB", "DVBE_BKG_MINB", "DVBE_DUGKS_UNROLL", "DVBE_BKG_UNROLL",
         "DVBE_PAIR_MINB", "DVBE_PAIR_DUGKS_UNROLL", "DVBE_PAIR_BKG_UNROLL", "DVBE_STAGES",
         "DVBE_PAIR_INNER_MAXREG", "DVBE_RING_CONCURRENT", "DVBE_RING_FIRST", "DVBE_RING_PRIORITY", "DVBE_HALO",
         "DVBE_WALLS_PATH")


def _build_id(extra):
    """Hash of the sources, headers and knobs: names the build in the
    autotuner cache, so a changed kernel never reuses an old choice."""
    import hashlib
    h = hashlib.sha256(" ".join(NVCC_FLAGS + extra).encode())
    for name in sorted(SOURCES + HEADERS):
        with open(os.path.join(CSRC, name), "rb") as f:
            h.update(f.read())
    with open(os.path.join(ROOT, "include", "dvbe.h"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def _flags():
    """NVCC flags.  The step kernel's tuning knobs (occupancy target and
    row-loop unrolling per scheme, defaults in step_kernel.cuh) may be
    overridden by environment variables of the same names."""
    extra = ["-D%s=%d" % (k, int(os.environ[k])) for k in KNOBS if k in os.environ]
    return NVCC_FLAGS + extra


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "flags.txt")
    flags = " ".join(_flags())
    if not os.path.exists(stamp) or open(stamp).read() != flags:
        force = True
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "dvbe.h")]
    objs, jobs = [], []
    extra = [f for f in _flags() if f not in NVCC_FLAGS]
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        # the cache unit carries the build id, which depends on every source
        deps = [os.path.join(CSRC, x) for x in SOURCES] if src == "tune_cache.cu" else [s]
        if force or _stale(o, deps + hdrs):
            cmd = [nvcc()] + _flags() + (["-Xptxas", "-v"] if ptxas_info else [])
            if src == "tune_cache.cu":
                cmd.append('-DDVBE_BUILD_ID="%s"' % _build_id(extra))
            jobs.append(cmd + ["-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    if jobs:
        with concurrent.futures.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for cmd, r in ex.map(run, jobs):
                if verbose or ptxas_info:
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode != 0:
                    sys.stderr.write(r.stdout + r.stderr)
                    raise RuntimeError("nvcc failed: " + " ".join(cmd))
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc(), "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed: " + " ".join(cmd))
        os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(flags)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv)
    print(LIB)
