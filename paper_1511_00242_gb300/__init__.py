"""Python binding of libdvbe, the GB300 D2Q9 DUGKS / BKG finite-volume library.

Thin ctypes marshalling over the C ABI in include/dvbe.h: every function
named ``dvbe_*`` here calls the C function of the same name and raises
``DvbeError`` on a non-zero status.  ``Solver`` and ``Batch`` bundle the
calls for one problem described as a plain case dict (see workloads.py):

    nx, ny, xf, yf, RT, tau, dt, scheme ("dugks" | "bkg"),
    bc = [W, E, S, N], each a list of (kind, s0, s1, rho, ux, uy),
    kind in periodic | wall | diffuse | inflow | outflow | symmetry.

Every step of the method runs in the CUDA kernels of libdvbe.so; there is no
Python or CPU fallback.  If the library is missing, the first call raises.
PyTorch is optional plumbing: ``use_torch_allocator()`` routes the library's
device allocations through torch's caching allocator, and a torch stream
handle may be passed as ``stream``.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdvbe.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "dvbe.h")

KINDS = {"periodic": 0, "wall": 1, "diffuse": 2, "inflow": 3, "outflow": 4, "symmetry": 5,
         "outflow_neq": 6}
SCHEMES = {"dugks": 0, "bkg": 1, "cfree_upwind": 2, "cfree_central": 3}
PRECISIONS = {"f64": 0, "f32": 1, "f32_dev": 2, "f16_dev": 3, "bf16_dev": 4}
RECONS = {"linear": 0, "upwind_cell": 1}
PATHS = {"fused": 0, "multipass": 1}
STATUS = {0: "DVBE_OK", 1: "DVBE_ERR_INVALID_ARG", 2: "DVBE_ERR_CFL", 3: "DVBE_ERR_OOM",
          4: "DVBE_ERR_CUDA", 5: "DVBE_ERR_DIVERGED", 6: "DVBE_ERR_TIMEOUT",
          7: "DVBE_ERR_UNSUPPORTED"}
DVBE_OK, DVBE_ERR_INVALID_ARG, DVBE_ERR_CFL, DVBE_ERR_OOM = 0, 1, 2, 3
DVBE_ERR_CUDA, DVBE_ERR_DIVERGED, DVBE_ERR_TIMEOUT, DVBE_ERR_UNSUPPORTED = 4, 5, 6, 7

DEFAULT_WAIT_LIMIT = 16777216  # DVBE_DEFAULT_WAIT_LIMIT
_DP = ctypes.POINTER(ctypes.c_double)


class dvbe_bc_segment(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("s0", ctypes.c_double), ("s1", ctypes.c_double),
                ("rho", ctypes.c_double), ("ux", ctypes.c_double), ("uy", ctypes.c_double)]


class dvbe_params(ctypes.Structure):
    _fields_ = [("mesh", ctypes.c_void_p), ("RT", ctypes.c_double), ("tau", ctypes.c_double),
                ("dt", ctypes.c_double), ("rho0", ctypes.c_double), ("scheme", ctypes.c_int),
                ("precision", ctypes.c_int), ("bc", ctypes.POINTER(dvbe_bc_segment) * 4),
                ("nbc", ctypes.c_int * 4), ("allow_cfl_ge_1", ctypes.c_int),
                ("bkg_fd", ctypes.c_int), ("dev_scale", ctypes.c_double),
                ("cuda_stream", ctypes.c_void_p), ("recon", ctypes.c_int), ("path", ctypes.c_int)]


class dvbe_launch(ctypes.Structure):
    _fields_ = [("strip_rows", ctypes.c_int), ("warps_per_block", ctypes.c_int),
                ("blocks", ctypes.c_int), ("graph_chunk", ctypes.c_int)]


class DvbeError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None

_SIGS = {
    "dvbe_d2q9": [ctypes.c_double, _DP, _DP, ctypes.POINTER(ctypes.c_int)],
    "dvbe_mesh_create": [ctypes.c_int, ctypes.c_int, _DP, _DP, ctypes.POINTER(ctypes.c_void_p)],
    "dvbe_mesh_create_quad": [ctypes.c_int, ctypes.c_int, _DP, _DP, ctypes.POINTER(ctypes.c_void_p)],
    "dvbe_mesh_cells": [ctypes.c_void_p, _DP, _DP, _DP],
    "dvbe_mesh_destroy": [ctypes.c_void_p],
    "dvbe_mesh_geometry": [ctypes.c_void_p, _DP, _DP, _DP],
    "dvbe_faces_uniform": [ctypes.c_int, ctypes.c_double, ctypes.c_double, _DP],
    "dvbe_faces_tanh": [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _DP],
    "dvbe_faces_geometric": [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, _DP],
    "dvbe_dt_from_cfl": [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _DP],
    "dvbe_set_allocator": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p],
    "dvbe_solver_create": [ctypes.POINTER(dvbe_params), ctypes.POINTER(ctypes.c_void_p)],
    "dvbe_solver_destroy": [ctypes.c_void_p],
    "dvbe_init_equilibrium": [ctypes.c_void_p, _DP, _DP, _DP],
    "dvbe_init_chapman_enskog": [ctypes.c_void_p, _DP, _DP, _DP, ctypes.POINTER(_DP)],
    "dvbe_init_f": [ctypes.c_void_p, _DP],
    "dvbe_get_f": [ctypes.c_void_p, _DP],
    "dvbe_step": [ctypes.c_void_p, ctypes.c_longlong],
    "dvbe_step_async": [ctypes.c_void_p, ctypes.c_longlong],
    "dvbe_sync": [ctypes.c_void_p],
    "dvbe_step_count": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)],
    "dvbe_get_moments": [ctypes.c_void_p, _DP, _DP, _DP],
    "dvbe_conserved": [ctypes.c_void_p, _DP],
    "dvbe_residual": [ctypes.c_void_p, _DP],
    "dvbe_l2_error_u": [ctypes.c_void_p, _DP, _DP, _DP],
    "dvbe_get_launch": [ctypes.c_void_p, ctypes.POINTER(dvbe_launch)],
    "dvbe_set_launch": [ctypes.c_void_p, ctypes.POINTER(dvbe_launch)],
    "dvbe_autotune": [ctypes.c_void_p, ctypes.c_int, _DP],
    "dvbe_set_autotune_cache": [ctypes.c_char_p],
    "dvbe_device_state": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p),
                          ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                          ctypes.POINTER(ctypes.c_int)],
    "dvbe_launch_count": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)],
    "dvbe_set_wait_limit": [ctypes.c_void_p, ctypes.c_longlong],
    "dvbe_state_bytes": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)],
    "dvbe_pack_line": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                       ctypes.c_void_p],
    "dvbe_unpack_line": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                         ctypes.c_void_p],
    "dvbe_conserved_window": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              _DP],
    "dvbe_save_state": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t,
                        ctypes.POINTER(ctypes.c_longlong)],
    "dvbe_load_state": [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_longlong],
    "dvbe_batch_create": [ctypes.POINTER(dvbe_params), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)],
    "dvbe_batch_destroy": [ctypes.c_void_p],
    "dvbe_batch_init_equilibrium": [ctypes.c_void_p, ctypes.c_int, _DP, _DP, _DP],
    "dvbe_batch_step": [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int],
    "dvbe_batch_case_status": [ctypes.c_void_p, ctypes.c_int],
    "dvbe_batch_get_moments": [ctypes.c_void_p, ctypes.c_int, _DP, _DP, _DP],
    "dvbe_batch_get_f": [ctypes.c_void_p, ctypes.c_int, _DP],
    "dvbe_batch_set_launch": [ctypes.c_void_p, ctypes.POINTER(dvbe_launch)],
    "dvbe_batch_autotune": [ctypes.c_void_p, ctypes.c_int, _DP],
    "dvbe_batch_launch_count": [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong)],
    "dvbe_batch_set_wait_limit": [ctypes.c_void_p, ctypes.c_longlong],
    "dvbe_conserved_noalloc": [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                               ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p],
    "dvbe_last_error": [],
    "dvbe_version": [],
}


def lib():
    """Load libdvbe.so (built in-tree by paper_1511_00242_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            if name in ("dvbe_mesh_destroy", "dvbe_solver_destroy", "dvbe_batch_destroy"):
                fn.restype = None
            elif name in ("dvbe_last_error", "dvbe_version"):
                fn.restype = ctypes.c_char_p
            else:
                fn.restype = ctypes.c_int
        _lib = L
    return _lib


def declared_functions(header: str = HEADER):
    """Names of the functions include/dvbe.h declares."""
    txt = open(header).read()
    return sorted(set(re.findall(r"^DVBE_API\s+[^(]*?\b(dvbe_\w+)\s*\(", txt, flags=re.M)))


def dvbe_last_error() -> str:
    return lib().dvbe_last_error().decode()


def dvbe_version() -> str:
    return lib().dvbe_version().decode()


def _call(name, *args):
    st = getattr(lib(), name)(*args)
    if st != DVBE_OK:
        raise DvbeError(st, name, dvbe_last_error())
    return st


def _dp(a):
    return a.ctypes.data_as(_DP)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


# ---------------------------------------------------------------- host-only calls

def dvbe_d2q9(RT: float):
    xi, w, opp = np.zeros((9, 2)), np.zeros(9), np.zeros(9, dtype=np.int32)
    _call("dvbe_d2q9", RT, _dp(xi), _dp(w), opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return xi, w, opp


def dvbe_faces_uniform(n, a, b):
    out = np.zeros(n + 1)
    _call("dvbe_faces_uniform", n, a, b, _dp(out))
    return out


def dvbe_faces_tanh(n, a, b, beta):
    out = np.zeros(n + 1)
    _call("dvbe_faces_tanh", n, a, b, beta, _dp(out))
    return out


def dvbe_faces_geometric(n, a, d0, ratio):
    out = np.zeros(n + 1)
    _call("dvbe_faces_geometric", n, a, d0, ratio, _dp(out))
    return out


def dvbe_mesh_create(xf, yf):
    xf, yf = _f64(xf), _f64(yf)
    h = ctypes.c_void_p()
    _call("dvbe_mesh_create", len(xf) - 1, len(yf) - 1, _dp(xf), _dp(yf), ctypes.byref(h))
    return h


def dvbe_mesh_create_quad(X, Y):
    """Quadrilateral mesh from vertex arrays X, Y of shape [ny+1, nx+1]."""
    X, Y = _f64(X), _f64(Y)
    if X.ndim != 2 or X.shape != Y.shape:
        raise ValueError("X and Y must be 2-D arrays of one shape [ny+1, nx+1]")
    h = ctypes.c_void_p()
    _call("dvbe_mesh_create_quad", X.shape[1] - 1, X.shape[0] - 1, _dp(X), _dp(Y), ctypes.byref(h))
    return h


def dvbe_mesh_cells(mesh, nx, ny):
    xc, yc, vol = np.zeros((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx))
    _call("dvbe_mesh_cells", mesh, _dp(xc), _dp(yc), _dp(vol))
    return xc, yc, vol


def mesh_of(case: dict):
    """The library mesh of a case dict: vertex arrays X, Y (quadrilateral
    cells) or face coordinates xf, yf (tensor mesh)."""
    if "X" in case:
        return dvbe_mesh_create_quad(case["X"], case["Y"])
    return dvbe_mesh_create(case["xf"], case["yf"])


def dvbe_mesh_destroy(mesh):
    lib().dvbe_mesh_destroy(mesh)


def dvbe_mesh_geometry(mesh, nx, ny):
    xc, yc, vol = np.zeros(nx), np.zeros(ny), np.zeros((ny, nx))
    _call("dvbe_mesh_geometry", mesh, _dp(xc), _dp(yc), _dp(vol))
    return xc, yc, vol


def dvbe_dt_from_cfl(mesh, RT, cfl):
    dt = ctypes.c_double()
    _call("dvbe_dt_from_cfl", mesh, RT, cfl, ctypes.byref(dt))
    return dt.value


# ---------------------------------------------------------------- parameters

def make_params(case: dict, mesh, precision="f64", stream=None, allow_cfl_ge_1=False,
                bkg_fd=False, dev_scale=0.0, rho0=1.0, path="fused"):
    """dvbe_params for a case dict; returns (params, keep-alive list)."""
    p = dvbe_params()
    p.mesh = mesh
    p.RT, p.tau, p.dt = float(case["RT"]), float(case["tau"]), float(case["dt"])
    p.rho0 = float(rho0)
    sc = case.get("scheme", "dugks")
    p.scheme = SCHEMES[sc] if isinstance(sc, str) else int(sc)
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    keep = []
    for side in range(4):
        segs = case["bc"][side]
        arr = (dvbe_bc_segment * max(1, len(segs)))()
        for k, (kind, s0, s1, rho, ux, uy) in enumerate(segs):
            arr[k] = dvbe_bc_segment(KINDS[kind] if isinstance(kind, str) else int(kind),
                                     s0, s1, rho, ux, uy)
        keep.append(arr)
        p.bc[side] = ctypes.cast(arr, ctypes.POINTER(dvbe_bc_segment))
        p.nbc[side] = len(segs)
    p.allow_cfl_ge_1 = int(bool(allow_cfl_ge_1))
    p.bkg_fd = int(bool(bkg_fd))
    p.dev_scale = float(dev_scale)
    p.cuda_stream = stream if stream is None else ctypes.c_void_p(int(stream))
    p.recon = RECONS[case.get("recon", "linear")]
    p.path = PATHS[path]
    return p, keep


def dvbe_conserved_noalloc(f_tilde_ptr, precision, nx, ny, pitch, dx_ptr, dy_ptr, RT, rho0,
                           dev_scale, out_ptr, stream=None):
    """Allocation-free FP64 mass / momentum sums over caller-owned device
    buffers (all pointers are device addresses as ints); see include/dvbe.h."""
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    _call("dvbe_conserved_noalloc", ctypes.c_void_p(f_tilde_ptr), prec, int(nx), int(ny),
          int(pitch), ctypes.c_void_p(dx_ptr), ctypes.c_void_p(dy_ptr), float(RT), float(rho0),
          float(dev_scale), ctypes.c_void_p(out_ptr),
          None if stream is None else ctypes.c_void_p(int(stream)))


def dvbe_set_autotune_cache(path):
    """Autotuner cache file: a path, "" for the default, None for no cache."""
    _call("dvbe_set_autotune_cache", None if path is None else os.fsencode(path))


def dvbe_solver_create(params):
    h = ctypes.c_void_p()
    _call("dvbe_solver_create", ctypes.byref(params), ctypes.byref(h))
    return h


def dvbe_solver_destroy(s):
    lib().dvbe_solver_destroy(s)


def dvbe_step(s, n):
    _call("dvbe_step", s, n)


def dvbe_step_async(s, n):
    _call("dvbe_step_async", s, n)


def dvbe_sync(s):
    _call("dvbe_sync", s)


# ---------------------------------------------------------------- torch plumbing

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_torch_hooks = None


def use_torch_allocator(enable: bool = True):
    """Route libdvbe's device allocations through torch's caching allocator."""
    global _torch_hooks
    if not enable:
        _call("dvbe_set_allocator", None, None, None)
        _torch_hooks = None
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:  # out of memory: the library reports DVBE_ERR_OOM
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    hooks = (_ALLOC_FN(_alloc), _FREE_FN(_free))
    _call("dvbe_set_allocator", ctypes.cast(hooks[0], ctypes.c_void_p),
          ctypes.cast(hooks[1], ctypes.c_void_p), None)
    _torch_hooks = hooks


# ---------------------------------------------------------------- solver

class Solver:
    """One problem on the GPU: create, init, step, read back (dvbe_solver_*).

    case: dict with nx, ny, and either xf[nx+1], yf[ny+1] (face coordinates of
    a tensor mesh) or X, Y [ny+1][nx+1] (vertices of quadrilateral cells,
    which run the multi-pass FP64 step), RT, tau,
    dt, scheme ("dugks", "bkg", "cfree_upwind", "cfree_central"), optionally
    recon ("linear" or "upwind_cell", the latter on the multi-pass path), and bc, four
    lists (W, E, S, N) of segments (kind, s0, s1, rho, ux, uy) with kind one
    of "periodic", "wall", "diffuse", "inflow", "outflow", "outflow_neq",
    "symmetry".  precision: storage of f_tilde, "f64", "f32", "f32_dev",
    "f16_dev" or "bf16_dev".  path: "fused" (default) or "multipass" (FP64,
    face arrays in device memory).  stream: a cudaStream_t (e.g. a torch stream's
    cuda_stream) or None.  Host arrays are float64 [ny][nx] (fields) or
    [9][ny][nx] (f_tilde).  Errors raise DvbeError with the library's status.
    """

    def __init__(self, case: dict, precision="f64", stream=None, allow_cfl_ge_1=False,
                 bkg_fd=False, dev_scale=0.0, rho0=1.0, path="fused"):
        self.case = case
        self.nx, self.ny = int(case["nx"]), int(case["ny"])
        self.precision = precision
        mesh = mesh_of(case)
        try:
            params, keep = make_params(case, mesh, precision, stream, allow_cfl_ge_1, bkg_fd,
                                       dev_scale, rho0, path)
            self.h = dvbe_solver_create(params)
        finally:
            dvbe_mesh_destroy(mesh)

    def close(self):
        if getattr(self, "h", None):
            dvbe_solver_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _field(self, a):
        return _f64(a, (self.ny, self.nx))

    def init_equilibrium(self, rho, ux, uy):
        r, u, v = self._field(rho), self._field(ux), self._field(uy)
        _call("dvbe_init_equilibrium", self.h, _dp(r), _dp(u), _dp(v))

    def init_chapman_enskog(self, rho, ux, uy, derivs):
        r, u, v = self._field(rho), self._field(ux), self._field(uy)
        ds = [self._field(d) for d in derivs]
        arr = (_DP * 9)(*[_dp(d) for d in ds])
        _call("dvbe_init_chapman_enskog", self.h, _dp(r), _dp(u), _dp(v), arr)

    def init_f(self, f_tilde):
        f = _f64(f_tilde, (9, self.ny, self.nx))
        _call("dvbe_init_f", self.h, _dp(f))

    def get_f(self):
        f = np.zeros((9, self.ny, self.nx))
        _call("dvbe_get_f", self.h, _dp(f))
        return f

    def step(self, n: int):
        _call("dvbe_step", self.h, int(n))

    def step_async(self, n: int):
        _call("dvbe_step_async", self.h, int(n))

    def sync(self):
        _call("dvbe_sync", self.h)

    def status(self) -> int:
        return lib().dvbe_sync(self.h)

    def step_count(self) -> int:
        n = ctypes.c_longlong()
        _call("dvbe_step_count", self.h, ctypes.byref(n))
        return n.value

    def moments(self):
        r, u, v = (np.zeros((self.ny, self.nx)) for _ in range(3))
        _call("dvbe_get_moments", self.h, _dp(r), _dp(u), _dp(v))
        return r, u, v

    def conserved(self):
        out = np.zeros(3)
        _call("dvbe_conserved", self.h, _dp(out))
        return out

    def residual(self) -> float:
        r = ctypes.c_double()
        _call("dvbe_residual", self.h, ctypes.byref(r))
        return r.value

    def l2_error_u(self, ua, va) -> float:
        a, b = self._field(ua), self._field(va)
        e = ctypes.c_double()
        _call("dvbe_l2_error_u", self.h, _dp(a), _dp(b), ctypes.byref(e))
        return e.value

    def get_launch(self) -> dict:
        l = dvbe_launch()
        _call("dvbe_get_launch", self.h, ctypes.byref(l))
        return dict(strip_rows=l.strip_rows, warps_per_block=l.warps_per_block, blocks=l.blocks,
                    graph_chunk=l.graph_chunk)

    def set_launch(self, strip_rows=None, warps_per_block=None, blocks=None, graph_chunk=None):
        cur = self.get_launch()
        for k, v in dict(strip_rows=strip_rows, warps_per_block=warps_per_block, blocks=blocks,
                         graph_chunk=graph_chunk).items():
            if v is not None:
                cur[k] = int(v)
        l = dvbe_launch(cur["strip_rows"], cur["warps_per_block"], cur["blocks"], cur["graph_chunk"])
        _call("dvbe_set_launch", self.h, ctypes.byref(l))

    def autotune(self, steps: int = 5) -> float:
        ms = ctypes.c_double()
        _call("dvbe_autotune", self.h, int(steps), ctypes.byref(ms))
        return ms.value

    def device_state(self):
        p, pitch, plane, eb = ctypes.c_void_p(), ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
        _call("dvbe_device_state", self.h, ctypes.byref(p), ctypes.byref(pitch), ctypes.byref(plane),
              ctypes.byref(eb))
        return p.value, pitch.value, plane.value, eb.value

    def launch_count(self) -> int:
        n = ctypes.c_longlong()
        _call("dvbe_launch_count", self.h, ctypes.byref(n))
        return n.value

    def pack_line(self, axis, index, lo, hi, dev_ptr):
        """One line of cells of all nine fields into a device buffer [9][hi-lo]
        (axis 0: column `index` over rows lo..hi-1; axis 1: a row)."""
        _call("dvbe_pack_line", self.h, int(axis), int(index), int(lo), int(hi), ctypes.c_void_p(dev_ptr))

    def unpack_line(self, axis, index, lo, hi, dev_ptr):
        _call("dvbe_unpack_line", self.h, int(axis), int(index), int(lo), int(hi), ctypes.c_void_p(dev_ptr))

    def conserved_window(self, i0, j0, nx, ny):
        out = np.zeros(3)
        _call("dvbe_conserved_window", self.h, int(i0), int(j0), int(nx), int(ny), _dp(out))
        return out

    def save_state(self):
        """Checkpoint: (raw device storage of f_tilde as bytes, step count)."""
        n = ctypes.c_size_t()
        _call("dvbe_state_bytes", self.h, ctypes.byref(n))
        buf = ctypes.create_string_buffer(n.value)
        step = ctypes.c_longlong()
        _call("dvbe_save_state", self.h, buf, n.value, ctypes.byref(step))
        return buf.raw, step.value

    def load_state(self, state: bytes, step: int = 0):
        """Restart from a checkpoint of save_state (same problem and precision)."""
        _call("dvbe_load_state", self.h, state, len(state), int(step))

    def set_wait_limit(self, polls: int = None):
        """Polls of a pending row copy before a step gives up with
        DVBE_ERR_TIMEOUT (None: the library default)."""
        _call("dvbe_set_wait_limit", self.h, DEFAULT_WAIT_LIMIT if polls is None else int(polls))


class Batch:
    """Many independent cases stepped by one persistent launch per scheme
    (dvbe_batch_*).  cases: case dicts as for Solver (DUGKS or BKG), all with
    one precision.  A case whose density turns non-finite is flagged
    (case_status) and skipped from then on; the others continue."""

    def __init__(self, cases, precision="f32", allow_cfl_ge_1=False):
        self.cases = cases
        meshes, keeps = [], []
        arr = (dvbe_params * len(cases))()
        try:
            for k, case in enumerate(cases):
                m = mesh_of(case)
                meshes.append(m)
                p, keep = make_params(case, m, precision, allow_cfl_ge_1=allow_cfl_ge_1)
                keeps.append(keep)
                arr[k] = p
            h = ctypes.c_void_p()
            _call("dvbe_batch_create", arr, len(cases), ctypes.byref(h))
            self.h = h
        finally:
            for m in meshes:
                dvbe_mesh_destroy(m)

    def close(self):
        if getattr(self, "h", None):
            lib().dvbe_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_equilibrium(self, i, rho, ux, uy):
        c = self.cases[i]
        r, u, v = (_f64(a, (c["ny"], c["nx"])) for a in (rho, ux, uy))
        _call("dvbe_batch_init_equilibrium", self.h, i, _dp(r), _dp(u), _dp(v))

    def step(self, n, graph_chunk=0):
        _call("dvbe_batch_step", self.h, int(n), int(graph_chunk))

    def case_status(self, i) -> int:
        return lib().dvbe_batch_case_status(self.h, i)

    def moments(self, i):
        c = self.cases[i]
        r, u, v = (np.zeros((c["ny"], c["nx"])) for _ in range(3))
        _call("dvbe_batch_get_moments", self.h, i, _dp(r), _dp(u), _dp(v))
        return r, u, v

    def get_f(self, i):
        c = self.cases[i]
        f = np.zeros((9, c["ny"], c["nx"]))
        _call("dvbe_batch_get_f", self.h, i, _dp(f))
        return f

    def set_launch(self, strip_rows=32, warps_per_block=4, blocks=0):
        l = dvbe_launch(strip_rows, warps_per_block, blocks, 0)
        _call("dvbe_batch_set_launch", self.h, ctypes.byref(l))

    def autotune(self, steps=3) -> float:
        ms = ctypes.c_double()
        _call("dvbe_batch_autotune", self.h, int(steps), ctypes.byref(ms))
        return ms.value

    def launch_count(self) -> int:
        n = ctypes.c_longlong()
        _call("dvbe_batch_launch_count", self.h, ctypes.byref(n))
        return n.value

    def set_wait_limit(self, polls: int = None):
        _call("dvbe_batch_set_wait_limit", self.h, DEFAULT_WAIT_LIMIT if polls is None else int(polls))
