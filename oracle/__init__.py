"""ctypes binding of the plain FP64 CPU oracle (``dvbe_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU-baseline / reference leg may import this package.  The
product library never loads it, and it shares no code with the CUDA path.

Problems are described as plain data (see ``workloads.py``):

    case = dict(nx=, ny=, xf=, yf=, RT=, tau=, dt=, scheme="dugks"|"bkg"|"cfree_upwind"|"cfree_central",
                bc=[W, E, S, N])      # each side: list of (kind, s0, s1, rho, ux, uy)

with kind one of "periodic", "wall", "diffuse", "inflow", "outflow",
"symmetry".  Distribution arrays are float64 ``[9, ny, nx]``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dvbe_oracle.c")
_HDR = os.path.join(_HERE, "dvbe_oracle.h")
_SO = os.path.join(_HERE, "liboracle.so")

KINDS = {"periodic": 0, "wall": 1, "diffuse": 2, "inflow": 3, "outflow": 4, "symmetry": 5,
         "outflow_neq": 6}
SCHEMES = {"dugks": 0, "bkg": 1, "cfree_upwind": 2, "cfree_central": 3}
RECONS = {"linear": 0, "upwind_cell": 1}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off, so every operation
    rounds as written)."""
    stale = (not os.path.exists(_SO)) or any(
        os.path.getmtime(s) > os.path.getmtime(_SO) for s in (_SRC, _HDR))
    if force or stale:
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Seg(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("s0", ctypes.c_double), ("s1", ctypes.c_double),
                ("rho", ctypes.c_double), ("ux", ctypes.c_double), ("uy", ctypes.c_double)]


_DP = ctypes.POINTER(ctypes.c_double)


class _Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("xf", _DP), ("yf", _DP),
                ("RT", ctypes.c_double), ("tau", ctypes.c_double), ("dt", ctypes.c_double),
                ("scheme", ctypes.c_int), ("nbc", ctypes.c_int * 4),
                ("bc", ctypes.POINTER(_Seg) * 4), ("recon", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.orc_equilibrium.restype = None
        for name in ("orc_d2q9", "orc_faces_uniform", "orc_faces_tanh", "orc_faces_geometric",
                     "orc_dt_from_cfl", "orc_init_equilibrium", "orc_init_chapman_enskog",
                     "orc_step", "orc_step_bkg_fd", "orc_step_implicit", "orc_tilde_from_f",
                     "orc_moments", "orc_conserved", "orc_l2_error_u"):
            getattr(L, name).restype = ctypes.c_int
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_DP)


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


class Problem:
    """Owns the ctypes problem struct and keeps its arrays alive."""

    def __init__(self, case: dict):
        self.case = case
        self.nx, self.ny = int(case["nx"]), int(case["ny"])
        self.xf = np.ascontiguousarray(case["xf"], dtype=np.float64)
        self.yf = np.ascontiguousarray(case["yf"], dtype=np.float64)
        self._segs = []
        s = _Problem()
        s.nx, s.ny = self.nx, self.ny
        s.xf, s.yf = _dp(self.xf), _dp(self.yf)
        s.RT, s.tau, s.dt = float(case["RT"]), float(case["tau"]), float(case["dt"])
        s.scheme = SCHEMES[case.get("scheme", "dugks")]
        s.recon = RECONS[case.get("recon", "linear")]
        for side in range(4):
            segs = case["bc"][side]
            arr = (_Seg * len(segs))()
            for k, seg in enumerate(segs):
                kind, s0, s1, rho, ux, uy = seg
                arr[k] = _Seg(KINDS[kind], s0, s1, rho, ux, uy)
            self._segs.append(arr)
            s.nbc[side] = len(segs)
            s.bc[side] = ctypes.cast(arr, ctypes.POINTER(_Seg))
        self.s = s

    def ref(self):
        return ctypes.byref(self.s)

    def zeros9(self):
        return np.zeros((9, self.ny, self.nx), dtype=np.float64)


def d2q9(RT: float):
    xi = np.zeros((9, 2))
    w = np.zeros(9)
    opp = np.zeros(9, dtype=np.int32)
    _check(lib().orc_d2q9(ctypes.c_double(RT), _dp(xi), _dp(w),
                          opp.ctypes.data_as(ctypes.POINTER(ctypes.c_int))), "orc_d2q9")
    return xi, w, opp


def equilibrium(RT: float, rho: float, ux: float, uy: float) -> np.ndarray:
    out = np.zeros(9)
    lib().orc_equilibrium(ctypes.c_double(RT), ctypes.c_double(rho), ctypes.c_double(ux),
                          ctypes.c_double(uy), _dp(out))
    return out


def faces_uniform(n, a, b):
    out = np.zeros(n + 1)
    _check(lib().orc_faces_uniform(n, ctypes.c_double(a), ctypes.c_double(b), _dp(out)), "faces")
    return out


def faces_tanh(n, a, b, beta):
    out = np.zeros(n + 1)
    _check(lib().orc_faces_tanh(n, ctypes.c_double(a), ctypes.c_double(b),
                                ctypes.c_double(beta), _dp(out)), "faces")
    return out


def faces_geometric(n, a, d0, ratio):
    out = np.zeros(n + 1)
    _check(lib().orc_faces_geometric(n, ctypes.c_double(a), ctypes.c_double(d0),
                                     ctypes.c_double(ratio), _dp(out)), "faces")
    return out


def dt_from_cfl(xf, yf, RT, cfl):
    xf = np.ascontiguousarray(xf, dtype=np.float64)
    yf = np.ascontiguousarray(yf, dtype=np.float64)
    dt = ctypes.c_double()
    _check(lib().orc_dt_from_cfl(len(xf) - 1, len(yf) - 1, _dp(xf), _dp(yf), ctypes.c_double(RT),
                                 ctypes.c_double(cfl), ctypes.byref(dt)), "dt_from_cfl")
    return dt.value


def _f2(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def init_equilibrium(case: dict, rho, ux, uy) -> np.ndarray:
    P = Problem(case)
    out = P.zeros9()
    rho, ux, uy = _f2(rho), _f2(ux), _f2(uy)
    _check(lib().orc_init_equilibrium(P.ref(), _dp(rho), _dp(ux), _dp(uy), _dp(out)), "init_eq")
    return out


def init_chapman_enskog(case: dict, rho, ux, uy, derivs) -> np.ndarray:
    """derivs: sequence of 9 arrays (rho_t, ux_t, uy_t, rho_x, ux_x, uy_x, rho_y, ux_y, uy_y)."""
    P = Problem(case)
    out = P.zeros9()
    rho, ux, uy = _f2(rho), _f2(ux), _f2(uy)
    ds = [_f2(d) for d in derivs]
    arr = (_DP * 9)(*[_dp(d) for d in ds])
    _check(lib().orc_init_chapman_enskog(P.ref(), _dp(rho), _dp(ux), _dp(uy), arr, _dp(out)),
           "init_ce")
    return out


def step(case: dict, f_tilde: np.ndarray, nsteps: int) -> np.ndarray:
    P = Problem(case)
    f = np.array(f_tilde, dtype=np.float64, order="C", copy=True)
    _check(lib().orc_step(P.ref(), _dp(f), ctypes.c_longlong(nsteps)), "orc_step")
    return f


def step_bkg_fd(case: dict, f_tilde: np.ndarray, nsteps: int) -> np.ndarray:
    P = Problem(case)
    f = np.array(f_tilde, dtype=np.float64, order="C", copy=True)
    _check(lib().orc_step_bkg_fd(P.ref(), _dp(f), ctypes.c_longlong(nsteps)), "orc_step_bkg_fd")
    return f


def step_implicit(case: dict, f: np.ndarray, nsteps: int) -> np.ndarray:
    P = Problem(case)
    g = np.array(f, dtype=np.float64, order="C", copy=True)
    _check(lib().orc_step_implicit(P.ref(), _dp(g), ctypes.c_longlong(nsteps)), "orc_step_implicit")
    return g


def tilde_from_f(case: dict, f: np.ndarray) -> np.ndarray:
    P = Problem(case)
    f = _f2(f)
    out = P.zeros9()
    _check(lib().orc_tilde_from_f(P.ref(), _dp(f), _dp(out)), "tilde_from_f")
    return out


def moments(case: dict, f_tilde: np.ndarray):
    P = Problem(case)
    f = _f2(f_tilde)
    rho = np.zeros((P.ny, P.nx))
    ux = np.zeros_like(rho)
    uy = np.zeros_like(rho)
    _check(lib().orc_moments(P.ref(), _dp(f), _dp(rho), _dp(ux), _dp(uy)), "moments")
    return rho, ux, uy


def conserved(case: dict, f_tilde: np.ndarray) -> np.ndarray:
    P = Problem(case)
    f = _f2(f_tilde)
    out = np.zeros(3)
    _check(lib().orc_conserved(P.ref(), _dp(f), _dp(out)), "conserved")
    return out


def l2_error_u(case: dict, f_tilde: np.ndarray, ua, va) -> float:
    P = Problem(case)
    f = _f2(f_tilde)
    ua, va = _f2(ua), _f2(va)
    e = ctypes.c_double()
    _check(lib().orc_l2_error_u(P.ref(), _dp(f), _dp(ua), _dp(va), ctypes.byref(e)), "l2_error_u")
    return e.value


# ---------------------------------------------------------------- quad meshes
#
# A curvilinear structured mesh is a case dict with vertex arrays instead of
# face coordinates:
#
#     qcase = dict(nx=, ny=, X=[(ny+1), (nx+1)], Y=[(ny+1), (nx+1)], RT=, tau=, dt=,
#                  scheme=, recon=, bc=[W, E, S, N])
#
# cell (i, j) has the vertices (i, j), (i+1, j), (i+1, j+1), (i, j+1),
# counter-clockwise.

class _QuadProblem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("X", _DP), ("Y", _DP),
                ("RT", ctypes.c_double), ("tau", ctypes.c_double), ("dt", ctypes.c_double),
                ("scheme", ctypes.c_int), ("recon", ctypes.c_int), ("nbc", ctypes.c_int * 4),
                ("bc", ctypes.POINTER(_Seg) * 4)]


class QuadProblem:
    def __init__(self, case: dict):
        self.nx, self.ny = int(case["nx"]), int(case["ny"])
        self.X = np.ascontiguousarray(case["X"], dtype=np.float64)
        self.Y = np.ascontiguousarray(case["Y"], dtype=np.float64)
        assert self.X.shape == (self.ny + 1, self.nx + 1) == self.Y.shape
        self._segs = []
        s = _QuadProblem()
        s.nx, s.ny = self.nx, self.ny
        s.X, s.Y = _dp(self.X), _dp(self.Y)
        s.RT, s.tau, s.dt = float(case["RT"]), float(case["tau"]), float(case["dt"])
        s.scheme = SCHEMES[case.get("scheme", "dugks")]
        s.recon = RECONS[case.get("recon", "linear")]
        for side in range(4):
            segs = case["bc"][side]
            arr = (_Seg * len(segs))()
            for k, seg in enumerate(segs):
                kind, s0, s1, rho, ux, uy = seg
                arr[k] = _Seg(KINDS[kind], s0, s1, rho, ux, uy)
            self._segs.append(arr)
            s.nbc[side] = len(segs)
            s.bc[side] = ctypes.cast(arr, ctypes.POINTER(_Seg))
        self.s = s

    def ref(self):
        return ctypes.byref(self.s)


def _quad_lib():
    L = lib()
    for name in ("orc_quad_geometry", "orc_quad_step", "orc_quad_conserved", "orc_quad_dt_from_cfl"):
        getattr(L, name).restype = ctypes.c_int
    return L


def quad_geometry(case: dict):
    """Cell centres and volumes, each [ny, nx]."""
    P = QuadProblem(case)
    xc, yc, vol = (np.zeros((P.ny, P.nx)) for _ in range(3))
    _check(_quad_lib().orc_quad_geometry(P.ref(), _dp(xc), _dp(yc), _dp(vol)), "orc_quad_geometry")
    return xc, yc, vol


def quad_step(case: dict, f_tilde: np.ndarray, nsteps: int) -> np.ndarray:
    P = QuadProblem(case)
    f = np.array(f_tilde, dtype=np.float64, order="C", copy=True)
    assert f.shape == (9, P.ny, P.nx)
    _check(_quad_lib().orc_quad_step(P.ref(), _dp(f), ctypes.c_longlong(nsteps)), "orc_quad_step")
    return f


def quad_conserved(case: dict, f_tilde: np.ndarray) -> np.ndarray:
    P = QuadProblem(case)
    out = np.zeros(3)
    _check(_quad_lib().orc_quad_conserved(P.ref(), _dp(_f2(f_tilde)), _dp(out)), "orc_quad_conserved")
    return out


def quad_dt_from_cfl(case: dict, cfl: float) -> float:
    P = QuadProblem(case)
    dt = ctypes.c_double()
    _check(_quad_lib().orc_quad_dt_from_cfl(P.ref(), ctypes.c_double(cfl), ctypes.byref(dt)),
           "orc_quad_dt_from_cfl")
    return dt.value


def quad_init_equilibrium(case: dict, rho, ux, uy) -> np.ndarray:
    """f_tilde = f_eq(rho, u) cell by cell (pointwise: the mesh plays no part)."""
    nx, ny = int(case["nx"]), int(case["ny"])
    flat = dict(nx=nx, ny=ny, xf=np.arange(nx + 1.0), yf=np.arange(ny + 1.0), RT=case["RT"],
                tau=case["tau"], dt=case["dt"], bc=[[("periodic", -1e300, 1e300, 1, 0, 0)]] * 4)
    return init_equilibrium(flat, rho, ux, uy)
