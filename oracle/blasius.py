"""Blasius boundary layer by shooting (test infrastructure; oracle side).

The similarity solution of the laminar flat-plate boundary layer the paper
compares against (Sec 3.3): f''' + f f''/2 = 0, f(0) = f'(0) = 0,
f'(inf) = 1, with eta = y sqrt(U / (nu x)).  Then u/U = f'(eta) and
v / (U / (2 sqrt(Re_x))) = eta f' - f.  Solved with classical RK4 on
[0, eta_max] and bisection on f''(0).
"""
from __future__ import annotations

import numpy as np


def _rhs(s):
    f, fp, fpp = s
    return np.array([fp, fpp, -0.5 * f * fpp])


def _integrate(fpp0: float, eta_max: float, n: int):
    h = eta_max / n
    s = np.array([0.0, 0.0, fpp0])
    out = np.zeros((n + 1, 3))
    out[0] = s
    for k in range(n):
        k1 = _rhs(s)
        k2 = _rhs(s + 0.5 * h * k1)
        k3 = _rhs(s + 0.5 * h * k2)
        k4 = _rhs(s + h * k3)
        s = s + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        out[k + 1] = s
    return out


def solve(eta_max: float = 12.0, n: int = 2400):
    """Returns (eta, f, f', f'') and f''(0)."""
    lo, hi = 0.1, 1.0
    for _ in range(100):
        mid = 0.5 * (lo + hi)
        if _integrate(mid, eta_max, n)[-1, 1] < 1.0:
            lo = mid
        else:
            hi = mid
    fpp0 = 0.5 * (lo + hi)
    sol = _integrate(fpp0, eta_max, n)
    eta = np.linspace(0.0, eta_max, n + 1)
    return eta, sol[:, 0], sol[:, 1], sol[:, 2], fpp0


def profiles(y, x: float, U: float, nu: float):
    """u/U and v/(U/(2 sqrt(Re_x))) at height(s) y and distance x from the leading edge."""
    eta_grid, f, fp, _, _ = solve()
    eta = np.asarray(y) * np.sqrt(U / (nu * x))
    u = np.interp(eta, eta_grid, fp, right=1.0)
    vs = np.interp(eta, eta_grid, eta_grid * fp - f, right=(eta_grid * fp - f)[-1])
    return u, vs
