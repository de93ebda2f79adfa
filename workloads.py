"""Seeded synthetic workloads shared by the tests, the bench and smoke().

This module only describes problems: face coordinates of the meshes, initial
macroscopic fields (rho, u), analytic reference fields, random perturbations
and the batched case table.  It holds none of the scheme's arithmetic (no
equilibrium, no transforms, no fluxes); the CUDA library and the CPU oracle
each turn these inputs into distributions on their own.

A case is a plain dict:

    nx, ny          cells
    xf, yf          face coordinates (float64, nx+1 / ny+1)
    RT, tau, dt     velocity-model temperature, relaxation time, time step
    scheme          "dugks" | "bkg"
    bc              [W, E, S, N]; each a list of (kind, s0, s1, rho, ux, uy)
                    kind in periodic | wall | diffuse | inflow | outflow | symmetry

Workloads follow the paper's test problems (Sec 3): Taylor-Green vortex,
lid-driven cavity, flat-plate boundary layer.
"""
from __future__ import annotations

import math

import numpy as np

RT_LATTICE = 1.0 / 3.0  # c_s = 1/sqrt(3) in all of the paper's runs (Sec 3)
INF = 1.0e300           # segment end that covers a whole side


def uniform_faces(n: int, a: float, b: float) -> np.ndarray:
    return a + (b - a) * np.arange(n + 1, dtype=np.float64) / n


def tanh_faces(n: int, a: float, b: float, beta: float) -> np.ndarray:
    """Both-end clustering: x(s) = a + (b-a) (1 + tanh(beta(2s-1))/tanh(beta)) / 2."""
    s = np.arange(n + 1, dtype=np.float64) / n
    return a + (b - a) * 0.5 * (1.0 + np.tanh(beta * (2.0 * s - 1.0)) / math.tanh(beta))


def geometric_faces(n: int, a: float, d0: float, ratio: float) -> np.ndarray:
    i = np.arange(n + 1, dtype=np.float64)
    if ratio == 1.0:
        return a + d0 * i
    return a + d0 * (ratio ** i - 1.0) / (ratio - 1.0)


def centres(f: np.ndarray) -> np.ndarray:
    return 0.5 * (f[1:] + f[:-1])


def cfl_dt(xf, yf, cfl: float, RT: float = RT_LATTICE) -> float:
    """Time step for a stated CFL number: cfl * (smallest cell width) / |xi|_max
    with |xi|_max = sqrt(6 RT) for D2Q9 (problem set-up, Sec 2.2)."""
    dmin = min(np.min(np.diff(xf)), np.min(np.diff(yf)))
    return cfl * dmin / math.sqrt(6.0 * RT)


def periodic_bc():
    side = [("periodic", -INF, INF, 0.0, 0.0, 0.0)]
    return [list(side), list(side), list(side), list(side)]


def wall(ux=0.0, uy=0.0, kind="wall", s0=-INF, s1=INF):
    return (kind, s0, s1, 1.0, ux, uy)


# --------------------------------------------------------------------------
# Taylor-Green vortex
# --------------------------------------------------------------------------

def taylor_green_box(n: int, u0: float = 0.01, nu: float = 0.05, cfl: float = 0.5,
                     scheme: str = "dugks", dt_over_tau: float | None = None):
    """Periodic [0, 2 pi]^2 Taylor-Green vortex, rho0 = 1, f = f_eq initially.

    u = -u0 cos x sin y, v = u0 sin x cos y, p = p0 - rho0 u0^2 (cos 2x + cos 2y)/4,
    rho = rho0 + (p - p0)/RT.  Velocity decays as exp(-2 nu t).
    dt = cfl * dx / sqrt(6 RT) (cfl = 0.5 gives dt = 0.5 dx / sqrt(2)).
    With dt_over_tau given, nu is set from the CFL time step instead.
    """
    L = 2.0 * math.pi
    xf = uniform_faces(n, 0.0, L)
    yf = uniform_faces(n, 0.0, L)
    dt = cfl_dt(xf, yf, cfl)
    if dt_over_tau is not None:
        tau = dt / dt_over_tau
        nu = tau * RT_LATTICE
    tau = nu / RT_LATTICE
    case = dict(nx=n, ny=n, xf=xf, yf=yf, RT=RT_LATTICE, tau=tau, dt=dt, scheme=scheme,
                bc=periodic_bc(), nu=nu, u0=u0, name=f"taylor-green {n}x{n}")
    x, y = np.meshgrid(centres(xf), centres(yf))
    rho = 1.0 - u0 * u0 * (np.cos(2 * x) + np.cos(2 * y)) / 4.0 / RT_LATTICE
    ux = -u0 * np.cos(x) * np.sin(y)
    uy = u0 * np.sin(x) * np.cos(y)
    return case, (rho, ux, uy)


def taylor_green_box_analytic(case, t: float):
    x, y = np.meshgrid(centres(case["xf"]), centres(case["yf"]))
    d = math.exp(-2.0 * case["nu"] * t)
    u0 = case["u0"]
    return -u0 * np.cos(x) * np.sin(y) * d, u0 * np.sin(x) * np.cos(y) * d


def taylor_green_paper(n: int, scheme: str = "dugks", dt_over_tau: float = 2.0):
    """The set-up of Sec 3.1: unit box, U0 = 1e-2/sqrt(3), nu = 1e-4/sqrt(3),
    dt = 2 tau (Table tab:tv_Nerr; other dt/tau for the time-step sweep of
    Fig. tv_dtErr), Chapman-Enskog initial state from the analytic solution.

    Returns (case, fields, derivs, t_c) with derivs = (rho_t, ux_t, uy_t, rho_x,
    ux_x, uy_x, rho_y, ux_y, uy_y) of the analytic solution at t = 0 and
    t_c = ln 2 / (8 nu pi^2) the half-life time.
    """
    U0 = 1e-2 / math.sqrt(3.0)
    nu = 1e-4 / math.sqrt(3.0)
    tau = nu / RT_LATTICE
    dt = dt_over_tau * tau
    xf = uniform_faces(n, 0.0, 1.0)
    yf = uniform_faces(n, 0.0, 1.0)
    case = dict(nx=n, ny=n, xf=xf, yf=yf, RT=RT_LATTICE, tau=tau, dt=dt, scheme=scheme,
                bc=periodic_bc(), nu=nu, U0=U0, name=f"taylor-green (paper) {n}x{n}")
    pi = math.pi
    x, y = np.meshgrid(centres(xf), centres(yf))
    c2x, s2x, c2y, s2y = np.cos(2 * pi * x), np.sin(2 * pi * x), np.cos(2 * pi * y), np.sin(2 * pi * y)
    ux = -U0 * c2x * s2y
    uy = U0 * s2x * c2y
    p = -U0 * U0 / 4.0 * (np.cos(4 * pi * x) + np.cos(4 * pi * y))
    rho = 1.0 + p / RT_LATTICE
    derivs = (
        -16.0 * pi * pi * nu * p / RT_LATTICE,          # rho_t
        -8.0 * pi * pi * nu * ux,                       # ux_t
        -8.0 * pi * pi * nu * uy,                       # uy_t
        pi * U0 * U0 * np.sin(4 * pi * x) / RT_LATTICE,  # rho_x
        2.0 * pi * U0 * s2x * s2y,                      # ux_x
        2.0 * pi * U0 * c2x * c2y,                      # uy_x
        pi * U0 * U0 * np.sin(4 * pi * y) / RT_LATTICE,  # rho_y
        -2.0 * pi * U0 * c2x * c2y,                     # ux_y
        -2.0 * pi * U0 * s2x * s2y,                     # uy_y
    )
    t_c = math.log(2.0) / (8.0 * nu * pi * pi)
    return case, (rho, ux, uy), derivs, t_c


def taylor_green_paper_analytic(case, t: float):
    pi = math.pi
    x, y = np.meshgrid(centres(case["xf"]), centres(case["yf"]))
    d = math.exp(-8.0 * pi * pi * case["nu"] * t)
    U0 = case["U0"]
    return (-U0 * np.cos(2 * pi * x) * np.sin(2 * pi * y) * d,
            U0 * np.sin(2 * pi * x) * np.cos(2 * pi * y) * d)


# --------------------------------------------------------------------------
# Lid-driven cavity, Couette flow, flat plate
# --------------------------------------------------------------------------

def cavity(n: int, Re: float = 1000.0, U: float = 0.1, cfl: float = 0.5, scheme: str = "dugks",
           stretch_beta: float | None = None, kind: str = "wall"):
    """Unit square, lid (north wall) moving at U in x, other walls at rest, fluid
    at rest initially; nu = U L / Re.  Optional tanh clustering toward all walls."""
    if stretch_beta:
        xf = tanh_faces(n, 0.0, 1.0, stretch_beta)
    else:
        xf = uniform_faces(n, 0.0, 1.0)
    yf = xf.copy()
    nu = U / Re
    tau = nu / RT_LATTICE
    dt = cfl_dt(xf, yf, cfl)
    bc = [[wall(kind=kind)], [wall(kind=kind)], [wall(kind=kind)], [wall(U, 0.0, kind=kind)]]
    case = dict(nx=n, ny=n, xf=xf, yf=yf, RT=RT_LATTICE, tau=tau, dt=dt, scheme=scheme, bc=bc,
                nu=nu, name=f"cavity Re={Re:g} {n}x{n}" + (" tanh" if stretch_beta else ""))
    rho = np.ones((n, n))
    return case, (rho, np.zeros((n, n)), np.zeros((n, n)))


def couette(nx: int, ny: int, U: float = 0.05, nu: float = 0.1, cfl: float = 0.5,
            scheme: str = "dugks", H: float = 1.0, kind: str = "wall", RT: float = RT_LATTICE):
    """Periodic in x; fixed wall at y=0, wall moving at U at y=H; fluid at rest.
    kind: "wall" (bounce-back) or "diffuse"; tau = nu / RT."""
    xf = uniform_faces(nx, 0.0, H * nx / ny)
    yf = uniform_faces(ny, 0.0, H)
    tau = nu / RT
    dt = cfl_dt(xf, yf, cfl, RT)
    per = [("periodic", -INF, INF, 0.0, 0.0, 0.0)]
    bc = [list(per), list(per), [wall(kind=kind)], [wall(U, 0.0, kind=kind)]]
    case = dict(nx=nx, ny=ny, xf=xf, yf=yf, RT=RT, tau=tau, dt=dt, scheme=scheme, bc=bc,
                nu=nu, U=U, name=f"couette {nx}x{ny} {kind}")
    return case, (np.ones((ny, nx)), np.zeros((ny, nx)), np.zeros((ny, nx)))


def cavity_four_lids(nx: int = 14, ny: int = 10, U: float = 0.05, scheme: str = "dugks",
                     kind: str = "wall", tau: float = 0.01, cfl: float = 0.5, RT: float = RT_LATTICE):
    """A box whose four walls all move tangentially: S at -U and N at +U in x,
    W at -0.6 U and E at +0.6 U in y, on a tanh-clustered mesh
    ([0, 1.4] x [0, 1]).  The problem is unchanged by a rotation through 180
    degrees about the box centre (x -> Lx - x, y -> Ly - y, u -> -u), which
    maps each corner to the opposite one."""
    xf = tanh_faces(nx, 0.0, 1.4, 1.2)
    yf = tanh_faces(ny, 0.0, 1.0, 1.0)
    bc = [[wall(0.0, -0.6 * U, kind=kind)], [wall(0.0, 0.6 * U, kind=kind)],
          [wall(-U, 0.0, kind=kind)], [wall(U, 0.0, kind=kind)]]
    case = dict(nx=nx, ny=ny, xf=xf, yf=yf, RT=RT, tau=tau, dt=cfl_dt(xf, yf, cfl, RT),
                scheme=scheme, bc=bc, name=f"four-lid box {nx}x{ny} {kind}")
    return case


def rotation_symmetric_state(case, seed: int, amp_u: float = 0.02, amp_rho: float = 0.01):
    """Random (rho, ux, uy) unchanged by the 180-degree rotation of the cell
    grid: rho(i, j) = rho(n-1-i, m-1-j), u(i, j) = -u(n-1-i, m-1-j)."""
    (r, u, v), _ = random_state(case, seed, amp_u=amp_u, amp_rho=amp_rho)
    R = lambda a: a[::-1, ::-1]
    return 0.5 * (r + R(r)), 0.5 * (u - R(u)), 0.5 * (v - R(v))


def free_stream_channel(n: int = 24, scheme: str = "dugks", rho_inf: float = 1.0,
                        tau: float = 0.01, cfl: float = 0.5, RT: float = RT_LATTICE):
    """[0, 1] x [0, 4/n] periodic in y with free-stream faces on W and E at
    (rho_inf, 0, 0); the caller chooses the initial state."""
    xf = uniform_faces(n, 0.0, 1.0)
    yf = uniform_faces(4, 0.0, 4.0 / n)
    per = [("periodic", -INF, INF, 0.0, 0.0, 0.0)]
    fs = [("inflow", -INF, INF, rho_inf, 0.0, 0.0)]
    return dict(nx=n, ny=4, xf=xf, yf=yf, RT=RT, tau=tau, dt=cfl_dt(xf, yf, cfl, RT),
                scheme=scheme, bc=[list(fs), list(fs), list(per), list(per)],
                name=f"free-stream channel {n}x4")


def flat_plate(nx_up: int = 40, nx_plate: int = 88, ny: int = 64, U: float = 0.1,
               Re_L: float = 1e5, L: float = 1.0, dy_min: float | None = None,
               height: float = 0.5, up_len: float = 0.5, dx_min: float | None = None,
               cfl: float = 0.5, scheme: str = "dugks", outflow: str = "outflow"):
    """Laminar boundary layer over a flat plate on 0 <= x <= L (Sec 3.3).

    Domain [-up_len, L] x [0, height].  y faces grow geometrically from dy_min
    with the ratio solved so that ny cells span exactly `height`; x faces are
    clustered at the leading edge by two geometric runs (upstream and along the
    plate), each ratio solved to fit its length.  Boundaries: inflow
    equilibrium (west, north), zero-gradient outflow (east; `outflow` =
    "outflow_neq" for the set-density outflow), symmetry before the plate and a
    no-slip wall on it (south).  Fluid starts at the free stream.
    """
    nu = U * L / Re_L
    if dy_min is None:
        dy_min = L / 5000.0
    if dx_min is None:
        dx_min = L / 2000.0
    ry = solve_geometric_ratio(ny, dy_min, height)
    yf = geometric_faces(ny, 0.0, dy_min, ry)
    yf[-1] = height
    rp = solve_geometric_ratio(nx_plate, dx_min, L)
    ru = solve_geometric_ratio(nx_up, dx_min, up_len)
    plate = geometric_faces(nx_plate, 0.0, dx_min, rp)
    plate[-1] = L
    up = -geometric_faces(nx_up, 0.0, dx_min, ru)[::-1]
    up[0] = -up_len
    xf = np.concatenate([up[:-1], plate])
    nx = len(xf) - 1
    tau = nu / RT_LATTICE
    dt = cfl_dt(xf, yf, cfl)
    inflow = ("inflow", -INF, INF, 1.0, U, 0.0)
    bc = [[inflow], [(outflow, -INF, INF, 1.0, 0.0, 0.0)],
          [("symmetry", -INF, 0.0, 1.0, 0.0, 0.0), ("wall", 0.0, INF, 1.0, 0.0, 0.0)],
          [inflow]]
    case = dict(nx=nx, ny=ny, xf=xf, yf=yf, RT=RT_LATTICE, tau=tau, dt=dt, scheme=scheme, bc=bc,
                nu=nu, U=U, ry=ry, name=f"flat plate {nx}x{ny}")
    return case, (np.ones((ny, nx)), np.full((ny, nx), U), np.zeros((ny, nx)))


def flat_plate_paper(dy_min: float, cfl: float = 0.5, scheme: str = "dugks", outflow: str = "outflow"):
    """The flat-plate set-up of Sec 3.3: U0 = 0.1, L = 94.76, Re = 1e5; y cells
    grow by 1.1 from dy_min, as many as needed for a height just above 50;
    120 x cells, 80 on the plate, from dx_min = 0.1 at the leading edge,
    growing by 1.1 upstream (40 cells) and, on the plate, by the ratio that
    fits L (1.049, where the paper prints 1.05)."""
    ny = int(math.ceil(math.log(1.0 + 50.0 * 0.1 / dy_min) / math.log(1.1)))
    height = dy_min * (1.1 ** ny - 1.0) / 0.1
    up_len = 0.1 * (1.1 ** 40 - 1.0) / 0.1
    return flat_plate(nx_up=40, nx_plate=80, ny=ny, U=0.1, Re_L=1e5, L=94.76, dy_min=dy_min,
                      height=height, up_len=up_len, dx_min=0.1, cfl=cfl, scheme=scheme,
                      outflow=outflow)


def solve_geometric_ratio(n: int, d0: float, length: float) -> float:
    """Ratio r with d0 (r^n - 1)/(r - 1) = length (bisection)."""
    if abs(d0 * n - length) <= 1e-15 * length:
        return 1.0
    lo, hi = (1.0 + 1e-15, 10.0) if d0 * n < length else (1e-6, 1.0 - 1e-15)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        val = d0 * (mid ** n - 1.0) / (mid - 1.0)
        if (val < length) == (d0 * n < length):
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


# --------------------------------------------------------------------------
# Random perturbations and batched case tables
# --------------------------------------------------------------------------

def random_state(case, seed: int, amp_u: float = 0.02, amp_rho: float = 0.01,
                 amp_neq: float = 0.0):
    """Smooth-free random macroscopic fields and an optional random
    non-equilibrium offset delta[9, ny, nx] (scaled per direction by amp_neq)."""
    rng = np.random.default_rng(seed)
    ny, nx = case["ny"], case["nx"]
    rho = 1.0 + amp_rho * rng.uniform(-1, 1, (ny, nx))
    ux = amp_u * rng.uniform(-1, 1, (ny, nx))
    uy = amp_u * rng.uniform(-1, 1, (ny, nx))
    delta = amp_neq * rng.uniform(-1, 1, (9, ny, nx))
    return (rho, ux, uy), delta


class SplitMix64:
    """splitmix64 (Steele, Lea, Flood 2014): state += 0x9E3779B97F4A7C15, then
    the two xor-shift-multiply rounds and a final xor-shift."""

    M = (1 << 64) - 1

    def __init__(self, seed: int):
        self.s = seed & self.M

    def next_u64(self) -> int:
        self.s = (self.s + 0x9E3779B97F4A7C15) & self.M
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.M
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))


def batched_cases(ncases: int = 512, seed: int = 1511, side_max: int = 512,
                  side_step: int = 32):
    """The batched workload: half Taylor-Green boxes, half cavities; schemes
    alternate DUGKS / BKG; side uniform over multiples of side_step in
    [side_step, side_max]; Re log-uniform in [100, 5000]; CFL uniform in
    [0.1, 0.95].  Returns a list of (case, fields)."""
    g = SplitMix64(seed)
    out = []
    nsides = side_max // side_step
    for i in range(ncases):
        side = side_step * (1 + min(int(g.uniform() * nsides), nsides - 1))
        Re = 10.0 ** (2.0 + g.uniform() * (math.log10(5000.0) - 2.0))
        cfl = 0.1 + 0.85 * g.uniform()
        scheme = "dugks" if i % 2 == 0 else "bkg"
        if i < ncases // 2:
            u0 = 0.01
            # Re = u0 * 2 pi / nu for the 2 pi periodic box
            nu = u0 * 2.0 * math.pi / Re
            case, fields = taylor_green_box(side, u0=u0, nu=nu, cfl=cfl, scheme=scheme)
        else:
            case, fields = cavity(side, Re=Re, cfl=cfl, scheme=scheme)
        case["Re"] = Re
        case["cfl"] = cfl
        out.append((case, fields))
    return out


def cavity_at_ratio(point, ratio: float):
    """Lid-driven cavity for the stability map (Sec 3.2, Fig. cavity_stab):
    point = (scheme, n, cfl); lid U = 0.1 c, fluid at rest (impulsive start),
    n x n uniform mesh, dt from the CFL number and tau = dt / ratio (so
    nu = tau RT and Re = U L / nu follow from the ratio)."""
    scheme, n, cfl = point
    xf = uniform_faces(n, 0.0, 1.0)
    dt = cfl_dt(xf, xf, cfl)
    tau = dt / ratio
    Re = 0.1 * 1.0 / (tau * RT_LATTICE)
    case, fields = cavity(n, Re=Re, U=0.1, cfl=cfl, scheme=scheme)
    case["U"] = 0.1
    return case, fields


# ---------------------------------------------------------------- quad meshes
# Vertex arrays X, Y of shape [(ny+1), (nx+1)]; cell (i, j) has the vertices
# (i, j), (i+1, j), (i+1, j+1), (i, j+1), counter-clockwise.

def quad_from_faces(case):
    """The tensor mesh of a case dict as vertex arrays (same problem)."""
    X, Y = np.meshgrid(np.asarray(case["xf"], float), np.asarray(case["yf"], float))
    out = {k: v for k, v in case.items() if k not in ("xf", "yf")}
    out.update(X=X, Y=Y)
    return out


def quad_reindexed(case):
    """The tensor mesh of a case dict with its index directions turned: quad
    index i runs along +y, j along -x (vertex (i, j) at (xf[nx - j], yf[i])).
    Sides map W->S, E->N, S->E, N->W of the tensor problem.  Returns the quad
    case and the maps between [9, ny, nx] tensor arrays and quad arrays."""
    xf, yf = np.asarray(case["xf"], float), np.asarray(case["yf"], float)
    nx, ny = case["nx"], case["ny"]
    jj, ii = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), indexing="ij")
    X, Y = xf[nx - jj], yf[ii]
    W_, E_, S_, N_ = case["bc"]
    q = {k: v for k, v in case.items() if k not in ("xf", "yf")}
    q.update(nx=ny, ny=nx, X=X, Y=Y, bc=[S_, N_, E_, W_])

    def to_quad(a):   # tensor cell (i, j) -> quad cell (i' = j, j' = nx - 1 - i)
        return np.ascontiguousarray(np.swapaxes(a, -1, -2)[..., ::-1, :])

    def from_quad(a):
        return np.ascontiguousarray(np.swapaxes(a[..., ::-1, :], -1, -2))
    return q, to_quad, from_quad


def quad_sheared(case, s: float):
    """The tensor mesh of a case dict sheared along x: vertex (i, j) at
    (xf[i] + s (yf[j] - yf[0]), yf[j])."""
    q = quad_from_faces(case)
    q["X"] = q["X"] + s * (q["Y"] - q["Y"][0, 0])
    return q


def quad_wavy_periodic(n: int, L: float = 2 * math.pi, amp: float = 0.05):
    """Doubly periodic n x n mesh of [0, L)^2 with smooth sinusoidal
    distortion of the mesh lines (vertices x = a + A L sin(2 pi a / L)
    sin(2 pi b / L), y = b + A L sin(2 pi a / L) sin(2 pi b / L)); the sides
    stay straight and translates of one another."""
    a = np.linspace(0.0, L, n + 1)
    A, B = np.meshgrid(a, a)
    d = amp * L * np.sin(2 * math.pi * A / L) * np.sin(2 * math.pi * B / L)
    return A + d, B + d


def quad_random_interior(nx: int, ny: int, seed: int, amp: float = 0.2, L=(1.0, 1.0)):
    """A rectangle [0, Lx] x [0, Ly] with interior vertices moved at random by
    up to amp of a cell (boundary vertices slide along their side only)."""
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(np.linspace(0.0, L[0], nx + 1), np.linspace(0.0, L[1], ny + 1))
    dx, dy = L[0] / nx, L[1] / ny
    X[1:-1, 1:-1] += amp * dx * rng.uniform(-1, 1, (ny - 1, nx - 1))
    Y[1:-1, 1:-1] += amp * dy * rng.uniform(-1, 1, (ny - 1, nx - 1))
    X[[0, -1], 1:-1] += amp * dx * rng.uniform(-1, 1, (2, nx - 1))
    Y[1:-1, [0, -1]] += amp * dy * rng.uniform(-1, 1, (ny - 1, 2))
    return X, Y


def quad_min_edge(X, Y):
    """Shortest cell edge of a vertex mesh."""
    ex = np.hypot(np.diff(X, axis=1), np.diff(Y, axis=1))
    ey = np.hypot(np.diff(X, axis=0), np.diff(Y, axis=0))
    return float(min(ex.min(), ey.min()))


def taylor_green_quad(n: int, amp: float = 0.05, u0: float = 0.01, cfl: float = 0.5,
                      dt_over_tau: float = 10.0, scheme: str = "dugks"):
    """The Taylor-Green box on the wavy doubly periodic n x n mesh of
    [0, 2 pi)^2: the analytic fields at the cells' vertex-mean points, dt
    from the CFL number on the shortest edge, tau = dt / dt_over_tau."""
    X, Y = quad_wavy_periodic(n, L=2 * math.pi, amp=amp)
    x = 0.25 * (X[:-1, :-1] + X[:-1, 1:] + X[1:, 1:] + X[1:, :-1])
    y = 0.25 * (Y[:-1, :-1] + Y[:-1, 1:] + Y[1:, 1:] + Y[1:, :-1])
    dt = cfl * quad_min_edge(X, Y) / math.sqrt(6.0 * RT_LATTICE)
    tau = dt / dt_over_tau
    case = dict(nx=n, ny=n, X=X, Y=Y, RT=RT_LATTICE, tau=tau, dt=dt, scheme=scheme, bc=periodic_bc(),
                nu=tau * RT_LATTICE, u0=u0, name=f"taylor-green wavy quad {n}x{n}")
    rho = 1.0 - u0 * u0 * (np.cos(2 * x) + np.cos(2 * y)) / 4.0 / RT_LATTICE
    return case, (rho, -u0 * np.cos(x) * np.sin(y), u0 * np.sin(x) * np.cos(y))
