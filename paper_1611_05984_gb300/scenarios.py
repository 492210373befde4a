"""Seeded synthetic workloads for the Celeris step (arXiv 1611.05984).

This module only *generates inputs*: bed elevations, boundary/forcing settings
and initial states, as plain numpy arrays and numbers.  It holds none of the
method's arithmetic (no reconstruction, flux, bed corners, depths or solves),
so that the CUDA path and the CPU oracle can both be fed the very same inputs
without sharing any part of the method.

Workloads (the paper's validation data are not available, so every input is
synthetic; the shapes follow the paper's problem statement):
  * ``soliton_channel``  solitary wave on a flat 1 m channel, solid walls
    (Sec. 2.7 soliton, Sec. 2.4.1 walls).
  * ``beach``            1:30 planar beach (offshore depth 10 m) plus seeded
    Gaussian shoals, sine-wave maker on the west side (Sec. 2.4.2), sponge
    layers on north and south (Sec. 2.4.3), solid east wall behind dry land,
    Manning friction (Sec. 2.6).
  * ``beach_directional`` the same generator with several superposed sine
    components of random period, direction and phase.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Tuple

import numpy as np

G = 9.81
SOLID, SPONGE, SINE = 0, 1, 2
W, E, S, N = 0, 1, 2, 3


@dataclasses.dataclass
class Side:
    type: int = SOLID
    width: int = 0
    comps: Tuple[Tuple[float, float, float, float], ...] = ()  # (amp, T, dir, phase)


@dataclasses.dataclass
class Scenario:
    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    dt: float
    z: np.ndarray                      # (ny, nx) float64, cell-centre bed
    steps: int
    model: int = 0                     # 0 = Boussinesq, 1 = NLSW
    g: float = G
    Bd: float = 1.0 / 15.0
    theta: float = 1.3
    eps: float = 5e-12
    K: int = 0
    ws: float = 0.0
    friction: int = 0                  # 0 none, 1 quadratic, 2 Manning
    fcoef: float = 0.0
    sides: Dict[int, Side] = dataclasses.field(default_factory=dict)
    solitons: List[Tuple[float, float, float, float]] = dataclasses.field(default_factory=list)
    w0: Optional[np.ndarray] = None    # initial state; None -> rest
    P0: Optional[np.ndarray] = None
    Q0: Optional[np.ndarray] = None

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def initial_state(self):
        """(w, P, Q) at t=0.  Rest is w = w_s everywhere; the solver raises w to
        the bed on land when the state is set."""
        sh = (self.ny, self.nx)
        w = np.full(sh, self.ws) if self.w0 is None else np.asarray(self.w0, np.float64)
        P = np.zeros(sh) if self.P0 is None else np.asarray(self.P0, np.float64)
        Q = np.zeros(sh) if self.Q0 is None else np.asarray(self.Q0, np.float64)
        return w, P, Q


def courant_dt(cr: float, dx: float, dy: float, dmax: float, g: float = G) -> float:
    """Fixed step from a Courant number and the deepest still water."""
    return cr * min(dx, dy) / math.sqrt(g * dmax)


def make_beach(nx: int, ny: int, dx: float, slope: float = 1.0 / 30.0,
               d0: float = 10.0, nshoal: int = 8, seed: int = 2,
               dy: Optional[float] = None) -> np.ndarray:
    """Planar beach rising to the east plus Gaussian shoals.

    z = max(-d0, slope (x - x_s)) with the still-water shoreline at
    x_s = 0.85 L_x, plus nshoal shoals H_k exp(-r^2/W_k^2), H_k ~ U(1,4) m,
    W_k ~ U(20,80) m, centres uniform in x in [0.1 L_x, x_s - 0.1 L_x],
    y in [0.1 L_y, 0.9 L_y].  Returns (ny, nx) float64.
    """
    dy = dx if dy is None else dy
    rng = np.random.default_rng(seed)
    Lx, Ly = nx * dx, ny * dy
    xs = 0.85 * Lx
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    X, Y = np.meshgrid(x, y)
    z = np.maximum(-d0, (X - xs) * slope)
    Hk = rng.uniform(1.0, 4.0, nshoal)
    Wk = rng.uniform(20.0, 80.0, nshoal)
    xk = rng.uniform(0.1 * Lx, max(xs - 0.1 * Lx, 0.1 * Lx), nshoal)
    yk = rng.uniform(0.1 * Ly, 0.9 * Ly, nshoal)
    for k in range(nshoal):
        r2 = (X - xk[k]) ** 2 + (Y - yk[k]) ** 2
        z = z + Hk[k] * np.exp(-r2 / Wk[k] ** 2)
    return np.ascontiguousarray(z)


def soliton_channel(nx: int = 256, ny: int = 32, dx: float = 0.05, H: float = 0.1,
                    x0: float = 6.4, K: int = 0, steps: int = 1000,
                    cr: float = 0.2) -> Scenario:
    """Solitary wave (H = 0.1 m) on a flat 1 m channel with solid walls."""
    z = np.full((ny, nx), -1.0)
    dt = courant_dt(cr, dx, dx, 1.0)
    return Scenario(name=f"soliton_channel_{nx}x{ny}", nx=nx, ny=ny, dx=dx, dy=dx,
                    dt=dt, z=z, steps=steps, K=K,
                    sides={s: Side(SOLID) for s in (W, E, S, N)},
                    solitons=[(H, 0.0, x0, 0.5 * ny * dx)])


def beach(nx: int = 2048, ny: int = 2048, dx: float = 1.0, seed: int = 2,
          nshoal: int = 8, amp: float = 0.3, period: float = 8.0,
          sponge: int = 50, manning: float = 0.015, steps: int = 10000,
          K: int = 1, cr: float = 0.1, slope: float = 1.0 / 30.0,
          d0: float = 10.0, eps: float = 1e-8) -> Scenario:
    """Beach-and-shoal grid: west sine maker, north/south sponges, east wall.

    K = 1 corrector iteration and Courant 0.1 (on the deepest still water):
    on a 2-D grid with depth/dx = 10 the predictor alone (K = 0) and any even
    K let the explicitly extrapolated mixed-derivative terms (Eq. 16-17) grow
    without bound, and the AB3/AM4 pair with the KP07 flux needs a Courant
    number near 0.1 at the moving shoreline.  The desingularisation tolerance
    of Eq. 14 is 1e-8 (films thinner than about 1 cm on this 1 m grid), where
    the paper's sample value 5e-12 was set for a 5 cm laboratory grid."""
    z = make_beach(nx, ny, dx, slope=slope, d0=d0, nshoal=nshoal, seed=seed)
    dt = courant_dt(cr, dx, dx, d0)
    sides = {W: Side(SINE, 0, ((amp, period, 0.0, 0.0),)), E: Side(SOLID),
             S: Side(SPONGE, sponge), N: Side(SPONGE, sponge)}
    return Scenario(name=f"beach_{nx}x{ny}", nx=nx, ny=ny, dx=dx, dy=dx, dt=dt,
                    z=z, steps=steps, K=K, friction=2, fcoef=manning, sides=sides,
                    eps=eps)


def beach_directional(nx: int = 8192, ny: int = 8192, dx: float = 1.0, seed: int = 3,
                      nshoal: int = 8, ncomp: int = 3, amp: float = 0.1,
                      sponge: int = 50, manning: float = 0.015, steps: int = 2000,
                      K: int = 1, cr: float = 0.1) -> Scenario:
    """Beach-and-shoal grid forced by ncomp superposed sine components with
    periods U(6,14) s, directions U(-30, 30) deg and phases U(0, 2 pi)."""
    sc = beach(nx, ny, dx, seed=seed, nshoal=nshoal, sponge=sponge, manning=manning,
               steps=steps, K=K, cr=cr)
    rng = np.random.default_rng(seed + 1000)
    T = rng.uniform(6.0, 14.0, ncomp)
    th = np.deg2rad(rng.uniform(-30.0, 30.0, ncomp))
    ph = rng.uniform(0.0, 2.0 * math.pi, ncomp)
    comps = tuple((amp, float(T[m]), float(th[m]), float(ph[m])) for m in range(ncomp))
    sc.sides[W] = Side(SINE, 0, comps)
    sc.name = f"beach_directional_{nx}x{ny}"
    return sc


def flat_basin(nx: int, ny: int, dx: float, depth: float, dt: float,
               dy: Optional[float] = None, **kw) -> Scenario:
    """Flat bed at -depth with solid walls everywhere (used by invariant tests)."""
    dy = dx if dy is None else dy
    z = np.full((ny, nx), -depth)
    return Scenario(name=f"flat_{nx}x{ny}", nx=nx, ny=ny, dx=dx, dy=dy, dt=dt, z=z,
                    steps=0, sides={s: Side(SOLID) for s in (W, E, S, N)}, **kw)


def random_bed(nx: int, ny: int, seed: int, lo: float, hi: float,
               smooth: int = 2) -> np.ndarray:
    """Seeded random bed in [lo, hi], box-smoothed `smooth` times."""
    rng = np.random.default_rng(seed)
    z = rng.uniform(lo, hi, (ny, nx))
    for _ in range(smooth):
        zp = np.pad(z, 1, mode="edge")
        z = (zp[:-2, 1:-1] + zp[2:, 1:-1] + zp[1:-1, :-2] + zp[1:-1, 2:] + zp[1:-1, 1:-1]) / 5.0
    return np.ascontiguousarray(z)


def ensemble(n: int = 256, seed: int = 4, steps: int = 5000, K: int = 1, cr: float = 0.1,
             d0: float = 10.0, nx_range=(128, 1024), ny_range=(128, 512)) -> list:
    """n beach scenarios of uneven size and forcing, for ensemble runs.

    Per scenario: n_x ~ U{128..1024}, n_y ~ U{128..512}, sine amplitude
    a ~ U(0.05, 1) m, period T ~ U(5, 15) s, beach slope ~ U(1/50, 1/10),
    shoal count ~ U{0..12}, bed seed seed * 1000 + k.  The grid spacing is
    the larger of 1 m and the spacing that puts the toe of the beach (depth
    d0) at 15 % of the domain length, so that every maker stands in water d0
    deep; dt follows from Courant cr on d0; sponges of n_y / 8 cells (at most
    50) on the north and south sides."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        nx = int(rng.integers(nx_range[0], nx_range[1] + 1))
        ny = int(rng.integers(ny_range[0], ny_range[1] + 1))
        a = float(rng.uniform(0.05, 1.0))
        T = float(rng.uniform(5.0, 15.0))
        slope = float(rng.uniform(1.0 / 50.0, 1.0 / 10.0))
        nshoal = int(rng.integers(0, 13))
        dx = max(1.0, math.ceil(d0 / slope / (0.7 * nx) * 4.0) / 4.0)
        sc = beach(nx, ny, dx, seed=seed * 1000 + k, nshoal=nshoal, amp=a, period=T,
                   sponge=min(50, ny // 8), steps=steps, K=K, cr=cr, slope=slope, d0=d0)
        sc.name = f"ensemble{k}_{nx}x{ny}"
        out.append(sc)
    return out


# ----------------------------------------------------------------------
# The paper's validation geometries (Sec. 4), as synthetic workloads: the
# laboratory records are not available, so only the set-ups are rebuilt.

def whalin(nx: int = 2000, ny: int = 65, a: float = 0.0075, period: float = 2.0,
           dt: float = 0.001, K: int = 1, steps: int = 20000, sponge_m: float = 5.0) -> Scenario:
    """Whalin's semicircular shoal (Sec. 4.2, Eq. 37): a 35 m x 6.096 m
    tank, still water 0.4572 m deep over the flat part, the bed rising by
    1/25 between x = 10.67 - G(y) and 18.29 - G(y) to 0.3048 m
    (G(y) = sqrt(y (6.096 - y))), so the shallow end is 0.1524 m deep.  Sine
    maker on the west (a = 0.0075 m, T = 2 s), a 5 m sponge on the east, walls
    north and south, dt = 0.001 s on 2000 x 65 cells.  Eq. 37 prints the
    ramp as (10.67 - G - x)/25, which is negative on its own interval; the
    ramp that reaches 0.3048 m at x = 18.29 - G is (x - 10.67 + G)/25.  K = 1
    (an odd corrector count keeps the explicit mixed terms stable at
    depth/dx = 26)."""
    Lx, Ly, h0 = 35.0, 6.096, 0.4572
    dx, dy = Lx / nx, Ly / ny
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dy)
    Gy = np.sqrt(Y * (Ly - Y))
    rise = np.clip((X - 10.67 + Gy) / 25.0, 0.0, 0.3048)
    z = -h0 + rise
    sides = {W: Side(SINE, 0, ((a, period, 0.0, 0.0),)), E: Side(SPONGE, int(round(sponge_m / dx))),
             S: Side(SOLID), N: Side(SOLID)}
    return Scenario(name=f"whalin_{nx}x{ny}", nx=nx, ny=ny, dx=dx, dy=dy, dt=dt, z=z, steps=steps, K=K,
                    sides=sides)


def planar_beach_soliton(H_over_d: float = 0.28, d: float = 1.0, slope: float = 1.0 / 19.85,
                         f: float = 0.0, K: int = 1, eps: float = 1e-8) -> Scenario:
    """Solitary-wave run-up on a planar beach (Sec. 4.1): slope 1:19.85,
    still-water depth d, dx / d = 0.25 and dt sqrt(g/d) = 0.03 (dx / d =
    0.0625 and dt sqrt(g/d) = 0.0075 for H/d < 0.01), a tank one depth wide,
    sponge on the west, walls elsewhere, quadratic friction f.  The beach sits
    near the east end; the tank holds a 20 d sponge, the soliton (centred one
    half-length, arccosh(sqrt(20)) / gamma with gamma = sqrt(3H/(4d^3)), off the
    toe) and land up to 1.5 d above the still water."""
    fine = H_over_d < 0.01
    dx = (0.0625 if fine else 0.25) * d
    dt = (0.0075 if fine else 0.03) * math.sqrt(d / G)
    H = H_over_d * d
    half = math.acosh(math.sqrt(20.0)) / math.sqrt(3.0 * H / (4.0 * d ** 3))
    sponge = 20.0 * d
    x_toe = sponge + 2.0 * half + 2.0 * d
    x_top = x_toe + 2.5 * d / slope           # land rises to 1.5 d above the still water
    nx = int(math.ceil(x_top / dx))
    ny = max(4, int(round(d / dx)))
    x = (np.arange(nx) + 0.5) * dx
    z = np.tile(np.maximum(-d, -d + (x - x_toe) * slope), (ny, 1))
    sides = {W: Side(SPONGE, int(round(sponge / dx))), E: Side(SOLID), S: Side(SOLID), N: Side(SOLID)}
    sc = Scenario(name=f"planar_beach_H{H_over_d:g}", nx=nx, ny=ny, dx=dx, dy=dx, dt=dt, z=z,
                  steps=int(round(((x_toe + d / slope - (x_toe - half)) / math.sqrt(G * d)
                                   + 40.0 * math.sqrt(d / G)) / dt)), K=K, friction=1 if f > 0 else 0, fcoef=f,
                  sides=sides, eps=eps, solitons=[(H, 0.0, x_toe - half, 0.5 * ny * dx)])
    sc.runup_delta = slope * dx / 3.0
    return sc


def conical_island(H_over_d: float = 0.09, n: int = 601, dt: float = 0.005, K: int = 1,
                   eps: float = 1e-10) -> Scenario:
    """Solitary wave on a conical island (Sec. 4.3): a 30 m x 30 m domain on
    n x n cells, still water 0.32 m deep, an island of 7.2 m base diameter
    and 1/4 side slope at the centre (shoreline radius 2.32 m), a soliton of
    height H near the west side, sponges west and east (parallel to the
    crest), walls north and south, no friction, dt = 0.005 s.  The text gives
    no island top; the cone is cut flat at 0.625 m above the tank floor (a top
    diameter of 2.2 m), above any run-up of these cases."""
    L, d = 30.0, 0.32
    dx = L / n
    X, Y = np.meshgrid((np.arange(n) + 0.5) * dx, (np.arange(n) + 0.5) * dx)
    r = np.hypot(X - 0.5 * L, Y - 0.5 * L)
    z = -d + np.clip((3.6 - r) / 4.0, 0.0, 0.625)
    H = H_over_d * d
    half = math.acosh(math.sqrt(20.0)) / math.sqrt(3.0 * H / (4.0 * d ** 3))
    sponge = 1.5
    x0 = sponge + half
    sides = {W: Side(SPONGE, int(round(sponge / dx))), E: Side(SPONGE, int(round(sponge / dx))),
             S: Side(SOLID), N: Side(SOLID)}
    sc = Scenario(name=f"conical_island_H{H_over_d:g}_{n}", nx=n, ny=n, dx=dx, dy=dx, dt=dt, z=z,
                  steps=int(round(20.0 / dt)), K=K, sides=sides, eps=eps, solitons=[(H, 0.0, x0, 0.5 * L)])
    sc.runup_delta = 0.25 * dx / 3.0
    sc.center = (0.5 * L, 0.5 * L)
    # gauges by role: the toe in front, the shoreline in front, on the north
    # side and behind (the paper's gauge numbers refer to its Fig. 10)
    sc.gauges_xy = [(0.5 * L - 3.6 - 0.5, 0.5 * L), (0.5 * L - 2.32 - 0.1, 0.5 * L),
                    (0.5 * L, 0.5 * L + 2.32 + 0.1), (0.5 * L + 2.32 + 0.1, 0.5 * L)]
    return sc


def partition(cells, parts: int) -> list:
    """Indices of the items split into `parts` groups of nearly equal total
    cells: largest first, each to the group with the fewest cells so far
    (ties to the lowest group).  Every index appears exactly once."""
    groups = [[] for _ in range(parts)]
    load = [0] * parts
    for k in sorted(range(len(cells)), key=lambda k: (-cells[k], k)):
        g = min(range(parts), key=lambda r: (load[r], r))
        groups[g].append(k)
        load[g] += cells[k]
    return [sorted(g) for g in groups]


def hump_beach(n: int = 512, seed: int = 5, steps: int = 2000, H: float = 0.5, width: float = 30.0,
               ngauges: int = 16, K: int = 1, cr: float = 0.1):
    """Gauge-misfit workload for the adjoint: the beach-and-shoal bed
    (make_beach, seed 5) on n x n cells of 1 m, a Gaussian hump of water
    H exp(-r^2 / width^2) offshore as the initial state, sponges on the west,
    north and south, a wall behind the dry east, Manning 0.015, K = 1,
    Courant 0.1, and ngauges seeded gauges in water deeper than 2 m.
    Returns (scenario, gauges)."""
    sc = beach(n, n, 1.0, seed=seed, steps=steps, K=K, cr=cr, sponge=min(50, n // 10))
    sc.sides[W] = Side(SPONGE, min(50, n // 10))
    X, Y = np.meshgrid(np.arange(n) + 0.5, np.arange(n) + 0.5)
    sc.w0 = np.maximum(sc.z, H * np.exp(-((X - 0.4 * n) ** 2 + (Y - 0.5 * n) ** 2) / width ** 2))
    sc.name = f"hump_beach_{n}"
    rng = np.random.default_rng(seed + 2000)
    deep = np.argwhere(sc.z < -2.0)
    pick = rng.choice(len(deep), size=ngauges, replace=False)
    gauges = [(int(deep[k][1]), int(deep[k][0])) for k in pick]
    return sc, gauges


def hump_beach_target(sc: Scenario, seed: int = 5) -> Scenario:
    """The run the misfit compares against: the hump_beach scenario with its
    hump 10 % higher and wider and moved by (8, -6) m, and its bed raised by
    4 seeded Gaussian bumps offshore (0.1-0.3 m, widths 20-40 m)."""
    import copy
    t = copy.deepcopy(sc)
    n = sc.nx
    X, Y = np.meshgrid((np.arange(n) + 0.5) * sc.dx, (np.arange(sc.ny) + 0.5) * sc.dy)
    rng = np.random.default_rng(seed + 3000)
    for _ in range(4):
        cx, cy = rng.uniform(0.15, 0.6) * n * sc.dx, rng.uniform(0.2, 0.8) * sc.ny * sc.dy
        t.z = t.z + rng.uniform(0.1, 0.3) * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / rng.uniform(20, 40) ** 2)
    hump = np.asarray(sc.w0) - np.maximum(sc.z, sc.ws)
    amp = float(hump.max())
    wid = float(np.sqrt(np.sum(hump > amp / np.e) / math.pi))   # radius where the hump falls to 1/e
    t.w0 = np.maximum(t.z, 1.1 * amp * np.exp(-((X - 0.4 * n * sc.dx - 8.0) ** 2 + (Y - 0.5 * sc.ny * sc.dy + 6.0) ** 2)
                                              / (1.1 * wid) ** 2))
    t.name = sc.name + "_target"
    return t
