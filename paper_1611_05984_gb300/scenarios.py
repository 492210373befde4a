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
