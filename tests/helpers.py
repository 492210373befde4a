"""Test helpers: build an oracle or a GPU solver from a seeded scenario.

Only the seeded inputs (``paper_1611_05984_gb300.scenarios``) are shared by the
two sides; each side computes the method on its own.
"""
from __future__ import annotations

import numpy as np

from paper_1611_05984_gb300 import scenarios as sc


def oracle_from(s: sc.Scenario, **over):
    import oracle
    kw = dict(model=s.model, g=s.g, Bd=s.Bd, theta=s.theta, eps=s.eps, K=s.K,
              ws=s.ws, friction=s.friction, fcoef=s.fcoef)
    kw.update(over)
    o = oracle.Oracle(s.z, s.dx, s.dy, s.dt, **kw)
    for side, sd in s.sides.items():
        o.set_boundary(side, sd.type, sd.width, sd.comps)
    o.set_state(*s.initial_state())
    for (H, th, x0, y0) in s.solitons:
        o.add_solitary(H, th, x0, y0)
    return o


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def tilted_bed_scenario(model=0, K=1, friction=1, nsteps=10, sine=False):
    """A state away from the method's kinks over an undulating bed: a tilted
    free surface and discharge with cubic terms and a short ripple, every
    slope of one sign (depth 0.35-0.6 m on 48 x 36 cells of 0.5 m, wet
    everywhere), a sponge on the east, walls elsewhere, optionally a sine
    maker on the west.  Returns (scenario, gauges, X, Y)."""
    import math
    nx, ny, dx, d0 = 48, 36, 0.5, 0.5
    dt = 0.1 * dx / math.sqrt(9.81 * d0)
    s = sc.flat_basin(nx, ny, dx, d0, dt, model=model, K=K, friction=friction, fcoef=0.01, eps=1e-8)
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx)
    xs, ys = X / (nx * dx), Y / (ny * dx)
    s.w0 = 0.04 * xs + 0.03 * xs ** 3 + 0.02 * ys + 0.015 * ys ** 3 + 0.004 * xs * ys \
        + 3e-4 * np.sin(2 * math.pi * X / 4.0) * np.sin(2 * math.pi * Y / 4.0)
    s.P0 = 0.02 + 0.01 * xs + 0.01 * xs ** 3
    s.Q0 = 0.01 + 0.005 * ys + 0.006 * ys ** 3
    s.z = -0.5 + 0.08 * xs + 0.04 * ys ** 2 + 0.01 * np.sin(2 * math.pi * X / 6.0) * np.cos(2 * math.pi * Y / 9.0)
    s.sides[sc.E] = sc.Side(sc.SPONGE, 6)
    if sine:
        s.sides[sc.W] = sc.Side(sc.SINE, 0, ((0.002, 4.0, 0.2, 0.3),))
    s.steps = nsteps
    rng = np.random.default_rng(9)
    gauges = [(int(rng.integers(4, nx - 4)), int(rng.integers(3, ny - 3))) for _ in range(6)]
    return s, gauges, X, Y


def tangent_run(s, gauges, dz, dw, dP=None, dQ=None):
    """The tangent-linear oracle over scenario s: (eta, d eta) at the gauges
    after steps 1..s.steps for the input direction (dz, dw, dP, dQ)."""
    import oracle
    t = oracle.TangentOracle(s.z, dz, s.dx, s.dy, s.dt, model=s.model, g=s.g, Bd=s.Bd, theta=s.theta,
                             eps=s.eps, K=s.K, ws=s.ws, friction=s.friction, fcoef=s.fcoef)
    for side, sd in s.sides.items():
        t.set_boundary(side, sd.type, sd.width, sd.comps)
    w, P, Q = s.initial_state()
    zero = np.zeros_like(w)
    t.set_state(w, P, Q, dw, zero if dP is None else dP, zero if dQ is None else dQ)
    t.set_gauges(gauges, 1, s.steps)
    t.step(s.steps)
    return t.read_gauges(s.steps)
