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
