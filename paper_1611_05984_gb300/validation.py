"""The paper's three validation set-ups (Sec. 4) run on the GPU path.

The laboratory records (Synolakis, Whalin, Briggs et al.) are not available,
so this prints what the solver computes on the rebuilt geometries, for a
reader to compare with the paper's figures:

  * planar beach (Sec. 4.1): maximum vertical run-up R / d of solitary waves
    on a 1:19.85 slope for a range of H / d and friction factors, beside the
    run-up law R / d = 2.831 sqrt(cot beta) (H / d)^(5/4) for non-breaking
    waves (Synolakis 1987);
  * Whalin's shoal (Sec. 4.2): amplitudes of the first three harmonics of
    eta along the tank's centreline (FFT over whole wave periods);
  * conical island (Sec. 4.3): horizontal run-up around the island, scaled by
    the initial shoreline radius (2.32 m), and the largest elevation at four
    gauges (front toe, front, side and back shorelines).

Run-up uses the tracking of ``Solver.runup_enable`` with delta = s dx / 3.

    python -m paper_1611_05984_gb300.validation [planar|whalin|island] [--f64]
"""
from __future__ import annotations

import json
import math
import sys

import numpy as np

from . import celeris
from . import scenarios as sc


def _solver(s, dtype):
    return celeris.from_scenario(s, dtype=dtype)


def vertical_runup(maxw, bed, ws=0.0):
    """Highest water level reached on initially dry cells (bed above w_s),
    relative to w_s; 0 if the water never got above the still shoreline."""
    land = (bed > ws) & np.isfinite(maxw)
    return float(np.max(maxw[land]) - ws) if np.any(land) else 0.0


def horizontal_runup(maxw, bed, center, dx, nangle=36, ws=0.0):
    """Per direction around the island (0 = west face, counter-clockwise in
    steps of 360 / nangle degrees): the smallest distance from the centre of
    an initially dry cell that was ever wet, or of the first wet cell if none."""
    ny, nx = maxw.shape
    X, Y = np.meshgrid((np.arange(nx) + 0.5) * dx, (np.arange(ny) + 0.5) * dx)
    r = np.hypot(X - center[0], Y - center[1])
    ang = np.mod(np.arctan2(Y - center[1], -(X - center[0])), 2 * math.pi)
    sector = np.minimum((ang / (2 * math.pi) * nangle).astype(int), nangle - 1)
    wet = np.isfinite(maxw)
    out = []
    for k in range(nangle):
        m = (sector == k) & wet & (r < 3.6)
        out.append(float(np.min(r[m])) if np.any(m) else float("nan"))
    return out


def planar(dtype, cases=((0.005, 0.0), (0.01, 0.0), (0.02, 0.0), (0.05, 0.0), (0.1, 0.0), (0.2, 0.0),
                         (0.28, 0.0), (0.3, 0.0), (0.3, 0.001), (0.3, 0.01), (0.4, 0.0), (0.5, 0.0))):
    import torch
    rows = []
    for H, f in cases:
        s = sc.planar_beach_soliton(H, f=f)
        g = _solver(s, dtype)
        g.runup_enable(s.runup_delta)
        g.step(s.steps)
        ok = g.check_finite()
        R = vertical_runup(g.runup().double().cpu().numpy(), g.field("Bbar").double().cpu().numpy())
        law = 2.831 * math.sqrt(19.85) * H ** 1.25
        rows.append({"H_over_d": H, "f": f, "R_over_d": R, "law_nonbreaking": law, "finite": ok,
                     "cells": s.cells, "steps": s.steps})
        del g
        torch.cuda.empty_cache()
    return rows


def whalin(dtype, periods_skip=10, periods=4):
    s = sc.whalin()
    g = _solver(s, dtype)
    T = 2.0
    n_skip = int(round(periods_skip * T / s.dt))
    n_rec = int(round(periods * T / s.dt))
    j = s.ny // 2
    stride = 8
    ii = np.arange(0, s.nx, stride)
    g.set_gauges([(int(i), j) for i in ii], 10, n_rec // 10 + 1)
    g.step(n_skip)
    g.read_gauges(n_rec // 10 + 1)        # drop the spin-up records
    g.step(n_rec)
    rec = g.read_gauges(n_rec // 10 + 1)  # (records, gauges), one every 10 steps
    spec = np.abs(np.fft.rfft(rec - rec.mean(0), axis=0)) * 2.0 / rec.shape[0]
    base = periods                        # bin of the wave frequency
    harm = {f"h{m}": [float(v) for v in spec[m * base]] for m in (1, 2, 3)}
    return {"x": [float((i + 0.5) * s.dx) for i in ii], "a": 0.0075, "finite": g.check_finite(),
            "records": int(rec.shape[0]), **harm}


def island(dtype, cases=(0.04, 0.09, 0.18), n=601, dt=0.005):
    import torch
    out = []
    for H in cases:
        s = sc.conical_island(H, n=n, dt=dt)
        g = _solver(s, dtype)
        g.runup_enable(s.runup_delta)
        gij = [(int(x / s.dx), int(y / s.dx)) for x, y in s.gauges_xy]
        g.set_gauges(gij, 2, s.steps // 2 + 1)
        g.step(s.steps)
        ok = g.check_finite()
        maxw = g.runup().double().cpu().numpy()
        hr = horizontal_runup(maxw, g.field("Bbar").double().cpu().numpy(), s.center, s.dx)
        rec = g.read_gauges(s.steps // 2 + 1)
        out.append({"H_over_d": H, "finite": ok, "runup_radius_over_2.32": [r / 2.32 for r in hr],
                    "gauge_max_eta_over_d": [float(v) / 0.32 for v in rec.max(0)],
                    "gauges": ["front toe", "front shore", "side shore", "back shore"],
                    "vertical_runup_over_d": vertical_runup(maxw, g.field("Bbar").double().cpu().numpy()) / 0.32})
        del g
        torch.cuda.empty_cache()
    return out


def main(argv):
    import torch
    dtype = torch.float64 if "--f64" in argv else torch.float32
    which = [a for a in argv if not a.startswith("--")] or ["planar", "whalin", "island"]
    res = {}
    for w in which:
        res[w] = {"planar": planar, "whalin": whalin, "island": island}[w](dtype)
    print(json.dumps(res))


if __name__ == "__main__":
    main(sys.argv[1:])
