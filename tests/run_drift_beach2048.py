"""Drift of the CUDA path against the FP64 oracle over the full run of the
2048 x 2048 beach (10,000 steps, dt = 0.0101 s, about 101 s of simulated
time, 12.6 wave periods): relative L2 of eta = w - w_s, and of P and Q,
every 500 steps.

The oracle needs about 4.2e10 cell-updates for this run, an hour or more of
CPU, so the script runs in phases that share nothing but files of sampled
values:

  python tests/run_drift_beach2048.py gpu SAMPLES.npz [--steps N] [--every K]
      steps the CUDA library (FP32 and FP64, the benchmark's launch
      configuration) and keeps eta, P and Q of a fixed seeded sample of 1/32
      of the cells (131,072 cells) every K steps in FP32, and eta every 2K
      steps in FP64;
  python tests/run_drift_beach2048.py oracle ORACLE.npz [--steps N] [--every K]
      runs the oracle over the same steps on this host's cores and keeps the
      same cells every K steps (the file grows as the run goes);
  python tests/run_drift_beach2048.py compare SAMPLES.npz ORACLE.npz DRIFT.json
      writes, per snapshot, the relative L2 over the sampled cells of each
      GPU precision against the oracle.

The sample is drawn by numpy's default_rng(2048) without replacement, the
same cells for every snapshot; a relative L2 over 131,072 cells spread over
the whole grid estimates the full-grid one to within a few per cent of its
value.  Test infrastructure: this file runs the oracle.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def sample_cells(ncells: int, frac: int = 32) -> np.ndarray:
    rng = np.random.default_rng(2048)
    return np.sort(rng.choice(ncells, ncells // frac, replace=False))


def gpu_phase(out: str, steps: int, every: int):
    import torch

    from paper_1611_05984_gb300 import celeris
    from paper_1611_05984_gb300 import scenarios as sc
    s = sc.beach(nx=2048, ny=2048)
    idx = torch.as_tensor(sample_cells(s.cells), device="cuda")
    rec = {"every": every, "nsteps": steps}
    # FP32: eta, P and Q every `every` steps, kept in FP32; FP64: eta every
    # 2 * every steps (the file stays under 64 MB)
    for prec, dt, stride, fields in (("f32", torch.float32, 1, 3), ("f64", torch.float64, 2, 1)):
        g = celeris.from_scenario(s, dtype=dt)
        vals = []
        t0 = time.time()
        for k, done in enumerate(range(every, steps + 1, every)):
            g.step(every)
            if (k + 1) % stride == 0:
                w, P, Q = g.state()
                vals.append(torch.stack([v.reshape(-1)[idx] for v in (w, P, Q)[:fields]]).cpu().numpy())
            if not g.check_finite():
                raise RuntimeError(f"{prec}: non-finite state at step {done}")
        torch.cuda.synchronize()
        rec[prec] = np.stack(vals)                       # [snapshots, fields, cells]
        print(f"{prec}: {steps} steps in {time.time() - t0:.1f} s (with the sample reads)", flush=True)
        g.close()
    np.savez_compressed(out, **rec)


def oracle_phase(out: str, steps: int, every: int):
    from paper_1611_05984_gb300 import scenarios as sc
    from tests.helpers import oracle_from
    s = sc.beach(nx=2048, ny=2048)
    idx = sample_cells(s.cells)
    o = oracle_from(s)
    vals = []
    t0 = time.time()
    for done in range(every, steps + 1, every):
        o.step(every)
        w, P, Q = o.state()
        vals.append(np.stack([v.reshape(-1)[idx] for v in (w, P, Q)]))
        np.savez(out, every=every, nsteps=done, oracle=np.stack(vals))
        print(f"oracle step {done} ({time.time() - t0:.0f} s)", flush=True)


def compare_phase(gpu: str, orc: str, out: str):
    from paper_1611_05984_gb300 import scenarios as sc
    g, o = np.load(gpu), np.load(orc)
    every = int(g["every"])
    assert int(o["every"]) == every
    n = min(int(g["nsteps"]), int(o["nsteps"])) // every
    ws = sc.beach(nx=2048, ny=2048).ws
    res = {"workload": "beach_2048x2048", "steps": [], "every": every, "cells_sampled": int(o["oracle"].shape[2]),
           "f32": {"eta": [], "P": [], "Q": []}, "f64": {"steps": [], "eta": []}}

    def rel(a, b):
        den = np.linalg.norm(b)
        return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))

    for k in range(n):
        done = (k + 1) * every
        ref = o["oracle"][k]
        res["steps"].append(done)
        a = g["f32"][k].astype(np.float64)
        for j, name in enumerate(("eta", "P", "Q")):
            sh = ws if name == "eta" else 0.0
            res["f32"][name].append(rel(a[j] - sh, ref[j] - sh))
        if (k + 1) % 2 == 0:
            res["f64"]["steps"].append(done)
            res["f64"]["eta"].append(rel(g["f64"][(k + 1) // 2 - 1][0] - ws, ref[0] - ws))
    with open(out, "w") as f:
        json.dump(res, f, indent=1)
    for k, done in enumerate(res["steps"]):
        line = f"step {done:6d}: f32 eta {res['f32']['eta'][k]:.3e}  P {res['f32']['P'][k]:.3e}  Q {res['f32']['Q'][k]:.3e}"
        if done in res["f64"]["steps"]:
            line += f"  f64 eta {res['f64']['eta'][res['f64']['steps'].index(done)]:.3e}"
        print(line)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("phase", choices=["gpu", "oracle", "compare"])
    ap.add_argument("files", nargs="+")
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--every", type=int, default=500)
    a = ap.parse_args()
    if a.phase == "gpu":
        gpu_phase(a.files[0], a.steps, a.every)
    elif a.phase == "oracle":
        oracle_phase(a.files[0], a.steps, a.every)
    else:
        compare_phase(*a.files[:3])


if __name__ == "__main__":
    main()
