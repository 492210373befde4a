"""Autotuner of the line solver's split (the per-line tridiagonal solves of
Eq. 21-23): for each class of line lengths, the rows each thread of a
register-path solve owns (2, 4 or 8, hence the block size), picked by timing.

A class is timed on an ensemble of square beach grids whose lines all have
the class's length (as many grids as make about 4 million cells), with the
ensemble's own line kernel; the candidate with the least time per line
element wins.  The choice applies to every later cel_step and ensemble
(cel_set_line_split), so ensembles and single grids keep agreeing bit for
bit.  Results are cached as JSON per device and precision.

  python -m paper_1611_05984_gb300.autotune [--precision f32|f64] [--out FILE]
"""
from __future__ import annotations

import argparse
import json
import os
import time
from typing import Dict, Iterable, Optional

from . import build as _build
from . import celeris
from . import scenarios as sc

CLASSES = (128, 256, 512, 1024, 2048)


def _candidates(n: int, real_bytes: int):
    limit = 1024 if real_bytes == 4 else 512
    out = []
    for m in (2, 4, 8):
        t = -(-(-(-n // m)) // 32) * 32
        if t <= limit:
            out.append(m)
    return out


def _time_lines(n: int, dtype, cells: int, steps: int) -> float:
    """Seconds of line solves per line element, ensemble of n x n beaches."""
    count = max(1, cells // (n * n))
    members = []
    K = 1
    for k in range(count):
        s = sc.beach(nx=n, ny=n, dx=max(1.0, 400.0 / n), seed=7000 + k, nshoal=2, sponge=max(2, n // 16))
        K = s.K
        members.append(celeris.from_scenario(s, dtype=dtype))
    ens = celeris.Ensemble(members, stream=members[0].stream)
    ens.step(8)                                       # Euler start-up and the history
    ens.profile_enable(8 * 2 * steps + 16)
    ens.step(steps)
    prof = ens.profile_read()
    ens.profile_disable()
    ens.close()
    for m in members:
        m.close()
    ms, _ = prof["lines"]
    elements = steps * (K + 1) * 2 * n * n * count
    return ms * 1e-3 / elements


def tune(precision: str = "f32", classes: Iterable[int] = CLASSES, cells: int = 1 << 22, steps: int = 6,
         out: Optional[str] = None) -> Dict:
    """Time every candidate of every class and install the fastest; returns
    (and writes to `out`) {"device", "precision", "classes": [[rows, rows
    per thread, ps per element of each candidate], ...]}."""
    import torch
    dtype = torch.float32 if precision == "f32" else torch.float64
    rb = 4 if precision == "f32" else 8
    celeris.reset_line_splits()
    table = []
    t0 = time.time()
    for n in classes:
        times = {}
        for m in _candidates(n, rb):
            celeris.set_line_split(rb, n, m)
            times[m] = _time_lines(n, dtype, cells, steps)
        best = min(times, key=times.get)
        celeris.set_line_split(rb, n, best)
        table.append([n, best, {str(m): round(t * 1e12, 3) for m, t in times.items()}])
    res = {"device": torch.cuda.get_device_name(), "precision": precision, "classes": table,
           "seconds": round(time.time() - t0, 1),
           "what": "rows per thread of the line solver per class of line lengths (the class's largest length), "
                   "the fastest of the candidates, timed on ensembles of square beaches; ps per line element"}
    if out:
        os.makedirs(os.path.dirname(os.path.abspath(out)), exist_ok=True)
        with open(out, "w") as f:
            json.dump(res, f, indent=1)
    return res


def apply(table) -> None:
    """Install a tuned table (the dict tune() returns, or the path of its JSON)."""
    if isinstance(table, str):
        with open(table) as f:
            table = json.load(f)
    rb = 4 if table["precision"] == "f32" else 8
    for n, m, *_ in table["classes"]:
        celeris.set_line_split(rb, int(n), int(m))


def default_cache(precision: str) -> str:
    import torch
    name = "".join(c if c.isalnum() else "_" for c in torch.cuda.get_device_name())
    return os.path.join(_build.OUT_DIR, f"line_splits_{name}_{precision}.json")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = tune(a.precision, out=a.out or default_cache(a.precision))
    print(json.dumps(res))


if __name__ == "__main__":
    main()
