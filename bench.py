#!/usr/bin/env python
"""Benchmark of the Celeris extended-Boussinesq step on GB300.

Metric: cell-updates/s (interior cells x time steps / second) of the full
time step (stencil + update, x-line and y-line tridiagonal solves, for the
AB3 predictor and the AM4 corrector stage) on the 2048 x 2048 beach-and-shoal
workload (FP32, seeded synthetic bed: 1:30 beach, 8 Gaussian shoals, sine
maker on the west, 50-cell sponges north and south, Manning n = 0.015).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  N > 1 runs N independent replicas (the single-grid
step has no natural shard: every step couples whole rows and columns through
the tridiagonal solves), one per GPU, weak scaling.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# Algorithmic values moved per cell by one launch of each kernel:
#   stencil, AB3 predictor with K >= 1 (ring history): reads w, P, Q, bed
#     corners, R^{n-1}, R^{n-2} of w, U*, V* and the mixed terms F*, G* at n-1,
#     n-2 (14); writes w, dU*, dV*, R^n (3), F*^n, G*^n and 3 AM4 bases (11);
#   stencil, AM4 corrector: reads w, P, Q, corners, 3 bases (7), writes 3;
#   stencil, predictor with K = 0 (carries a, b): reads 10, writes 9;
#   line solves (x-rows and y-columns in one launch): per family the right
#     side, depth and P^n (or Q^n) read, P^{n+1} (or Q^{n+1}) written: 2 x 4.
VALUES = {"stencil_pred_k": 14 + 11, "stencil_pred_0": 10 + 9, "stencil_corr": 7 + 3, "lines": 8}
# The same split on the contract's count of algorithmic values per cell-update
# (the method's minimum with the AB3 history held as two combined carries per
# variable, K = 0: 25 values per step; each AM4 corrector iteration about 14
# more).  The stencil's share of the predictor: w, P, Q, the bed corners, 2
# carries read and 2 written for each of w, U*, V*, w^{n+1}, U*, V* written
# (19); the line solves': U*, V* and the bed read (once per family), P, Q
# written (6); a corrector's stencil: 14 - 6 = 8.
CONTRACT = {"stencil_pred": 19, "stencil_corr": 8, "lines": 6}
# FP64: the kernels are bound by the FP64 pipe, not by memory, so the FP64
# line's roofline is arithmetic.  Double-precision operations per cell of one
# launch, 2 DFMA + DADD + DMUL, counted by ncu on the 2048^2 beach
# (smsp__sass_thread_inst_executed_op_{dfma,dadd,dmul}_pred_on.sum / cells):
# the AB3 predictor stencil, the AM4 corrector stencil, one line-solve launch
# (both families).  The peak: 2 DFMA per clock per SM x 2 x 152 SMs x 2.07 GHz.
FP64_FLOPS = {"stencil_pred": 562.6, "stencil_corr": 517.5, "lines": 117.9}
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="beach2048",
                    choices=["beach2048", "beach8192", "beach512", "whalin2000", "conical601", "ensemble256",
                             "adjoint512", "adjoint2048"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--ckpt", type=int, default=None,
                    help="adjoint workloads: checkpoint spacing (0 keeps every step; default: every step kept "
                         "where it fits in 70%% of the free memory, else 100)")
    ap.add_argument("--ensemble-steps", type=int, default=50,
                    help="default workload: steps of the ensemble measurement in the line (0: none)")
    ap.add_argument("--adjoint-steps", type=int, default=2000,
                    help="default workload: steps of the adjoint measurement in the line (0: none)")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the line solver's built-in split instead of autotuning it first")
    ap.add_argument("--dependent-launch", default="on", choices=["on", "off"],
                    help="programmatic dependent launch of the step's kernels (cel_set_dependent_launch)")
    return ap.parse_args()


def workload(name):
    from paper_1611_05984_gb300 import scenarios as sc
    if name == "beach2048":
        return sc.beach(nx=2048, ny=2048)
    if name == "beach8192":
        return sc.beach_directional(nx=8192, ny=8192)
    if name == "beach512":
        return sc.beach(nx=512, ny=512, sponge=20)
    if name == "whalin2000":
        return sc.whalin()
    if name == "conical601":
        return sc.conical_island(0.18)
    raise ValueError(f"{name} is not a single-grid workload")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.index)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _oracle_for(s):
    import oracle
    o = oracle.Oracle(s.z, s.dx, s.dy, s.dt, model=s.model, g=s.g, Bd=s.Bd, theta=s.theta, eps=s.eps,
                      K=s.K, ws=s.ws, friction=s.friction, fcoef=s.fcoef)
    for side, sd in s.sides.items():
        o.set_boundary(side, sd.type, sd.width, sd.comps)
    o.set_state(*s.initial_state())
    return o


def _row_crop(s, rows):
    """The first `rows` rows of the same bed and boundaries: the cross-shore
    profile (sine maker, shoals, beach, wall) is kept, the alongshore extent cut."""
    import copy
    if rows >= s.ny:
        return s
    c = copy.copy(s)
    c.z = s.z[:rows].copy()
    c.ny = rows
    c.sides = dict(s.sides)
    c.name = f"{s.name}[rows 0:{rows}]"
    return c


def _sample_rows(s, seconds_per_step):
    """Rows of a crop whose oracle step takes about seconds_per_step."""
    import time as _t
    probe = _row_crop(s, min(s.ny, 64))
    o = _oracle_for(probe)
    o.step(3)
    t0 = _t.perf_counter()
    o.step(2)
    per_row = (_t.perf_counter() - t0) / 2 / probe.ny
    return max(16, min(s.ny, int(seconds_per_step / max(per_row, 1e-9))))


def cpu_baseline(s, seconds):
    """The FP64 oracle, as it stands, on this host's cores: a bounded sample of
    the same workload (a row crop if a full step is too slow), timed after the
    two Euler start-up steps, about `seconds` of CPU work."""
    import oracle
    rows = _sample_rows(s, seconds / 4)
    c = _row_crop(s, rows)
    o = _oracle_for(c)
    o.step(2)
    t0 = time.perf_counter()
    n = 0
    while True:
        o.step(1)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds or n >= 50:
            break
    return {"value": c.cells * n / el, "unit": "cell-updates/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{c.name}, FP64, {n} AB3+AM4 steps after the 2 Euler start-up steps, {el:.1f} s"}


def run_reference(args):
    """Reference arm: the CPU oracle on this host (rank 0 only), each step one
    oracle step on a row crop of the workload sized to keep the run to about
    two minutes."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    if args.workload in ("ensemble256", "adjoint512", "adjoint2048"):
        print(json.dumps({"impl": "reference", "unavailable": "the oracle has no ensemble mode and no adjoint (its "
                          "tangent-linear build gives one directional derivative per run, not the gradient); "
                          "its arm runs the single-grid workloads"}), flush=True)
        return
    s = workload(args.workload)
    rows = _sample_rows(s, 120.0 / (args.steps + args.warmup + 2))
    c = _row_crop(s, rows)
    o = _oracle_for(c)
    o.step(2 + args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    v = c.cells * args.steps / el
    line = {"impl": "reference", "metric": "cell-updates/s", "value": v, "unit": "cell-updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * el / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": s.name, "nx": s.nx, "ny": s.ny, "cells": s.cells,
                       "corrector_iters": s.K, "dt": s.dt, "sample_rows": rows},
            "cpu_baseline": {"value": v, "unit": "cell-updates/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{c.name}, FP64, {args.steps} timed steps after "
                                       f"{args.warmup + 2} untimed"},
            "e2e": {"value": v, "unit": "cell-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ensemble(args):
    """The 256-scenario ensemble (uneven beaches of 128..1024 x 128..512
    cells, about 4.8e7 cells in all, FP32 by default): cell-updates/s of the
    ensemble step (one launch per kernel kind and stage over all members)
    against the same members stepped one cel_step per scenario in turn, both
    timed with CUDA events on the one stream, after the same warm-up."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:   # scenarios are independent: each rank steps its share, no data-path collective
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    line = measure_ensemble(args.steps, args.warmup, args.precision, world, rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def measure_ensemble(steps, warmup, precision, world=1, rank=0):
    """One measurement of the ensemble against one launch per scenario (see
    run_ensemble); returns the JSON object (every rank takes part)."""
    import torch
    import torch.distributed as dist

    from paper_1611_05984_gb300 import celeris
    from paper_1611_05984_gb300 import scenarios as sc

    class _A:
        pass
    args = _A()
    args.steps, args.warmup, args.precision = steps, warmup, precision

    def barrier():
        if world > 1:
            dist.barrier()

    dtype = torch.float32 if args.precision == "f32" else torch.float64
    es = 4 if args.precision == "f32" else 8
    every = sc.ensemble()
    share = celeris.ensemble_share([s.cells for s in every], rank, world)
    scens = [every[k] for k in share]
    members = [celeris.from_scenario(s, dtype=dtype) for s in scens]
    cells = sum(s.cells for s in scens)
    total_cells = sum(s.cells for s in every)
    stream = members[0].stream
    ens = celeris.Ensemble(members, stream=stream)
    for m in members:                      # the same warm-up for the one-at-a-time loop's kernels
        m.step(1)
    # then the ensemble: after 7 steps every argument block of the 6-step
    # cycle is uploaded; the next 6 capture the cycle as a graph, the rest
    # replay it, so the timed steps start at the captured cycle's phase
    ens.step(7)
    ens.step(6 * max(2, (args.warmup + 5) // 6))
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.4)
    torch.cuda.synchronize()
    # the timed steps: one call, captured 6-step cycles replayed as graphs
    g0 = ens.graph_steps()
    barrier()
    torch.cuda.synchronize()
    e[0].record(stream)
    ens.step(args.steps)
    e[1].record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = ens.last_launch_count()
    graph_steps = ens.graph_steps() - g0
    # the same steps as one persistent cooperative launch per call
    ens.use_persistent(True)
    ens.step(1)
    torch.cuda.synchronize()
    ep = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    p0 = ens.persistent_steps()
    barrier()
    torch.cuda.synchronize()
    ep[0].record(stream)
    ens.step(args.steps)
    ep[1].record(stream)
    torch.cuda.synchronize()
    barrier()
    ens.check()
    persistent_steps = ens.persistent_steps() - p0
    persistent_launches = ens.last_launch_count()
    ens.use_persistent(False)
    ms_pers = max_over_ranks(ep[0].elapsed_time(ep[1]))
    # the per-kernel split, from a short profiled run after the timed one
    # (profiling launches every kernel on its own, without graphs)
    ens.profile_enable(8 * (scens[0].K + 1) * 12 + 16)
    ens.step(12)
    prof = ens.profile_read()
    ens.profile_disable()
    prof_steps = 12
    # the same members one at a time: one cel_step of all K steps per member
    # (launch-bound on small grids, with the least host work per launch), and
    # interleaved (every member one step, K times)
    barrier()
    torch.cuda.synchronize()
    e[2].record(stream)
    single_launches = 0
    for m in members:
        m.step(args.steps)
        single_launches += m.last_launch_count()
    e[3].record(stream)
    torch.cuda.synchronize()
    barrier()
    e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e4.record(stream)
    for _ in range(args.steps):
        for m in members:
            m.step(1)
    e5.record(stream)
    torch.cuda.synchronize()
    barrier()
    # the same one-at-a-time loop with plain launches (no programmatic
    # dependent launch between the members' kernels)
    dl = celeris.dependent_launch()
    celeris.set_dependent_launch(False)
    e6, e7 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e6.record(stream)
    for m in members:
        m.step(args.steps)
    e7.record(stream)
    torch.cuda.synchronize()
    celeris.set_dependent_launch(dl)
    barrier()
    clk = clocks.stop()
    ms_ens = max_over_ranks(e[0].elapsed_time(e[1]))
    ms_runs = max_over_ranks(e[2].elapsed_time(e[3]))
    ms_inter = max_over_ranks(e4.elapsed_time(e5))
    ms_one = min(ms_runs, ms_inter)
    ms_plain = max_over_ranks(e6.elapsed_time(e7))
    finite = all(m.check_finite() for m in members)
    value = total_cells * args.steps / (ms_ens / 1e3)
    one = total_cells * args.steps / (ms_one / 1e3)
    peak, peak_src = peaks()
    # algorithmic bytes over all members: the per-cell values of the
    # single-grid kernels (predictor + K corrector stencils, K + 1 line stages)
    K = scens[0].K
    bytes_of = {"stencil": cells * es * prof_steps * (CONTRACT["stencil_pred"] + K * CONTRACT["stencil_corr"]),
                "lines": cells * es * prof_steps * (K + 1) * CONTRACT["lines"], "ghosts": 0}
    kernels = {k: {"ms_total": v[0], "launches": v[1],
                   "gbs_algorithmic": bytes_of[k] / (v[0] / 1e3) / 1e9 if v[0] > 0 and bytes_of[k] else None}
               for k, v in prof.items()}
    dominant = max(kernels, key=lambda k: kernels[k]["ms_total"])
    achieved = kernels[dominant]["gbs_algorithmic"]
    gbs = (bytes_of["stencil"] + bytes_of["lines"]) * args.steps / prof_steps / (ms_ens / 1e3) / 1e9
    ens.close()
    for m in members:
        m.close()
    line = {"metric": "ensemble cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_ens / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
            "data": "synthetic",
            "config": {"workload": "ensemble256", "members": len(every), "cells": total_cells,
                       "members_rank0": len(scens), "corrector_iters": K,
                       "parallelism": f"scenarios partitioned over {world} ranks by cell count",
                       "l2": "inputs larger than L2 (%.1f GB of workspaces)"
                             % (sum(m.workspace.numel() for m in members) / 1e9)},
            "single_launch": {"value": one, "ms_per_step": ms_one / args.steps,
                              "what": "the same members one at a time, the faster of: one cel_step(K steps) "
                                      "per member in turn, and every member one cel_step(1) per step "
                                      "(the library's default launches: programmatic dependent launch)",
                              "ms_per_step_per_member_runs": ms_runs / args.steps,
                              "ms_per_step_interleaved": ms_inter / args.steps,
                              "gpu_launches": single_launches},
            "speedup_vs_single_launch": value / one,
            "single_launch_plain": {"ms_per_step": ms_plain / args.steps, "speedup": ms_plain / ms_ens,
                                    "what": "one cel_step(K steps) per member in turn with plain launches "
                                            "(cel_set_dependent_launch(0))"},
            "roofline": {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None, "peak_source": peak_src,
                         "per_kernel": kernels, "per_kernel_from": f"a profiled run of {prof_steps} steps after "
                                                                  "the timed ones, kernel by kernel",
                         "step_gbs_algorithmic": gbs},
            "graph_steps": graph_steps, "line_splits": TUNED,
            "persistent": {"ms_per_step": ms_pers / args.steps,
                           "value": total_cells * args.steps / (ms_pers / 1e3),
                           "speedup_vs_single_launch": ms_one / ms_pers, "steps": persistent_steps,
                           "gpu_launches": persistent_launches,
                           "what": "the same steps as one persistent cooperative launch per call "
                                   "(cel_ensemble_use_persistent), grid-wide barriers between phases"},
            "finite": finite, "gpu_launches": launches, "clocks": clk}
    return line


def run_adjoint(args):
    """Cost of the discrete adjoint on the hump-on-beach workload (512^2, or
    2048^2 for adjoint2048; Boussinesq, K = 1, 16 gauges): the time of the
    gauge-misfit gradients with respect to the initial w and the bed
    (forward, reverse, and the recomputation where checkpoints are used)
    against the time of the forward steps alone, both with CUDA events on
    the solver's stream; --steps is the run length.  Every step of the
    forward run is kept where that takes at most 70 % of the free device memory
    (ckpt_every 0), else checkpoints every 100 steps; the scratch is
    allocated before the timed region.  The observations are the gauges of
    a target run from a perturbed hump over a perturbed bed."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    print(json.dumps(measure_adjoint(args.steps, args.warmup, args.precision,
                                     2048 if args.workload == "adjoint2048" else 512, args.ckpt)), flush=True)


def measure_adjoint(steps, warmup, precision, n=512, ckpt_request=None):
    """One measurement of the adjoint's cost (see run_adjoint).  ckpt_request:
    the checkpoint spacing (0 keeps every step); None picks every step kept
    where it fits in 70 % of the free memory, else 100."""
    import torch

    from paper_1611_05984_gb300 import celeris
    from paper_1611_05984_gb300 import scenarios as sc

    class _A:
        pass
    args = _A()
    args.steps, args.warmup, args.precision = steps, warmup, precision
    dtype = torch.float32 if args.precision == "f32" else torch.float64
    s, gauges = sc.hump_beach(n=n, steps=args.steps)
    g = celeris.from_scenario(s, dtype=dtype)
    stream = g.stream
    t = celeris.from_scenario(sc.hump_beach_target(s), dtype=dtype)
    t.set_gauges(gauges, 1, args.steps)
    t.step(args.steps)
    obs = torch.as_tensor(t.read_gauges(args.steps)).to(device="cuda", dtype=dtype)
    t.close()
    g.step(args.warmup)
    free, _ = torch.cuda.mem_get_info()
    if ckpt_request is None:
        ckpt = 0 if celeris.adjoint_scratch_bytes(g, args.steps, len(gauges), 0, bed=True) <= 0.7 * free else 100
    else:
        ckpt = ckpt_request
    scratch = torch.empty(celeris.adjoint_scratch_bytes(g, args.steps, len(gauges), ckpt, bed=True),
                          dtype=torch.uint8, device="cuda")
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    g.set_state(*s.initial_state())
    torch.cuda.synchronize()
    ev[0].record(stream)
    g.step(args.steps)
    ev[1].record(stream)
    torch.cuda.synchronize()
    g.set_state(*s.initial_state())
    torch.cuda.synchronize()
    ev[2].record(stream)
    loss, eta, grad, grad_z = celeris.gauge_misfit_gradient(g, args.steps, gauges, obs, ckpt_every=ckpt, bed=True,
                                                            scratch=scratch)
    ev[3].record(stream)
    torch.cuda.synchronize()
    fwd, adj = ev[0].elapsed_time(ev[1]), ev[2].elapsed_time(ev[3])
    line = {"metric": "adjoint cost / forward cost", "value": adj / fwd, "unit": "ratio", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": adj / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": args.precision,
            "data": "synthetic",
            "config": {"workload": s.name, "nx": s.nx, "ny": s.ny, "corrector_iters": s.K, "gauges": len(gauges),
                       "ckpt_every": ckpt, "scratch_gb": scratch.numel() / 1e9},
            "forward_ms_per_step": fwd / args.steps, "loss": loss,
            "grad_finite": bool(torch.isfinite(grad).all().item() and torch.isfinite(grad_z).all().item()),
            "grad_w_norm": float(torch.linalg.norm(grad.double()).item()),
            "grad_z_norm": float(torch.linalg.norm(grad_z.double()).item())}
    g.close()
    del scratch
    torch.cuda.empty_cache()
    return line


TUNED = None


def tune_lines(args):
    """The line solver's split per class of line lengths, picked by the
    project's autotuner on this GPU before anything is measured (every
    measurement below runs under it)."""
    global TUNED
    if args.no_tune:
        return
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    from paper_1611_05984_gb300 import autotune
    TUNED = autotune.tune(args.precision, cells=1 << 21, steps=4)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    from paper_1611_05984_gb300 import celeris
    celeris.set_dependent_launch(args.dependent_launch == "on")
    tune_lines(args)
    if args.workload == "ensemble256":
        run_ensemble(args)
        return
    if args.workload in ("adjoint512", "adjoint2048"):
        run_adjoint(args)
        return
    import torch
    import torch.distributed as dist

    from paper_1611_05984_gb300 import celeris

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    dtype = torch.float32 if args.precision == "f32" else torch.float64
    es = 4 if args.precision == "f32" else 8
    s = workload(args.workload)
    sol = celeris.from_scenario(s, dtype=dtype)
    stream = sol.stream
    sol.step(args.warmup)
    torch.cuda.synchronize()

    # ---- timed region: K steps, inputs resident in HBM, nothing recorded
    # between the kernels (an event between two kernels costs the step about
    # 7 %: the next launch waits for it)
    clocks = Clocks(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.4)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sol.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = sol.last_launch_count()
    ms = max_over_ranks(e0.elapsed_time(e1))
    value = whole_job_rate(s.cells, args.steps, ms)
    # ---- the per-kernel split: the same K steps again, right after, with
    # CUDA events around every kernel on the solver's stream
    sol.profile_enable(3 * (s.K + 1) * args.steps + 16)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    sol.step(args.steps)
    p1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    prof = sol.profile_read()
    sol.profile_disable()
    ms_profiled = max_over_ranks(p0.elapsed_time(p1))

    # ---- roofline of the dominant kernel (bytes per launch / event time)
    peak, peak_src = peaks()
    st_ms, st_n = prof["stencil"]
    nstages_corr = s.K * args.steps
    nstages_pred = args.steps
    pred_vals = VALUES["stencil_pred_k"] if s.K > 0 else VALUES["stencil_pred_0"]
    st_bytes = s.cells * es * (nstages_pred * pred_vals + nstages_corr * VALUES["stencil_corr"])
    kernels = {k: {"ms_total": v[0], "launches": v[1]} for k, v in prof.items()}
    dominant = max(kernels, key=lambda k: kernels[k]["ms_total"])
    line_bytes = s.cells * es * VALUES["lines"] * (nstages_pred + nstages_corr)
    # the contract's count (CONTRACT): achieved and frac are on it
    c_st = s.cells * es * (nstages_pred * CONTRACT["stencil_pred"] + nstages_corr * CONTRACT["stencil_corr"])
    c_ln = s.cells * es * CONTRACT["lines"] * (nstages_pred + nstages_corr)
    bytes_of = {"stencil": c_st, "lines": c_ln, "ghosts": 0}
    ring_of = {"stencil": st_bytes, "lines": line_bytes, "ghosts": 0}
    dk = kernels[dominant]
    achieved = bytes_of[dominant] / (dk["ms_total"] / 1e3) / 1e9 if dk["ms_total"] > 0 else 0.0
    ring_achieved = ring_of[dominant] / (dk["ms_total"] / 1e3) / 1e9 if dk["ms_total"] > 0 else 0.0
    for k in kernels:
        kk = kernels[k]
        kk["us_per_launch"] = 1e3 * kk["ms_total"] / kk["launches"] if kk["launches"] else None
        kk["gbs_algorithmic"] = (bytes_of[k] / (kk["ms_total"] / 1e3) / 1e9
                                 if kk["ms_total"] > 0 and bytes_of[k] else None)
        kk["gbs_ring_history"] = (ring_of[k] / (kk["ms_total"] / 1e3) / 1e9
                                  if kk["ms_total"] > 0 and ring_of[k] else None)
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tj = json.load(f)
        ent = tj.get(f"{dominant}:{args.workload}:{args.precision}")
        if ent and ent.get("source_hash") == celeris_source_hash():
            traffic = ent["bytes_per_launch"]
    except Exception:
        traffic = None
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic, "peak_source": peak_src,
                "count": "contract: 25 values per cell-update at K = 0, about 14 more per corrector "
                         "(stencil 19 + 8 per corrector, line solves 6 per stage)",
                "ring_history": {"achieved": ring_achieved, "frac": ring_achieved / peak,
                                 "count": "values this implementation's kernels must move: stencil 25 (predictor "
                                          "with the AB3/AM4 ring history) + 10 per corrector, line solves 8 "
                                          "per stage (P^n read for the increment form)"},
                "per_kernel": kernels,
                "per_kernel_from": "the same K steps run again right after the timed ones, with CUDA events "
                                   "around every kernel on the solver's stream (%.4f ms per step with them)"
                                   % (ms_profiled / args.steps),
                "step_bytes_algorithmic": (c_st + c_ln) / args.steps,
                "step_gbs_algorithmic": (c_st + c_ln) / (ms / 1e3) / 1e9 / world,
                "step_frac": (c_st + c_ln) / (ms / 1e3) / 1e9 / world / peak,
                "step_bytes_ring_history": (st_bytes + line_bytes) / args.steps}
    if args.precision == "f64" and s.K > 0:
        # the FP64 pipe bounds the FP64 kernels: the line's roofline is
        # arithmetic, with the memory figures beside it
        fl_of = {"stencil": s.cells * (nstages_pred * FP64_FLOPS["stencil_pred"] +
                                       nstages_corr * FP64_FLOPS["stencil_corr"]),
                 "lines": s.cells * FP64_FLOPS["lines"] * (nstages_pred + nstages_corr), "ghosts": 0}
        dk = kernels[dominant]
        tf = fl_of[dominant] / (dk["ms_total"] / 1e3) / 1e12 if dk["ms_total"] > 0 else 0.0
        roofline = {"bound": "alu", "kernel": dominant, "achieved": tf, "peak": FP64_PEAK_TFLOPS,
                    "unit": "TFLOP/s", "frac": tf / FP64_PEAK_TFLOPS, "traffic": traffic,
                    "peak_source": "derived: 2 DFMA per clock per SM x 2 FLOP x 152 SMs x 2.07 GHz (the nominal "
                                   "1.25 TFLOP/s FP64)",
                    "count": "FP64 operations per cell counted by ncu (2 DFMA + DADD + DMUL): stencil 562.6 "
                             "(predictor) / 517.5 (corrector), line solves 117.9 per stage",
                    "hbm": {k: roofline[k] for k in ("achieved", "peak", "unit", "frac", "peak_source", "count")},
                    "per_kernel": kernels}

    # ---- headless rendering of the final state (Fresnel water, hillshaded land)
    rp = celeris.render_params("fresnel", zmin=-10.0, zmax=3.0, exaggeration=10.0, view=(0.5, 0.3, -0.8))
    img = sol.render(rp)
    for _ in range(3):
        sol.render(rp, out=img)
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(20):
        sol.render(rp, out=img)
    r1.record(stream)
    torch.cuda.synchronize()
    rms = r0.elapsed_time(r1) / 20
    render = {"mode": "fresnel", "ms_per_frame": rms, "pixels_per_s": s.cells / (rms / 1e3),
              "what": "cel_render of the final state into a device RGBA8 image, one pixel per cell"}

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = end_to_end(s, dtype, es, args.steps, celeris, torch, world, barrier)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(s, args.cpu_seconds)

    # ---- the two growth patterns the metric names, on one GPU: the
    # ensemble's speed-up over one launch per scenario, and the adjoint's
    # cost over the forward run at the configured checkpoint spacing (100),
    # with the every-step-kept figure beside it
    ensemble = adjoint = None
    if world == 1 and args.workload == "beach2048" and args.precision == "f32":
        sol.close()
        if args.ensemble_steps > 0:
            el = measure_ensemble(args.ensemble_steps, 5, "f32")
            ensemble = {"workload": "ensemble256", "members": el["config"]["members"],
                        "cells": el["config"]["cells"], "steps": el["steps"],
                        "speedup_vs_single_launch": el["speedup_vs_single_launch"],
                        "value": el["value"], "unit": "cell-updates/s", "ms_per_step": el["ms_per_step"],
                        "single_launch": {"value": el["single_launch"]["value"],
                                          "ms_per_step": el["single_launch"]["ms_per_step"]},
                        "single_launch_plain": el["single_launch_plain"],
                        "gpu_launches": el["gpu_launches"], "graph_steps": el["graph_steps"],
                        "persistent": {k: el["persistent"][k] for k in
                                       ("ms_per_step", "speedup_vs_single_launch", "steps", "gpu_launches")},
                        "finite": el["finite"]}
        if args.adjoint_steps > 0:
            a100 = measure_adjoint(args.adjoint_steps, 5, "f32", 512, 100)
            a0 = measure_adjoint(args.adjoint_steps, 5, "f32", 512, 0)
            dl = celeris.dependent_launch()
            celeris.set_dependent_launch(False)
            ap = measure_adjoint(args.adjoint_steps, 5, "f32", 512, 100)
            celeris.set_dependent_launch(dl)
            adjoint = {"workload": a100["config"]["workload"], "steps": args.adjoint_steps,
                       "ckpt_every": 100, "cost_ratio": a100["value"],
                       "forward_ms_per_step": a100["forward_ms_per_step"],
                       "adjoint_ms_per_step": a100["ms_per_step"],
                       "every_step_kept": {"ckpt_every": 0, "cost_ratio": a0["value"],
                                           "adjoint_ms_per_step": a0["ms_per_step"],
                                           "scratch_gb": a0["config"]["scratch_gb"]},
                       "plain_launches": {"ckpt_every": 100, "cost_ratio": ap["value"],
                                          "forward_ms_per_step": ap["forward_ms_per_step"],
                                          "adjoint_ms_per_step": ap["ms_per_step"],
                                          "what": "the same with cel_set_dependent_launch(0)"},
                       "grad_finite": a100["grad_finite"] and a0["grad_finite"],
                       "what": "dL/dw0 and dL/dz of the 16-gauge misfit (forward with checkpoints, "
                               "recomputation and reverse) over the forward steps alone, CUDA events"}

    if rank == 0:
        line = {"metric": "cell-updates/s", "value": value, "unit": "cell-updates/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": args.precision, "data": "synthetic",
                "config": {"workload": s.name, "nx": s.nx, "ny": s.ny, "cells": s.cells,
                           "corrector_iters": s.K, "dt": s.dt, "courant": 0.1,
                           "parallelism": f"replicas{world}", "dependent_launch": args.dependent_launch,
                           "l2": "inputs larger than L2 (workspace %.0f MB > 129 MB)"
                                 % (sol.workspace.numel() / 1e6)},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "render": render,
                "ensemble": ensemble, "adjoint": adjoint, "line_splits": TUNED,
                "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def max_over_ranks(ms: float) -> float:
    """The slowest rank's time (ms); every rank gets it.  Single process: ms."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(cells_per_rank: int, steps: int, ms: float) -> float:
    """Cell-updates/s of the whole job: every replica advanced cells_per_rank
    cells `steps` times within the slowest rank's ms."""
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    return world * cells_per_rank * steps / (ms / 1e3)


def celeris_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("celeris_kernels.cu", "celeris_internal.cuh", "celeris_physics.cuh"):
        with open(os.path.join(ROOT, "paper_1611_05984_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def end_to_end(s, dtype, es, steps, celeris, torch, world, barrier):
    """Same metric through the public calls a user makes, with host buffers:
    bed and initial state copied from pinned host memory, the solver created,
    then every step followed by a read of the step's gauge record (16 gauges,
    device -> pinned host, queued behind the step without stalling the next
    one: cel_read_gauges_async); the final free surface is copied back, and
    the clock stops once everything is on the host."""
    import numpy as np
    npdt = np.float32 if es == 4 else np.float64
    z_h = torch.from_numpy(s.z.astype(npdt)).pin_memory()
    w0, P0, Q0 = (torch.from_numpy(a.astype(npdt)).pin_memory() for a in s.initial_state())
    eta_h = torch.empty((s.ny, s.nx), dtype=dtype).pin_memory()
    rng = np.random.default_rng(17)
    gij = np.stack([rng.integers(0, s.nx // 2, 16), rng.integers(0, s.ny, 16)], 1)
    stream = torch.cuda.current_stream()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    z_d = z_h.to("cuda", non_blocking=True)
    sol = celeris.Solver(z_d, s.dx, s.dy, s.dt, dtype=dtype, model=s.model, g=s.g, Bd=s.Bd, theta=s.theta,
                         eps=s.eps, K=s.K, ws=s.ws, friction=s.friction, fcoef=s.fcoef)
    for side, sd in s.sides.items():
        sol.set_boundary(side, sd.type, sd.width, sd.comps)
    sol.set_state(w0.to("cuda", non_blocking=True), P0.to("cuda", non_blocking=True),
                  Q0.to("cuda", non_blocking=True))
    sol.set_gauges(gij, 1, 4)
    rec_h = torch.empty((steps, 16), dtype=dtype).pin_memory()
    got = 0
    for k in range(steps):
        sol.step(1)
        got += sol.read_gauges_async(rec_h[k:k + 1])
    w, _, _ = sol.state()
    eta_h.copy_(w, non_blocking=True)
    stream.synchronize()
    el = time.perf_counter() - t0
    barrier()
    assert got == steps and bool(torch.isfinite(rec_h).all())
    h2d = 4 * s.cells * es
    d2h = steps * 16 * es + s.cells * es
    return {"value": world * s.cells * steps / el, "unit": "cell-updates/s",
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "what": "bed + state H2D, create, per-step gauge read (queued, pinned), final eta D2H"}


if __name__ == "__main__":
    main()
