"""Ensembles (cel_ensemble_*): many grids stepped with one launch per kernel
kind and stage, against the same grids stepped one cel_step at a time.

The bar is bitwise equality of w, P and Q for every member: the ensemble
launches the same per-tile and per-line code with the same arguments, so
nothing may differ, in FP32 or in FP64.  The member mix covers uneven and
ragged sizes, lines of different segment lengths (several line launches per
stage), sine makers with one and three components, sponges, walls, the NLSW
model, friction laws and per-member dt.
"""
import math

import numpy as np
import pytest

from paper_1611_05984_gb300 import scenarios as sc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dtype(prec):
    return torch.float64 if prec == "f64" else torch.float32


def _members(K):
    out = [sc.beach(nx=200, ny=150, sponge=20, K=K),
           sc.beach_directional(nx=160, ny=130, sponge=16, nshoal=3, K=K),
           sc.soliton_channel(nx=250, ny=30, K=K, x0=5.0)]
    # NLSW dam break on a dry bed
    nx, ny = 180, 40
    x = (np.arange(nx) + 0.5) * 0.05
    d = sc.flat_basin(nx, ny, 0.05, 0.0, 0.05 * 0.05 / math.sqrt(9.81), model=1, K=K)
    d.z = np.zeros((ny, nx))
    d.w0 = np.tile(np.where(x < 3.0, 1.0, 0.0), (ny, 1))
    out.append(d)
    # a long thin and a short wide grid: other segment lengths of the lines
    out.append(sc.flat_basin(1100, 36, 1.0, 4.0, 0.1 / math.sqrt(9.81 * 4.0), K=K, friction=1, fcoef=0.002))
    out[-1].sides[sc.W] = sc.Side(sc.SINE, 0, ((0.05, 6.0, 0.2, 0.4),))
    out.append(sc.flat_basin(20, 300, 1.0, 4.0, 0.1 / math.sqrt(9.81 * 4.0), K=K))
    out[-1].sides[sc.S] = sc.Side(sc.SINE, 0, ((0.03, 7.0, math.pi / 2, 0.0),))
    out[-1].sides[sc.N] = sc.Side(sc.SPONGE, 30)
    out += sc.ensemble(n=4, seed=9, K=K, nx_range=(40, 300), ny_range=(33, 200))
    return out


def _line_launch_class(n, es):
    # the line solver's configuration of a line of n rows: up to 8192 rows
    # (FP32) or 4096 (FP64), one segment per thread in registers, of 2 rows
    # up to 64, 4 up to 128, 8 above, in a multiple of 32 threads; longer
    # lines in shared-memory segments of 32 rows, a thread per 16 elements
    # (register-path lines of one block size share a launch)
    if n <= (8192 if es == 4 else 4096):
        sh = 1 if n <= 64 else (2 if n <= 128 else 3)
        return 0, 0, -(-(-(-n // (1 << sh))) // 32) * 32
    return 1, 5, -(-(-(-n // 16)) // 32) * 32


def _pairs(scens, prec):
    from paper_1611_05984_gb300 import celeris
    a = [celeris.from_scenario(s, dtype=_dtype(prec)) for s in scens]
    b = [celeris.from_scenario(s, dtype=_dtype(prec)) for s in scens]
    return a, b


def _assert_equal(a, b):
    for k, (x, y) in enumerate(zip(a, b)):
        assert x.check_finite() and y.check_finite(), f"member {k} blew up"
        for u, v, name in zip(x.state(), y.state(), "wPQ"):
            assert torch.equal(u, v), f"member {k}: {name} differs"


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_ensemble_bitwise_equals_single_runs(prec):
    """The whole mix with one AM4 iteration (K = 1)."""
    from paper_1611_05984_gb300 import celeris
    scens = _members(1)
    alone, together = _pairs(scens, prec)
    ens = celeris.Ensemble(together)
    for n in (1, 2, 9, 40):            # the Euler steps, then more than one cycle of the tables
        for s in alone:
            s.step(n)
        ens.step(n)
        _assert_equal(alone, together)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_poisoned_ensemble_equals_single_runs(prec):
    """Members built on workspaces of NaN bytes, stepped with argument tables
    of NaN bytes, still equal fresh members stepped alone bit for bit: neither
    the ensemble's launches nor its tables read memory nothing wrote."""
    from paper_1611_05984_gb300 import celeris
    scens = _members(1)
    alone = [celeris.from_scenario(s, dtype=_dtype(prec)) for s in scens]
    together = [celeris.from_scenario(s, dtype=_dtype(prec), poison=True) for s in scens]
    ens = celeris.Ensemble(together, poison=True)
    for n in (1, 2, 9):
        for s in alone:
            s.step(n)
        ens.step(n)
        _assert_equal(alone, together)


@pytest.mark.parametrize("K,prec", [(0, "f32"), (0, "f64"), (2, "f32")])
def test_ensemble_other_corrector_counts(K, prec):
    """K = 0 (predictor only, AB3 carries) and K = 2 (three stages per step)
    on the members that are stable without an odd K: the walled channel, the
    dam break and the flat basins."""
    from paper_1611_05984_gb300 import celeris
    scens = [m for m in _members(K) if m.name.startswith(("soliton", "flat"))]
    alone, together = _pairs(scens, prec)
    ens = celeris.Ensemble(together)
    for n in (3, 30):
        for s in alone:
            s.step(n)
        ens.step(n)
        _assert_equal(alone, together)


def test_ensemble_gauges_boundary_change_and_restore():
    from paper_1611_05984_gb300 import celeris
    scens = _members(1)[:4]
    alone, together = _pairs(scens, "f32")
    for s in alone + together:
        s.set_gauges([(5, 5), (20, 10)], 3, 50)
    ens = celeris.Ensemble(together)
    for s in alone:
        s.step(30)
    ens.step(30)
    _assert_equal(alone, together)
    for x, y in zip(alone, together):
        np.testing.assert_array_equal(x.read_gauges(50), y.read_gauges(50))
    # a new boundary on one member: the ensemble rebuilds its argument tables
    for s in (alone[0], together[0]):
        s.set_boundary(sc.S, sc.SOLID)
    # a checkpoint restored into every member (same step count for all)
    cks = [s.checkpoint() for s in together]
    for s in alone:
        s.step(25)
    ens.step(25)
    _assert_equal(alone, together)
    for s, ck in zip(together, cks):
        s.restore(ck)
    for s, ck in zip(alone, cks):
        s.restore(ck)
    for s in alone:
        s.step(12)
    ens.step(12)
    _assert_equal(alone, together)


def test_ensemble_launch_count():
    from paper_1611_05984_gb300 import celeris
    scens = _members(1)
    together = [celeris.from_scenario(s, dtype=torch.float32) for s in scens]
    ens = celeris.Ensemble(together)
    ens.step(3)
    first = ens.last_launch_count()
    ens.step(1)
    groups = len({_line_launch_class(n, 4) for s in scens for n in (s.nx, s.ny)})
    assert groups >= 2
    assert ens.last_launch_count() == 1 + 2 * (1 + groups)     # ghost tables + 2 stages
    assert first > 3 * (1 + groups)                            # Eckart tables, Euler steps


def test_ensemble_lockstep_and_argument_errors():
    from paper_1611_05984_gb300 import celeris
    scens = _members(1)[:3]
    together = [celeris.from_scenario(s, dtype=torch.float32) for s in scens]
    ens = celeris.Ensemble(together)
    ens.step(2)
    together[1].step(1)
    with pytest.raises(celeris.CelerisError, match="lockstep"):
        ens.step(1)
    with pytest.raises(celeris.CelerisError):
        celeris.Ensemble([together[0], together[0]])
    f64 = celeris.from_scenario(scens[0], dtype=torch.float64)
    with pytest.raises(celeris.CelerisError):
        celeris.Ensemble([together[0], f64])


def test_ensemble_256_uneven_scenarios_stay_finite():
    """The 256-scenario mix (about 4.8e7 cells, FP32), 300 steps."""
    from paper_1611_05984_gb300 import celeris
    members = [celeris.from_scenario(s, dtype=torch.float32) for s in sc.ensemble()]
    ens = celeris.Ensemble(members)
    ens.step(300)
    for m in members:
        assert m.check_finite()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_ensemble_members_match_the_oracle(prec):
    """Members of the ensemble against the FP64 oracle directly (not only
    against single-grid runs): four uneven beaches of the seeded ensemble
    generator and the soliton channel, stepped together 300 steps, each
    compared with its own oracle run every 100 steps (relative L2 of eta,
    FP64 <= 1e-10, FP32 <= 1e-4; P and Q within ten times that)."""
    from paper_1611_05984_gb300 import celeris
    from tests.helpers import oracle_from, rel_l2
    tol = {"f64": 1e-10, "f32": 1e-4}[prec]
    scens = sc.ensemble(n=4, seed=13, K=1, nx_range=(96, 420), ny_range=(64, 260))
    scens.append(sc.soliton_channel(nx=250, ny=30, K=1, x0=5.0))
    members = [celeris.from_scenario(s, dtype=_dtype(prec)) for s in scens]
    oracles = [oracle_from(s) for s in scens]
    ens = celeris.Ensemble(members, stream=members[0].stream)
    for done in (100, 200, 300):
        ens.step(100)
        torch.cuda.synchronize()
        for k, (s, m, o) in enumerate(zip(scens, members, oracles)):
            o.step(100)
            wo, Po, Qo = o.state()
            wg, Pg, Qg = (a.double().cpu().numpy() for a in m.state())
            e = rel_l2(wg - s.ws, wo - s.ws)
            assert e <= tol, f"member {k} ({s.name}): eta rel-L2 {e:.3e} at step {done}"
            for a, b, name in ((Pg, Po, "P"), (Qg, Qo, "Q")):
                if np.linalg.norm(b) > 1e-12:
                    assert rel_l2(a, b) <= 10 * tol, f"member {k}: {name} at step {done}"
    ens.close()


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_captured_cycles_equal_launches_one_by_one(prec):
    """Once the history is full, cel_ensemble_step replays captured 6-step
    cycles: the members must equal, bit for bit, those of the same ensemble
    launching every kernel one by one, and the members stepped alone.  Steps
    in uneven chunks start the cycles at several phases; a change of
    boundary in between discards the graphs, which are captured again."""
    from paper_1611_05984_gb300 import celeris
    scens = _members(1)
    ga = [celeris.from_scenario(s, dtype=_dtype(prec)) for s in scens]
    gb = [celeris.from_scenario(s, dtype=_dtype(prec)) for s in scens]
    alone = [celeris.from_scenario(s, dtype=_dtype(prec)) for s in scens]
    ea = celeris.Ensemble(ga)
    eb = celeris.Ensemble(gb)
    eb.use_graphs(False)
    total = 0
    for n in (3, 13, 7, 20, 1, 12):
        ea.step(n)
        eb.step(n)
        total += n
    assert ea.graph_steps() >= 36 and eb.graph_steps() == 0
    for m in alone:
        m.step(total)
    torch.cuda.synchronize()
    _assert_equal(ga, gb)
    _assert_equal(ga, alone)
    # a boundary change: tables and graphs rebuilt
    for grp in (ga, gb, alone):
        grp[0].set_boundary(sc.N, sc.SOLID)
    before = ea.graph_steps()
    ea.step(14)
    eb.step(14)
    for m in alone:
        m.step(14)
    torch.cuda.synchronize()
    assert ea.graph_steps() >= before + 6
    _assert_equal(ga, gb)
    _assert_equal(ga, alone)
    ea.close()
    eb.close()


@pytest.mark.parametrize("prec,K", [("f32", 1), ("f64", 1), ("f32", 2)])
def test_persistent_launch_equals_launches_one_by_one(prec, K):
    """With the persistent launch on, each call's steps (once the cycle's
    argument blocks are in the table) run as one cooperative launch whose
    blocks work through every phase between grid-wide barriers: the members
    must equal, bit for bit, the same ensemble launching every kernel one by
    one and the members stepped alone, over calls of uneven length and a
    boundary change.  (With two corrector iterations the random beaches grow
    unstable after about 60 steps, as even K does on such grids: that case
    runs fewer steps.)"""
    from paper_1611_05984_gb300 import celeris
    scens = _members(K)
    ga = [celeris.from_scenario(s, dtype=_dtype(prec)) for s in scens]
    gb = [celeris.from_scenario(s, dtype=_dtype(prec)) for s in scens]
    alone = [celeris.from_scenario(s, dtype=_dtype(prec)) for s in scens]
    ea = celeris.Ensemble(ga)
    ea.use_persistent(True, timeout_ms=2000.0)
    eb = celeris.Ensemble(gb)
    eb.use_graphs(False)
    first, second = ((8, 1, 13, 5, 20), (9, 11)) if K == 1 else ((8, 1, 7), (8, 3))
    total = 0
    for n in first:
        ea.step(n)
        eb.step(n)
        total += n
    taken = total - 8
    assert ea.persistent_steps() == taken, ea.persistent_steps()   # every call after the first 8 steps
    assert eb.persistent_steps() == 0
    ea.check()
    for m in alone:
        m.step(total)
    torch.cuda.synchronize()
    _assert_equal(ga, gb)
    _assert_equal(ga, alone)
    for grp in (ga, gb, alone):
        grp[1].set_boundary(sc.S, sc.SOLID)
    for n in second:
        ea.step(n)
        eb.step(n)
        for m in alone:
            m.step(n)
    ea.check()
    torch.cuda.synchronize()
    assert ea.persistent_steps() > taken
    _assert_equal(ga, gb)
    _assert_equal(ga, alone)
    ea.close()
    eb.close()


def test_persistent_barrier_wait_is_bounded():
    """Every wait of the persistent launch's grid-wide barrier has a bound: a
    barrier that expects one block more than the launch has runs out after
    the bound and reports it, and the GPU stays usable (a complete barrier,
    then persistent steps equal to launches one by one)."""
    import time

    from paper_1611_05984_gb300 import celeris
    scens = _members(1)[:3]
    ga = [celeris.from_scenario(s, dtype=torch.float32) for s in scens]
    gb = [celeris.from_scenario(s, dtype=torch.float32) for s in scens]
    ea = celeris.Ensemble(ga)
    eb = celeris.Ensemble(gb)
    eb.use_graphs(False)
    assert not ea.barrier_check(0, 1000.0)
    t0 = time.perf_counter()
    assert ea.barrier_check(1, 200.0)
    took = time.perf_counter() - t0
    assert 0.15 <= took < 10.0, took
    assert not ea.barrier_check(0, 1000.0)
    ea.use_persistent(True, timeout_ms=2000.0)
    ea.step(20)
    eb.step(20)
    ea.check()
    torch.cuda.synchronize()
    assert ea.persistent_steps() == 12
    _assert_equal(ga, gb)
    with pytest.raises(celeris.CelerisError):
        ea.use_persistent(True, timeout_ms=0.0)
    ea.close()
    eb.close()


def test_sharded_ensemble_shares_step_like_the_members_alone():
    """An ensemble sharded over two ranks (both shares built here, as each
    rank would build its own): the shares cover the scenarios once, and
    every member of either share equals, bit for bit, the member stepped
    alone."""
    from paper_1611_05984_gb300 import celeris
    scens = _members(1)
    e0, s0 = celeris.sharded_ensemble(scens, dtype=torch.float32, rank=0, world=2)
    e1, s1 = celeris.sharded_ensemble(scens, dtype=torch.float32, rank=1, world=2)
    assert sorted(s0 + s1) == list(range(len(scens))) and s0 and s1
    alone = [celeris.from_scenario(s, dtype=torch.float32) for s in scens]
    e0.step(11)
    e1.step(11)
    for m in alone:
        m.step(11)
    torch.cuda.synchronize()
    _assert_equal(e0.members + e1.members, [alone[k] for k in s0 + s1])
    e0.close()
    e1.close()


def test_ensemble_under_a_tuned_split():
    """With a line split set (as the autotuner sets it), the ensemble and the
    members stepped alone still agree bit for bit; an ensemble planned before
    the split changed refuses to step."""
    from paper_1611_05984_gb300 import celeris
    celeris.reset_line_splits()
    try:
        celeris.set_line_split(4, 512, 4)
        scens = _members(1)
        alone, together = _pairs(scens, "f32")
        ens = celeris.Ensemble(together)
        ens.step(15)
        for m in alone:
            m.step(15)
        torch.cuda.synchronize()
        _assert_equal(alone, together)
        celeris.set_line_split(4, 512, 2)
        with pytest.raises(celeris.CelerisError, match="splits changed"):
            ens.step(1)
        ens.close()
    finally:
        celeris.reset_line_splits()
