"""Host logic of bench.py's multi-GPU path, on CPU with two gloo ranks: the
timing is the max over ranks and the rate counts every replica's cells."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank)        # rank 1 is slower
        rate = bench.whole_job_rate(1000, 4, ms)
        q.put((rank, ms, rate))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, rate in got:
        assert ms == 15.0                                    # the slower rank
        assert rate == pytest.approx(2 * 1000 * 4 / 0.015)  # both replicas' cells


def test_single_process_defaults():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_rate(100, 10, 1000.0) == pytest.approx(1000.0)


def test_ensemble_partition_covers_and_balances():
    """The multi-rank ensemble bench gives each rank a share of the
    scenarios: every scenario exactly once, totals within one scenario."""
    from paper_1611_05984_gb300 import scenarios as sc
    cells = [s.cells for s in sc.ensemble()]
    for world in (1, 2, 3, 8):
        parts = sc.partition(cells, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(cells)))
        loads = [sum(cells[k] for k in p) for p in parts]
        assert max(loads) - min(loads) <= max(cells)
    assert sc.partition([5, 4, 3, 3, 2, 1], 2) == [[0, 3, 5], [1, 2, 4]]   # loads 9 and 9


def _share_worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_1611_05984_gb300 import celeris
    from paper_1611_05984_gb300 import scenarios as sc
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cells = [s.cells for s in sc.ensemble()]
        q.put((rank, celeris.ensemble_share(cells)))     # rank and world from the process group
    finally:
        dist.destroy_process_group()


def test_ensemble_share_under_a_process_group():
    """The library's sharding call, with rank and world taken from a gloo
    process group of two ranks: the two shares are disjoint, cover every
    scenario, and their cell totals differ by at most one scenario."""
    from paper_1611_05984_gb300 import celeris
    from paper_1611_05984_gb300 import scenarios as sc
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_share_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    cells = [s.cells for s in sc.ensemble()]
    assert sorted(got[0] + got[1]) == list(range(len(cells)))
    t0, t1 = (sum(cells[k] for k in got[r]) for r in (0, 1))
    assert abs(t0 - t1) <= max(cells)
    assert got[1] == celeris.ensemble_share(cells, 1, 2)       # explicit rank and world agree
    assert celeris.ensemble_share(cells) == list(range(len(cells)))   # no process group: everything
    with pytest.raises(ValueError):
        celeris.ensemble_share(cells, 2, 2)
