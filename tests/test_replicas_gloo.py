"""The N-replica accounting of bench.py on two CPU ranks (gloo): the job's
time is the slowest rank's, units and launches add up, one failing rank
invalidates the line."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    from paper_2004_02480_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [2.0, 3.0][rank]
        units = [10, 12][rank]
        res = replicas.aggregate(elapsed, units, launches=11 * units, ok=(rank == 0))
        q.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        res = out[r]
        assert res["world"] == 2 and res["elapsed_s"] == 3.0
        assert res["units"] == 22 and res["launches"] == 242
        assert res["ok"] is False                       # rank 1 reported a failure
        assert res["throughput"] == pytest.approx(22 / 3.0)


def test_single_process_identity():
    from paper_2004_02480_gb300 import replicas
    res = replicas.aggregate(2.0, 10, 110, True)
    assert res == {"world": 1, "elapsed_s": 2.0, "units": 10, "launches": 110, "ok": True,
                   "throughput": 5.0}


def test_lpt_partition_balances_and_covers():
    from paper_2004_02480_gb300 import replicas
    import numpy as np
    rng = np.random.default_rng(0)
    costs = rng.lognormal(0, 1, 257)
    for R in (1, 2, 3, 8):
        parts = replicas.lpt_partition(costs, R)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(257))                          # every item exactly once
        loads = [sum(costs[i] for i in p) for p in parts]
        lower = max(sum(costs) / R, max(costs))                  # no partition beats this
        assert max(loads) <= 4 / 3 * lower + 1e-9                # Graham's LPT bound
        assert parts == replicas.lpt_partition(costs, R)         # deterministic
    assert replicas.lpt_partition([5, 1, 1, 1, 1, 1], 2) == [[0], [1, 2, 3, 4, 5]]


def _lpt_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    from paper_2004_02480_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        costs = [replicas.batched_cost(1000 * (i % 7 + 1), 50 + 10 * i, 500 + 100 * i, 64)
                 for i in range(40)]
        mine = replicas.lpt_partition(costs, world)[rank]
        got = [None] * world
        dist.all_gather_object(got, mine)
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_two_rank_lpt_partition_is_disjoint_and_complete():
    """Each rank computes the LPT partition of the batched work on its own
    (no data-path collective); gathered, the ranks' parts are disjoint and
    cover every system."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_lpt_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts = out[0]
    assert parts == out[1]
    assert sorted(parts[0] + parts[1]) == list(range(40)) and not set(parts[0]) & set(parts[1])
