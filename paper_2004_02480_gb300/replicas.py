"""Whole-job accounting for N independent replicas (one process per GPU).

A single CSK solve does not shard usefully across GPUs (every step is a global
argmax), so N ranks solve N independent systems and the job's throughput is
the units all ranks processed divided by the slowest rank's time.  This module
holds that reduction; it works with any torch.distributed backend (NCCL on
GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def aggregate(elapsed_s: float, units: int, launches: int, ok: bool, device=None) -> dict:
    """Max of the elapsed times, sums of units and launches, AND of the
    validity flags, over all ranks of the default process group (identity
    when torch.distributed is not initialised)."""
    if not (dist.is_available() and dist.is_initialized()):
        return {"world": 1, "elapsed_s": elapsed_s, "units": units, "launches": launches,
                "ok": bool(ok), "throughput": units / elapsed_s}
    dev = device if device is not None else torch.device("cpu")
    t = torch.tensor([elapsed_s], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([units, launches, 0 if ok else 1], dtype=torch.int64, device=dev)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    world = dist.get_world_size()
    el = float(t[0])
    return {"world": world, "elapsed_s": el, "units": int(c[0]), "launches": int(c[1]),
            "ok": int(c[2]) == 0, "throughput": int(c[0]) / el}


def lpt_partition(costs, nranks: int) -> list[list[int]]:
    """Split independent work items over `nranks` replicas by the longest-
    processing-time rule: items in decreasing cost (ties by index) each go
    to the currently least-loaded rank (ties by rank).  Deterministic, so
    every rank computes the same partition from the same costs without any
    exchange; each rank then runs items partition[rank].  The largest load
    is at most 4/3 of the optimum (Graham 1969)."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * nranks
    parts: list[list[int]] = [[] for _ in range(nranks)]
    for i in order:
        r = min(range(nranks), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def batched_cost(m: int, n: int, d: int, nrhs: int) -> float:
    """Work estimate of one system of a batched solve: its sketch reads A
    (m n), and each of its nrhs units takes about 2 n steps of O(d)."""
    return float(m) * n + 2.0 * nrhs * n * d
