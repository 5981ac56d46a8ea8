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
