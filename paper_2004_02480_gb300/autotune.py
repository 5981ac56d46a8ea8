"""Autotuners of the two persistent launches.

Single system (:func:`tune_solve`): picks the CTA count (grid) and the GEMV
variant (rows of the sketch in shared memory or in registers) by timing a
fixed number of steps on the caller's own problem, and caches the choice in a
JSON file keyed by (rows, n, dtype, path, SM count).  Each candidate runs the
loop for `steps` steps with tol = 0 (so every candidate does the same work),
timed with CUDA events around the loop only.

Batched (:func:`tune_batched`): picks the threads per CTA and the CTAs per SM
of csk_solve_batched's persistent launch by timing whole calls on the
caller's batch, then installs the winner in the library
(csk_solve_batched_set_plan) under the batch's signature -- the histogram of
right-hand sides over (log2 d, log2 n) bins -- so later calls with
threads = grid = 0, graph captures included, use it.  The residual path is
not a candidate: the batched launch always takes the GRAM update, whose step
reads one row of G_s (d values) where the GEMV update reads all of At_s
(d n values), and G_s costs one tensor-core product shared by the system's
right-hand sides.
"""
from __future__ import annotations

import json
import os
import threading

import torch

from . import csk

_lock = threading.Lock()
CACHE = os.path.join(os.environ.get("XDG_CACHE_HOME", os.path.expanduser("~/.cache")), "csk",
                     "autotune.json")


def _key(rows: int, n: int, dtype: int, path: int, sms: int) -> str:
    return f"loop:rows={rows}:n={n}:dtype={dtype}:path={path}:sms={sms}"


def _load():
    try:
        with open(CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(cache):
    os.makedirs(os.path.dirname(CACHE), exist_ok=True)
    tmp = CACHE + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, CACHE)


def candidates(sms: int, rows: int | None = None):
    """CTA counts to time: fractions of the SM count, and for problems small
    enough that a few dozen CTAs hold all rows (a cheaper exchange), the
    counts 8..64 that leave at least 4 rows per CTA; also, for each number r
    = 1..10 of rows a warp of the register loop holds (8 warps a CTA), the
    fewest CTAs that hold every row at r rows per warp (the exchange gets
    cheaper with fewer CTAs, the step's arithmetic dearer)."""
    fr = [1.0, 0.9, 0.84, 0.75, 0.66, 0.6, 0.5]
    out = {max(1, int(round(sms * f))) for f in fr}
    if rows is not None:
        out |= {g for g in (8, 12, 16, 24, 32, 40, 48, 64) if g <= sms and 4 * g <= rows}
        for r in range(1, 11):
            g = -(-rows // (8 * r))
            if 1 <= g <= sms and 4 * g <= rows:
                out.add(g)
    return sorted(out, reverse=True)


def tune_solve(A: torch.Tensor, b: torch.Tensor, params: csk.csk_params, x_star=None,
               steps: int = 200, use_cache: bool = True) -> dict:
    """Best {grid, gemv_variant, us_per_step} for csk_solve on (A, b, params);
    also sets params.grid and params.gemv_variant."""
    dev = A.device
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    rows = int(params.d) if params.d > 0 else A.shape[0]
    key = _key(rows, A.shape[1], csk._dtype_code(A), int(params.path), sms)
    with _lock:
        cache = _load() if use_cache else {}
    if key in cache:
        best = cache[key]
    else:
        best = None
        variants = (1, 2) if params.path == csk.GEMV and A.dtype == torch.float32 else (0,)
        for variant in variants:
            for grid in [0] + candidates(sms, rows):         # 0: the library's own plan
                p = csk.csk_params_default(d=params.d, seed=params.seed, path=params.path,
                                           refresh_every=params.refresh_every, tol=0.0,
                                           max_iter=steps, grid=grid, gemv_variant=variant)
                ev = [None, None, torch.cuda.Event(enable_timing=True),
                      torch.cuda.Event(enable_timing=True)]
                csk.set_stage_events(p, ev)
                try:
                    csk.csk_solve(A, b, p, x_star=x_star)        # warm-up
                    ts = []
                    for _ in range(3):
                        csk.csk_solve(A, b, p, x_star=x_star)
                        ts.append(ev[2].elapsed_time(ev[3]))
                except csk.CskError:
                    continue                                   # shape not supported
                us = 1e3 * sorted(ts)[1] / (steps + 1)
                if best is None or us < best["us_per_step"]:
                    best = {"grid": grid, "gemv_variant": variant, "us_per_step": us}
        if best is None:
            raise RuntimeError("no loop configuration runs on this problem")
        if use_cache:
            with _lock:
                cache = _load()
                cache[key] = best
                _store(cache)
    params.grid = best["grid"]
    params.gemv_variant = best["gemv_variant"]
    return dict(best)


# threads per CTA of the batched loop, and the limits that bound its CTAs per
# SM: 128 registers a thread (its launch bound), 64K registers and 228 KB of
# shared memory per SM, the kernel's static shared memory
BATCH_THREADS = (128, 256, 384, 512)
_REGS_PER_THREAD, _REGS_PER_SM, _SMEM_PER_SM, _SMEM_STATIC = 128, 65536, 233472, 2048


def batched_smem_bytes(dmax: int, nmax: int) -> int:
    """Dynamic shared memory of a batched CTA: r and the row weights (d each)
    and x and x* (n each), FP32, padded to 4."""
    return (2 * ((dmax + 3) // 4 * 4) + 2 * ((nmax + 3) // 4 * 4)) * 4


def batched_candidates(sms: int, dmax: int, nmax: int, max_per_sm: int = 4):
    """(threads, grid) launch shapes to time: every thread count of
    BATCH_THREADS with 1 .. k CTAs per SM, k the most that registers and
    shared memory let stay resident (more would only queue)."""
    smem = batched_smem_bytes(dmax, nmax) + _SMEM_STATIC
    out = []
    for t in BATCH_THREADS:
        by_regs = _REGS_PER_SM // (_REGS_PER_THREAD * t)
        by_smem = _SMEM_PER_SM // smem
        k = min(max_per_sm, by_regs, by_smem)
        out += [(t, per * sms) for per in range(1, k + 1)]
    return out


def _batch_key(sig: int, sms: int) -> str:
    return f"batched:sig={sig}:sms={sms}"


def tune_batched(batch, ws=None, params=None, reps: int = 1, use_cache: bool = True) -> dict:
    """Time csk_solve_batched on ``batch`` for every candidate shape and
    install the fastest as the batch signature's plan; returns {threads,
    grid, ms, timings}.  Calls are synchronous and not captured (tuning runs
    before any graph capture)."""
    dev = batch[0].A.device
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    dmax = max(y.d for y in batch)
    nmax = max(y.A.shape[1] for y in batch)
    sig = csk.csk_solve_batched_signature(batch)
    key = _batch_key(sig, sms)
    with _lock:
        cache = _load() if use_cache else {}
    if key in cache:
        best = cache[key]
    else:
        if ws is None:
            ws = torch.empty(csk.csk_solve_batched_workspace_size(batch), dtype=torch.uint8,
                             device=dev)
        base = params if params is not None else csk.csk_params_default()
        timings = {}
        best = None
        for t, g in batched_candidates(sms, dmax, nmax):
            p = csk.csk_params_default(tol=base.tol, max_iter=base.max_iter,
                                       refresh_every=base.refresh_every, threads=t, grid=g)
            csk.csk_solve_batched(batch, p, ws=ws, sync=False)          # warm-up
            ts = []
            for _ in range(max(1, reps)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                csk.csk_solve_batched(batch, p, ws=ws, sync=False)
                e1.record()
                torch.cuda.synchronize(dev)
                ts.append(e0.elapsed_time(e1))
            ms = sorted(ts)[len(ts) // 2]
            timings[f"{t}x{g}"] = ms
            if best is None or ms < best["ms"]:
                best = {"threads": t, "grid": g, "ms": ms}
        best["timings"] = timings
        if use_cache:
            with _lock:
                cache = _load()
                cache[key] = best
                _store(cache)
    csk.csk_solve_batched_set_plan(batch, best["threads"], best["grid"])
    return dict(best)
