"""Autotuner for the persistent MWRK loop: picks the CTA count (grid) and the
GEMV variant (rows of the sketch in shared memory or in registers) by timing
a fixed number of steps on the caller's own problem, and caches the choice
in a JSON file keyed by (rows, n, dtype, path, SM count).

Each candidate runs the loop for `steps` steps with tol = 0 (so every
candidate does the same work), timed with CUDA events around the loop only.
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
    counts 8..64 that leave at least 4 rows per CTA."""
    fr = [1.0, 0.9, 0.84, 0.75, 0.66, 0.6, 0.5]
    out = {max(1, int(round(sms * f))) for f in fr}
    if rows is not None:
        out |= {g for g in (8, 12, 16, 24, 32, 40, 48, 64) if g <= sms and 4 * g <= rows}
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
