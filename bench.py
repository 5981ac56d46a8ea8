#!/usr/bin/env python
"""Benchmark of GPU count-sketch Kaczmarz (CSK) on one GB300 per rank.

Workload (one "step" = one whole solve, Algorithm 1 end to end): plain CSK in
FP32 with FP64 row norms, A 100000 x 500 iid N(0,1), x* iid N(0,1),
b = A x*, count sketch d = 5000 from a seed, x0 = 0, GEMV residual path,
stop at RES = ||x - x*||^2 / ||x*||^2 <= 1e-6 (Section 3).  Inputs are seeded
synthetic Gaussians (the paper's own data are MATLAB randn draws), resident in
HBM before the timed region; A (200 MB) is larger than the 129 MB L2.

Metric: solves per second (whole job, all ranks); ms_per_step is the
time-to-RSE<=1e-6 of one solve.  With N ranks each rank solves its own
independent system (weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
    python bench.py --workload {c1,precision,batched,serving}   # the other configurations
    python bench.py --workload noisy     # an inconsistent b, residual stopping rule

`--impl reference` times the plain CPU oracle (the paper's method restated
in C, FP64) on the same workload on this machine's host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

M, N_COLS, D, TOL = 100_000, 500, 5000, 1e-6
WORKLOAD = ("plain CSK FP32 with FP64 row norms: A 100000x500 iid N(0,1), x* iid N(0,1), b=Ax*, "
            "d=5000 count sketch, x0=0, GEMV residual path, stop at RES<=1e-6")
METRIC = "solves/s to RES<=1e-6 (plain GPU CSK, A 100000x500 FP32, d=5000)"
UNIT = "solves/s"
PROFILES = os.path.join(ROOT, "profiles")


def sketch_bytes(m, n, d, s=4):
    # read A and b, write+read perm (8 B/row), write At and bt, cnt/off (8 B/bucket)
    return s * m * n + s * m + 8 * m + s * d * n + s * d + 8 * d


LOOP_KERNELS = {1: "k_iterate_gemv", 2: "k_iterate_gemv_reg", 3: "k_iterate_gemv_stream"}
LOOP_VARIANTS = {0: "auto", 1: "shared-memory rows", 2: "register rows", 3: "streamed rows (TMA ring)"}


def gemv_bytes_per_eval(d, n, s=4):
    # At (d x n) once per residual evaluation, plus bt, x and the row update
    return s * d * n + s * (d + 2 * n)


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"csk_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


LOOP_SOURCES = ("iterate.cu", "common.cuh", "reduce.cuh", "async.cuh", "fp64.cuh", "own_sketch.cuh")


def _source_hash(*files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


def _traffic(kernel_tag: str, src_hash: str):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current kernel source (else None)."""
    path = os.path.join(PROFILES, f"{kernel_tag}.traffic.txt")
    if not os.path.exists(path):
        return None
    kv = {}
    for line in open(path):
        if ":" in line and not line.startswith("#"):
            k, v = line.split(":", 1)
            kv[k.strip()] = v.strip()
    if kv.get("source_hash") != src_hash:
        return None
    try:
        return float(kv["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _bf16_peak():
    """Dense BF16 tensor peak (TFLOP/s) for a kernel timed alone: the measured
    burst figure, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        if "bf16_tflops" in p:
            return float(p["bf16_tflops"]), "measured"
    return 1900.0, "fallback"


def gram_work(d, n, bm=128, bn=256, bk=64):
    """Work of csk_gram on d x n: the tiles it computes (those with an
    element on or above the diagonal) and their BF16 flops (3 products over
    the padded K), plus the FP32-equivalent flops of the dense product
    (2 d^2 n) and of its unique upper triangle (d (d + 1) n)."""
    dp = (d + bn - 1) // bn * bn
    kp = (n + bk - 1) // bk * bk
    nbi, nbj = dp // bm, dp // bn
    tiles = sum(nbj - (i * bm) // bn for i in range(nbi))
    return {"tiles": tiles, "bf16_flops": tiles * bm * bn * kp * 2 * 3,
            "dense_fp32_flops": 2 * d * d * n, "upper_fp32_flops": d * (d + 1) * n}


def oracle_solves(A64, b64, xs, seconds: float, min_solves: int = 1, max_solves: int = 10 ** 9,
                  threads: int | None = None):
    """Time whole oracle solves of the workload (FP64; all host cores, or
    `threads` of them -- 1 is the literal single-thread Algorithm 1)."""
    import oracle
    cores = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    n_done, its = 0, []
    while n_done < max_solves and (n_done < min_solves or time.perf_counter() - t0 < seconds):
        r = oracle.csk(A64, b64, D, 0, x_star=xs, tol=TOL, nthreads=cores)
        its.append(r.iters)
        n_done += 1
    dt = time.perf_counter() - t0
    return n_done, dt, cores, its


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    from paper_2004_02480_gb300 import synth
    s = synth.gaussian_system(M, N_COLS, 0, np.float32)
    A64, b64 = s.A.astype(np.float64), s.b.astype(np.float64)
    import oracle
    oracle.build()
    # warm-up solves, then K timed solves; cap the run at a few minutes
    t_w = time.perf_counter()
    for _ in range(max(0, args.warmup)):
        oracle_solves(A64, b64, s.x_star, 0.0, 1, 1)
        if time.perf_counter() - t_w > 60:
            break
    per = max(time.perf_counter() - t_w, 1e-3) / max(1, args.warmup)
    k_run = max(1, min(args.steps, int(180.0 / per) if args.warmup else args.steps))
    n_done, dt, cores, its = oracle_solves(A64, b64, s.x_star, 0.0, k_run, k_run)
    value = n_done / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "steps_run": n_done, "warmup": args.warmup,
        "ms_per_step": 1000.0 * dt / n_done, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded N(0,1), paper Section 3 recipe)",
        "config": {"workload": WORKLOAD, "m": M, "n": N_COLS, "d": D, "tol": TOL},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{n_done} whole oracle solves (sketch + literal Algorithm 1, "
                                   f"mean IT {np.mean(its):.1f}) on {cores} host threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- other configs
# `--workload` selects another of the five configurations; each prints one JSON
# line of its own metric.  The default (`plain`) is the line above.

def _events(torch, k):
    return [torch.cuda.Event(enable_timing=True) for _ in range(k)]


def run_c1(args):
    """plain CSK FP64: A 2000x50, d = 500 (time to RES <= 1e-6, IT vs the oracle)."""
    import torch
    import oracle
    from paper_2004_02480_gb300 import csk, synth
    csk.lib()
    dev = torch.device("cuda", 0)
    s = synth.gaussian_system(2000, 50, 0, np.float64)
    A, b, xs = (torch.from_numpy(v).to(dev) for v in (s.A, s.b, s.x_star))
    p = csk.csk_params_default(d=500, seed=0, tol=TOL)
    from paper_2004_02480_gb300 import autotune
    autotune.tune_solve(A, b, p, x_star=xs)               # loop CTA count, untimed
    ws = csk._workspace(csk.csk_solve_workspace_size(2000, 50, csk.CSK_F64, p), dev)
    x = torch.empty(50, dtype=torch.float64, device=dev)
    info = torch.zeros(64, dtype=torch.uint8, device=dev)
    for _ in range(max(3, args.warmup)):
        csk.csk_solve(A, b, p, x_star=xs, x_out=x, info=info, ws=ws, sync=False)
    torch.cuda.synchronize()
    e0, e1 = _events(torch, 2)
    e0.record()
    for _ in range(args.steps):
        csk.csk_solve(A, b, p, x_star=xs, x_out=x, info=info, ws=ws, sync=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    r = csk.read_info(info)
    # stage breakdown of one more solve (events between the stages)
    ev = _events(torch, 5)
    csk.set_stage_events(p, ev)
    stages = []
    for _ in range(5):
        csk.csk_solve(A, b, p, x_star=xs, x_out=x, info=info, ws=ws, sync=False)
        torch.cuda.synchronize()
        stages.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
    st = np.median(np.array(stages), axis=0)
    ref = oracle.csk(s.A, s.b, 500, 0, x_star=s.x_star)
    print(json.dumps({
        "metric": "time-to-RSE<=1e-6 (ms), plain CSK FP64, A 2000x50, d=500", "value": ms,
        "unit": "ms", "higher_is_better": False, "n_gpus": 1, "steps": args.steps,
        "dtype": "f64", "data": "synthetic (seeded N(0,1))",
        "config": {"workload": "plain CSK FP64: A 2000x50 iid N(0,1), x* iid N(0,1), b=Ax*, d=500, "
                               "x0=0, stop at RES<=1e-6", "grid": r["grid"]},
        "iters": r["iters"], "oracle_iters": ref.iters, "rse": r["rse"], "status": r["status"],
        "breakdown": {"setup_ms": float(st[0]), "sketch_ms": float(st[1]), "iterate_ms": float(st[2]),
                      "check_ms": float(st[3]),
                      "us_per_step": 1e3 * float(st[2]) / (r["iters"] + 1)}}),
        flush=True)
    return 0


def run_noisy(args):
    """Inconsistent system (outside the paper's consistent setting): the
    100000x500 FP32 workload with b = A x* + e, e iid Gaussian at 1e-3 of
    rms(A x*); no x*, so the loop stops on ||bt - At x||^2 / ||bt||^2 <= 1e-5,
    about ten times the least-squares floor of the sketched system."""
    import torch
    from paper_2004_02480_gb300 import csk, synth
    csk.lib()
    dev = torch.device("cuda", 0)
    m, n, d, tol = M, N_COLS, D, 1e-5
    s = synth.noisy_system(m, n, 0, 1e-3, np.float32)
    A, b = (torch.from_numpy(v).to(dev) for v in (s.A, s.b))
    from paper_2004_02480_gb300 import autotune
    p = csk.csk_params_default(d=d, seed=0, tol=tol, path=csk.GEMV)
    autotune.tune_solve(A, b, p)                      # grid and loop variant, untimed
    ws = csk._workspace(csk.csk_solve_workspace_size(m, n, csk.CSK_F32, p), dev)
    x = torch.empty(n, dtype=torch.float32, device=dev)
    info = torch.zeros(64, dtype=torch.uint8, device=dev)
    for _ in range(max(3, args.warmup)):
        csk.csk_solve(A, b, p, x_out=x, info=info, ws=ws, sync=False)
    torch.cuda.synchronize()
    e0, e1 = _events(torch, 2)
    e0.record()
    for _ in range(args.steps):
        csk.csk_solve(A, b, p, x_out=x, info=info, ws=ws, sync=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    r = csk.read_info(info)
    # least-squares floor of the sketched system (no x reaches a smaller residual)
    sk = csk.csk_sketch(A, d, 0, b)
    At, bt = sk.At.double().cpu().numpy(), sk.bt.double().cpu().numpy().ravel()
    xls = np.linalg.lstsq(At, bt, rcond=None)[0]
    floor = float(np.sum((bt - At @ xls) ** 2) / np.sum(bt * bt))
    xv = x.double().cpu().numpy()
    print(json.dumps({
        "metric": "time-to-residual tol (ms), inconsistent system, no x*", "value": ms, "unit": "ms",
        "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "dtype": "f32",
        "data": "synthetic (seeded N(0,1); b = A x* + 1e-3 rms(A x*) noise)",
        "config": {"workload": f"A {m}x{n} FP32, d={d}, b = A x* + e (relative noise 1e-3), no x*, "
                               f"stop at ||bt - At x||^2/||bt||^2 <= {tol}", "grid": r["grid"],
                   "variant": int(p.gemv_variant)},
        "whole_solve_us_per_step": 1e3 * ms / (r["iters"] + 1),
        "status": r["status"], "iters": r["iters"], "resid2": r["resid"] ** 2,
        "ls_floor_resid2": floor, "resid2_over_floor": r["resid"] ** 2 / floor,
        "rel_err_vs_noiseless_x": float(np.linalg.norm(xv - s.x_star) / np.linalg.norm(s.x_star)),
        "rel_err_vs_sketched_ls": float(np.linalg.norm(xv - xls) / np.linalg.norm(xls))}),
        flush=True)
    return 0


def run_precision(args):
    """precision form: A 1e6x1000 FP32 = G diag(sigma) Q, kappa 1e3, d = 20000,
    split-BF16 Gram, FP64 refresh every 100 steps."""
    import torch
    from paper_2004_02480_gb300 import csk, synth
    csk.lib()
    m, n, d = 1_000_000, 1000, 20000
    A, b, xs64 = synth.conditioned_system_device(m, n, 0, 1e3, "cuda")
    xs = xs64.float()
    p = csk.csk_params_default(d=d, seed=0, path=csk.GRAM, refresh_every=100, tol=TOL,
                               max_iter=20000)
    from paper_2004_02480_gb300 import autotune
    tuned = autotune.tune_solve(A, b, p, x_star=xs)       # loop CTA count, untimed
    ev = _events(torch, 5)
    csk.set_stage_events(p, ev)
    csk.csk_solve(A, b, p, x_star=xs)                     # warm-up
    rec = []
    for _ in range(max(1, min(args.steps, 5))):
        x, info = csk.csk_solve(A, b, p, x_star=xs)
        rec.append(([ev[i].elapsed_time(ev[i + 1]) for i in range(4)], ev[0].elapsed_time(ev[4]), info))
    st = np.median(np.array([r[0] for r in rec]), axis=0)
    tot = float(np.median([r[1] for r in rec]))
    info = rec[0][2]
    sk_bytes = sketch_bytes(m, n, d)
    print(json.dumps({
        "metric": "time-to-RSE<=1e-6 (ms), precision form, split-BF16 Gram path", "value": tot,
        "unit": "ms", "higher_is_better": False, "n_gpus": 1, "steps": len(rec), "dtype": "f32",
        "data": "synthetic (A = G diag(sigma) Q, G iid N(0,1), Q Haar, sigma log-spaced 1..1e3)",
        "config": {"workload": "A 1000000x1000 FP32, kappa 1e3, d=20000, GRAM path, FP64 refresh "
                               "every 100 steps, cap 20000 steps", "grid": info["grid"]},
        "status": info["status"], "iters": info["iters"], "rse": info["rse"], "resid": info["resid"],
        "note": "RES <= 1e-6 is out of reach within the 20000-step cap at kappa 1e3; the line "
                "reports the time to the cap and the RES reached",
        "breakdown": {"sketch_ms": st[0], "gram_and_norms_ms": st[1], "iterate_ms": st[2],
                      "check_ms": st[3], "us_per_step": 1e3 * st[2] / (info["iters"] + 1),
                      "sketch_gbs": sk_bytes / st[0] / 1e6,
                      "gram_tflops_fp32_equiv": 2.0 * d * d * n / st[1] / 1e9}}), flush=True)
    return 0


def batched_measure(torch, csk, dev, K, warmup, sample=32, rank=0, world=1):
    """The batched form: 256 systems (m log-uniform [5000, 200000], n uniform
    [50, 1000], d = 10 n) x 64 right-hand sides, A and X* iid N(0,1) FP32,
    B = A X*.  The launch shape comes from the batched autotuner (installed as
    the batch's plan, so the captured call with threads = grid = 0 uses it);
    the call is captured once in a CUDA graph and replayed K times.  The plain
    comparator solves a sample of the same (system, right-hand side) pairs one
    at a time with csk_solve, its loop CTA count and variant autotuned per
    shape for both residual paths, and takes the faster path per solve."""
    from paper_2004_02480_gb300 import autotune, synth
    S, R = 256, 64
    shapes = synth.batched_shapes(S, 5000, 200000, 50, 1000, seed=7)
    # with several replicas each takes its share of the systems (longest
    # processing time first; every rank computes the same partition)
    from paper_2004_02480_gb300 import replicas
    mine = replicas.lpt_partition([replicas.batched_cost(m, n, 10 * n, R) for m, n in shapes],
                                  world)[rank]
    batch = []
    for i in mine:
        m, n = shapes[i]
        g = torch.Generator(device=dev).manual_seed(11 + 7919 * i)
        A = torch.randn((m, n), generator=g, device=dev, dtype=torch.float32)
        X = torch.randn((n, R), generator=g, device=dev, dtype=torch.float32)
        batch.append(csk.BatchSystem(A=A, B=A @ X, d=10 * n, seed=1000 + i, Xstar=X))
    S = len(batch)
    ws = torch.empty(csk.csk_solve_batched_workspace_size(batch), dtype=torch.uint8, device=dev)
    tuned = autotune.tune_batched(batch, ws=ws, use_cache=False)
    p = csk.csk_params_default()            # threads = grid = 0: the installed plan
    st = torch.cuda.Stream(dev)
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        csk.csk_solve_batched(batch, p, ws=ws, sync=False)
    torch.cuda.current_stream().wait_stream(st)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        csk.csk_solve_batched(batch, p, ws=ws, sync=False)
    for _ in range(max(1, warmup)):
        graph.replay()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    e0, e1 = _events(torch, 2)
    e0.record()
    for _ in range(K):
        graph.replay()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / K
    recs = [np.frombuffer(y.info.cpu().numpy().tobytes(), dtype=csk.INFO_DTYPE) for y in batch]
    ok = all(int(r["status"].max()) == 0 and float(r["rse"].max()) <= TOL for r in recs)
    grids = {int(v) for r in recs for v in r["grid"]}
    its = np.concatenate([r["iters"] for r in recs])
    # plain single-system GPU CSK on a sample of the same solves (one RHS each)
    rng = np.random.default_rng(3)
    pairs = [(int(i), int(rng.integers(R))) for i in rng.integers(S, size=sample if rank == 0 else 0)]
    per_path = {"gram": [], "gemv": []}
    good = True
    for i, r in pairs:
        y = batch[i]
        b = y.B[:, r].contiguous()
        xsr = y.Xstar[:, r].contiguous()
        for name, path in (("gram", csk.GRAM), ("gemv", csk.GEMV)):
            pp = csk.csk_params_default(d=y.d, seed=y.seed, path=path, tol=TOL)
            autotune.tune_solve(y.A, b, pp, x_star=xsr)            # per shape, cached
            csk.csk_solve(y.A, b, pp, x_star=xsr)
            a0, a1 = _events(torch, 2)
            a0.record()
            _, inf = csk.csk_solve(y.A, b, pp, x_star=xsr, sync=False)
            a1.record()
            torch.cuda.synchronize()
            rr = csk.read_info(inf)
            good &= rr["status"] == 0 and rr["rse"] <= TOL
            per_path[name].append(a0.elapsed_time(a1))
    best_ms = [min(a, b) for a, b in zip(per_path["gram"], per_path["gemv"])]
    plain = None
    if pairs:
        plain = {"solves_per_s": 1e3 / float(np.mean(best_ms)),
                 "gram_solves_per_s": 1e3 / float(np.mean(per_path["gram"])),
                 "gemv_solves_per_s": 1e3 / float(np.mean(per_path["gemv"])),
                 "sampled_solves": len(pairs), "all_converged": bool(good),
                 "how": "csk_solve per (system, RHS), loop CTA count and variant autotuned per "
                        "shape (autotune.tune_solve) for the GRAM and GEMV paths, faster path "
                        "per solve"}
    job = replicas.aggregate(ms * 1e-3, S * R, 0, ok, device=dev)
    ms = job["elapsed_s"] * 1e3
    value = job["throughput"]
    return {"solves_per_s": value, "ms_per_launch": ms, "replays": K, "all_converged": bool(ok),
            "iters_mean": float(its.mean()), "iters_max": int(its.max()),
            "tuned": {"threads": tuned["threads"], "grid": tuned["grid"],
                      "candidates_ms": tuned.get("timings")},
            "grid_used": sorted(grids), "plain_single_system": plain,
            "speedup_over_plain": value / plain["solves_per_s"] if plain else None,
            "replicas": world, "systems_this_rank": S,
            "workload": "256 systems, m log-uniform [5000,200000], n uniform [50,1000], d=10n, "
                        "64 right-hand sides each, FP32, GRAM path, CUDA-graph replay"}


def sketch_gram_measure(torch, csk, dev, reps=5):
    """The precision form's sketch and Gram matrix: A 1e6 x 1000 FP32 =
    G diag(sigma) Q (kappa 1e3), d = 20000.  Whole csk_sketch call (sort
    chain, A pass, b pass) and whole csk_gram call (split, tcgen05 product,
    diagonal), each timed with CUDA events over `reps` calls after a warm-up;
    A (4 GB) is far larger than L2."""
    from paper_2004_02480_gb300 import synth
    m, n, d = 1_000_000, 1000, 20000
    A, b, _ = synth.conditioned_system_device(m, n, 0, 1e3, dev)
    sk = csk.csk_sketch(A, d, 0, b)
    ts = []
    for _ in range(reps):
        e0, e1 = _events(torch, 2)
        e0.record()
        sk = csk.csk_sketch(A, d, 0, b)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    sk_ms = float(np.median(ts))
    del A, b
    G = csk.csk_gram(sk.At, sk.norms2)
    tg = []
    for _ in range(reps):
        e0, e1 = _events(torch, 2)
        e0.record()
        G = csk.csk_gram(sk.At, sk.norms2)
        e1.record()
        torch.cuda.synchronize()
        tg.append(e0.elapsed_time(e1))
    g_ms = float(np.median(tg))
    del G
    hbm, hk = _peaks()
    bf16, bk = _bf16_peak()
    w = gram_work(d, n)
    sk_gbs = sketch_bytes(m, n, d) / (sk_ms * 1e-3) / 1e9
    issued = w["bf16_flops"] / (g_ms * 1e-3) / 1e12
    return {"workload": "A 1000000x1000 FP32 (kappa 1e3), d=20000",
            "sketch_ms": sk_ms, "sketch_gbs": sk_gbs, "sketch_frac_of_" + hk + "_hbm": sk_gbs / hbm,
            "gram_ms": g_ms,
            "gram_bf16_issued_tflops": issued, "gram_bf16_frac_of_" + bk + "_peak": issued / bf16,
            "gram_fp32_equiv_tflops_dense": w["dense_fp32_flops"] / (g_ms * 1e-3) / 1e12,
            "gram_fp32_equiv_tflops_upper": w["upper_fp32_flops"] / (g_ms * 1e-3) / 1e12,
            "note": "BF16 issued = computed 128x256 tiles (those touching the upper triangle) x 3 "
                    "products x padded K; dense = 2 d^2 n, upper = d (d+1) n FP32-equivalent flops"}


def run_batched(args):
    """batched form alone: its own JSON line (solves/s of the graph replay;
    with N ranks each replays its LPT share of the systems, no collective on
    the data path, and the job's time is the slowest rank's)."""
    import torch
    from paper_2004_02480_gb300 import csk
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    csk.lib()
    dev = torch.device("cuda", local)
    r = batched_measure(torch, csk, dev, max(1, min(args.steps, 10)), max(1, args.warmup),
                        rank=rank, world=world)
    if rank != 0:
        dist.destroy_process_group()
        return 0
    print(json.dumps({
        "metric": "solves/s at RES<=1e-6, batched form (one persistent launch in a CUDA graph)",
        "value": r["solves_per_s"], "unit": "solves/s", "higher_is_better": True, "n_gpus": world,
        "scaling": "strong",
        "steps": r["replays"], "warmup": max(1, args.warmup), "ms_per_step": r["ms_per_launch"],
        "dtype": "f32", "data": "synthetic (A, X* iid N(0,1), B = A X*)",
        "config": {"workload": r["workload"]}, **{k: v for k, v in r.items() if k != "workload"}}),
        flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_serving(args):
    """serving form: Poisson 2000 requests/s for `--seconds` (m log-uniform
    [2000, 100000], n [20, 500], d = 8 n, 1-16 right-hand sides), 120 GB budget."""
    from paper_2004_02480_gb300 import serve
    reqs = serve.poisson_requests(args.rate, args.seconds, 0)
    srv = serve.Server(budget_bytes=120e9, chunk=args.chunk, lanes=args.lanes)
    st = srv.run(reqs)
    print(json.dumps({
        "metric": "p50 latency (ms) under Poisson arrivals, continuous batching", "value": st["p50_ms"],
        "unit": "ms", "higher_is_better": False, "n_gpus": 1, "dtype": "f32",
        "data": "synthetic (seeded Gaussian systems generated on the device per request)",
        "config": {"workload": f"Poisson {args.rate}/s for {args.seconds} s, m log-uniform "
                               "[2000,100000], n [20,500], d=8n, 1-16 RHS, FP32, 120 GB budget"},
        **st}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=30)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched and sketch/Gram blocks (both outside the timed steps)")
    ap.add_argument("--grid", type=int, default=0, help="loop CTA count (0 = autotune)")
    ap.add_argument("--variant", type=int, default=0, help="loop variant 1-3 (0 = autotune)")
    ap.add_argument("--workload", default="plain",
                    choices=["plain", "c1", "precision", "batched", "serving", "noisy"],
                    help="plain: the 100000x500 line (default); c1: 2000x50 FP64; precision: "
                         "1e6x1000 kappa 1e3 GRAM; batched: 256 systems x 64 RHS; serving: "
                         "Poisson arrivals; noisy: 100000x500 with an inconsistent b")
    ap.add_argument("--seconds", type=float, default=60.0, help="serving: arrival window")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: requests per second")
    ap.add_argument("--chunk", type=int, default=512, help="serving: steps per unit per tick")
    ap.add_argument("--lanes", type=int, default=8, help="serving: streams with their own ticks")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "plain":
        return {"c1": run_c1, "precision": run_precision, "batched": run_batched,
                "serving": run_serving, "noisy": run_noisy}[args.workload](args)

    import torch
    import torch.distributed as dist

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2004_02480_gb300 import csk, synth
    csk.lib()   # fails loudly when libcsk.so is missing

    s = synth.gaussian_system(M, N_COLS, rank, np.float32)
    A = torch.from_numpy(s.A).to(dev)
    b = torch.from_numpy(s.b).to(dev)
    xs = torch.from_numpy(s.x_star.astype(np.float32)).to(dev)
    params = csk.csk_params_default(d=D, seed=rank, tol=TOL, path=csk.GEMV)
    from paper_2004_02480_gb300 import autotune
    if args.grid > 0 and args.variant > 0:
        params.grid, params.gemv_variant = args.grid, args.variant
        tuned = {"grid": args.grid, "gemv_variant": args.variant, "us_per_step": None}
    else:
        tuned = autotune.tune_solve(A, b, params, x_star=xs)  # grid and loop variant, untimed
    ws = csk._workspace(csk.csk_solve_workspace_size(M, N_COLS, csk.CSK_F32, params), dev)
    x = torch.empty(N_COLS, dtype=torch.float32, device=dev)
    K, W = args.steps, args.warmup
    infos = torch.empty((K, 64), dtype=torch.uint8, device=dev)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(K)]
    pk = [csk.csk_params_default(d=D, seed=rank, tol=TOL, path=csk.GEMV, grid=params.grid,
                                 gemv_variant=params.gemv_variant) for _ in range(K)]
    for i in range(K):
        csk.set_stage_events(pk[i], ev[i])

    for _ in range(W):
        csk.csk_solve(A, b, params, x_star=xs, x_out=x, info=infos[0], ws=ws, sync=False)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    l0 = csk.csk_kernel_launches()
    t0.record()
    for i in range(K):
        csk.csk_solve(A, b, pk[i], x_star=xs, x_out=x, info=infos[i], ws=ws, sync=False)
    t1.record()
    torch.cuda.synchronize()
    launches = csk.csk_kernel_launches() - l0
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = t0.elapsed_time(t1)

    recs = [csk.read_info(infos[i]) for i in range(K)]
    ok = all(r["status"] == 0 and r["rse"] <= TOL for r in recs)
    iters = [r["iters"] for r in recs]
    st_sketch = [ev[i][0].elapsed_time(ev[i][1]) for i in range(K)]
    st_iter = [ev[i][2].elapsed_time(ev[i][3]) for i in range(K)]
    st_check = [ev[i][3].elapsed_time(ev[i][4]) for i in range(K)]

    # ---- end to end through the host-buffer entry point (pinned host memory)
    # E solves of systems held in page-locked host memory through
    # csk_solve_host_many: every solve copies its A, b, x* in and its x and
    # info record out; the copies of solve k+1 overlap solve k.
    Ah = torch.from_numpy(s.A).pin_memory().numpy()
    bh = torch.from_numpy(s.b).pin_memory().numpy()
    xsh = torch.from_numpy(s.x_star.astype(np.float32)).pin_memory().numpy()
    E = max(1, args.e2e_steps)
    probs = [csk.HostProblem(A=Ah, b=bh, x_star=xsh) for _ in range(E)]
    wsh = csk._workspace(csk.csk_solve_host_many_workspace_size(probs, params), dev)
    csk.csk_solve_host_many(probs[:2], params, ws=wsh)
    if world > 1:
        dist.barrier()
    te = time.perf_counter()
    rc = csk.csk_solve_host_many(probs, params, ws=wsh)
    te = time.perf_counter() - te
    e2e_ok = rc == 0 and all(csk.info_dict(q.info)["rse"] <= TOL for q in probs)

    # the paper's comparison: MWRK on A itself (Remark 1, d = 0), same system;
    # each step reads all of A (200 MB, larger than L2) from HBM
    pm = csk.csk_params_default(d=0, tol=TOL, path=csk.GEMV)
    wsm = csk._workspace(csk.csk_solve_workspace_size(M, N_COLS, csk.CSK_F32, pm), dev)
    csk.csk_solve(A, b, pm, x_star=xs, ws=wsm)
    RM = 3
    mev = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(RM)]
    mrec = []
    for i in range(RM):
        csk.set_stage_events(pm, mev[i])
        _, inf_m = csk.csk_solve(A, b, pm, x_star=xs, ws=wsm)
        mrec.append(inf_m)
    torch.cuda.synchronize()
    m_tot = float(np.median([e[0].elapsed_time(e[4]) for e in mev]))
    m_loop = float(np.median([e[2].elapsed_time(e[3]) for e in mev]))
    m_it = mrec[0]["iters"]
    # the loop streams A once per residual evaluation (IT + 1 of them)
    m_gbs = (m_it + 1) * gemv_bytes_per_eval(M, N_COLS) / (m_loop * 1e-3) / 1e9
    mwrk = {"ms": m_tot, "loop_ms": m_loop, "iters": m_it, "rse": mrec[0]["rse"],
            "status": mrec[0]["status"], "stream_gbs": m_gbs}
    # Remark 1's residual-update form on the same A (r -= alpha A A_i^T: one
    # pass over A per step, against the chosen row), r recomputed every 50 steps
    pu = csk.csk_params_default(d=0, tol=TOL, path=csk.UPDATE, refresh_every=50)
    csk.csk_solve(A, b, pu, x_star=xs, ws=wsm)
    uev = [_events(torch, 5) for _ in range(RM)]
    urec = []
    for i in range(RM):
        csk.set_stage_events(pu, uev[i])
        _, inf_u = csk.csk_solve(A, b, pu, x_star=xs, ws=wsm)
        urec.append(inf_u)
    torch.cuda.synchronize()
    mwrk["update_ms"] = float(np.median([e[0].elapsed_time(e[4]) for e in uev]))
    mwrk["update_iters"] = urec[0]["iters"]
    mwrk["update_rse"] = urec[0]["rse"]
    del wsm

    # latency floor of one step: the same CTA count running only the
    # exchange (CTA reduction + mailbox round trip), 2000 rounds per launch
    # (about 25 ms of GPU time, outside the timed steps)
    floor_us = None
    if tuned["gemv_variant"] != 3:
        fl_ws = csk._workspace(csk.lib().csk_exchange_floor_workspace_size(recs[0]["grid"]), dev)
        fts = []
        for _ in range(6):
            f0, f1 = _events(torch, 2)
            f0.record()
            csk.csk_exchange_floor(recs[0]["grid"], 2000, device=dev, ws=fl_ws)
            f1.record()
            torch.cuda.synchronize()
            fts.append(f0.elapsed_time(f1))
        floor_us = 1e3 * float(np.median(fts[1:])) / 2000
    targets = None
    if world == 1 and not args.no_extras:
        targets = {"batched": batched_measure(torch, csk, dev, 3, 1),
                   "precision_sketch_gram": sketch_gram_measure(torch, csk, dev)}

    from paper_2004_02480_gb300 import replicas
    job = replicas.aggregate(ms * 1e-3, K, launches, ok, device=dev)
    job_e2e = replicas.aggregate(te, E, 0, e2e_ok, device=dev)
    ms, te, launches, ok, e2e_ok = (job["elapsed_s"] * 1e3, job_e2e["elapsed_s"], job["launches"],
                                    job["ok"], job_e2e["ok"])

    if rank != 0:
        dist.destroy_process_group()
        return 0

    hbm, peak_kind = _peaks()
    mean_it = float(np.mean(iters))
    it_ms = float(np.mean(st_iter))
    it_bytes = (mean_it + 1) * gemv_bytes_per_eval(D, N_COLS)
    achieved = it_bytes / (it_ms * 1e-3) / 1e9
    sk_ms = float(np.mean(st_sketch))
    sk_gbs = sketch_bytes(M, N_COLS, D) / (sk_ms * 1e-3) / 1e9
    src = _source_hash(*(f"paper_2004_02480_gb300/csrc/{f}" for f in LOOP_SOURCES))
    loop_kernel = LOOP_KERNELS.get(tuned["gemv_variant"], "k_iterate_gemv")
    traffic = _traffic(loop_kernel + "_100000x500_d5000", src)

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        A64, b64 = s.A.astype(np.float64), s.b.astype(np.float64)
        n_done, dt, cores, its = oracle_solves(A64, b64, s.x_star, args.cpu_seconds)
        n1, dt1, _, its1 = oracle_solves(A64, b64, s.x_star, 0.0, 1, 1, threads=1)
        cpu = {"value": n_done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{n_done} whole oracle solves of this workload (FP64 sketch + literal "
                         f"Algorithm 1 with the residual rows on {cores} OpenMP threads, mean IT "
                         f"{np.mean(its):.1f}) in {dt:.1f} s",
               "single_thread": {"value": n1 / dt1, "unit": UNIT, "cores": 1,
                                 "sample": f"{n1} whole oracle solve, literal Algorithm 1 on one "
                                           f"thread (IT {its1[0]}), {dt1:.1f} s"}}

    value = job["throughput"]
    us_step = 1e3 * it_ms / (mean_it + 1)
    hbm_eq = {"achieved_gbs": achieved, "peak_gbs": hbm, "frac": achieved / hbm,
              "note": "algorithmic bytes = (IT+1) residual evaluations x (4dn + 4(d+2n)); At stays "
                      "on chip, so this is not DRAM traffic (see traffic)"}
    if tuned["gemv_variant"] == 3 or floor_us is None:
        roofline = {"kernel": loop_kernel, "bound": "hbm", "achieved": achieved, "peak": hbm,
                    "unit": "GB/s", "frac": achieved / hbm, "peak_kind": peak_kind,
                    "traffic": traffic}
    else:
        # the loop keeps At on chip; a step is bound by the inter-CTA exchange
        roofline = {"kernel": loop_kernel, "bound": "latency", "achieved": 1e6 / us_step,
                    "peak": 1e6 / floor_us, "unit": "steps/s", "frac": floor_us / us_step,
                    "peak_kind": "measured: csk_exchange_floor on the same CTA count (the step's "
                                 "CTA reduction + mailbox round trip with no arithmetic)",
                    "us_per_step": us_step, "floor_us_per_step": floor_us,
                    "traffic": traffic, "hbm_equivalent": hbm_eq}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": W, "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded N(0,1), paper Section 3 recipe)",
        "config": {"workload": WORKLOAD, "m": M, "n": N_COLS, "d": D, "tol": TOL, "path": "gemv",
                   "parallelism": f"replicas x{world} (independent systems)",
                   "loop": {"grid": tuned["grid"], "variant": LOOP_VARIANTS.get(tuned["gemv_variant"]),
                            "autotuned_us_per_step": tuned["us_per_step"]},
                   "l2": "inputs larger than L2 (A = 200 MB > 129 MB)"},
        "valid": bool(ok),
        "breakdown": {"sketch_ms": sk_ms, "iterate_ms": it_ms, "check_ms": float(np.mean(st_check)),
                      "iters_mean": mean_it, "rse_max": max(r["rse"] for r in recs),
                      "grid": recs[0]["grid"],
                      "sketch_gbs": sk_gbs, "sketch_frac_of_" + peak_kind + "_hbm": sk_gbs / hbm},
        "roofline": roofline,
        "e2e": {"value": job_e2e["throughput"], "unit": UNIT,
                "h2d_bytes_per_step": int(s.A.nbytes + s.b.nbytes + 4 * N_COLS),
                "d2h_bytes_per_step": int(4 * N_COLS + 64), "valid": bool(e2e_ok),
                "call": f"csk_solve_host_many over {E} solves from page-locked host memory "
                        "(the copies of solve k+1 overlap solve k)"},
        "comparison": {"mwrk_unsketched_ms": mwrk["ms"], "mwrk_loop_ms": mwrk["loop_ms"],
                       "mwrk_iters": mwrk["iters"], "mwrk_rse": mwrk["rse"],
                       "mwrk_status": mwrk["status"],
                       "mwrk_update_form_ms": mwrk["update_ms"],
                       "mwrk_update_form_iters": mwrk["update_iters"],
                       "mwrk_update_form_rse": mwrk["update_rse"],
                       "mwrk_loop_kernel": "k_iterate_gemv_stream (A streamed from HBM every step)",
                       "mwrk_loop_gbs": mwrk["stream_gbs"],
                       "mwrk_loop_frac_of_" + peak_kind + "_hbm": mwrk["stream_gbs"] / hbm,
                       "csk_ms": ms / K, "csk_speedup_over_mwrk": mwrk["ms"] / (ms / K),
                       "note": "MWRK (d = 0, Remark 1) on the same A, b on the GPU, median of 3 "
                               "solves; not part of the timed steps"},
        "targets": targets,
        "gpu_launches": launches,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
