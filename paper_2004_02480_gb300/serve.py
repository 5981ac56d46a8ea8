"""Continuous-batching request loop for CSK solves on one GPU.

Requests (one system A x = B with 1..R right-hand sides each, Algorithm 1 per
right-hand side) arrive over time.  The loop runs on several lanes (CUDA
streams), each in ticks of `chunk` steps: a tick is one persistent batched
launch over the units of the lane's admitted requests (csk_batched_iterate,
resuming each unit where the previous tick left it); requests that arrived
meanwhile are admitted against the HBM budget and join the next tick of the
least-loaded lane, their sketch and Gram matrix formed first
(csk_batched_prepare) and kept resident until they finish.  Latency is
measured from a request's arrival to the moment its result is on the host.

With a fixed CTA shape (``threads``) a request's arithmetic does not depend
on the chunking or on the requests it shares a launch with, so its result is
the same alone and in the mix.

The admission and accounting policy (:class:`Admission`) is plain Python and
testable without a GPU; :class:`Server` drives the device through the C ABI.
"""
from __future__ import annotations

import collections
import math
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Request:
    rid: int
    arrival: float           # seconds after the start of the run
    m: int
    n: int
    d: int
    nrhs: int
    seed: int
    # filled in by the server
    t_admit: float = math.nan
    t_done: float = math.nan
    status: list = field(default_factory=list)
    rse: list = field(default_factory=list)
    iters: list = field(default_factory=list)
    x: np.ndarray | None = None


def arena_bytes(r: Request, workspace_bytes: int) -> int:
    """Bytes Server.solve_group carves from the arena for the request alone:
    its info records, A, B, X*, X (each range rounded up to the arena's
    256-byte alignment) and the batched workspace of its one system
    (``workspace_bytes`` = csk_solve_batched_workspace_size of it)."""
    up = lambda v: (int(v) + Arena.ALIGN - 1) // Arena.ALIGN * Arena.ALIGN  # noqa: E731
    return (up(64 * r.nrhs) + up(4 * r.m * r.n) + up(4 * r.m * r.nrhs) + 2 * up(4 * r.n * r.nrhs)
            + up(max(int(workspace_bytes), 256)))


def request_bytes(r: Request) -> int:
    """Device bytes a request holds while admitted: A, B, X*, X, info, and its
    part of the batched workspace (sketch, B sketch, norms, Gram matrix, plus
    sort and operand scratch bounded by its own sizes)."""
    f, al = 4, 256
    up = lambda v: (int(v) + al - 1) // al * al  # noqa: E731
    ldg = (r.d + 31) // 32 * 32
    core = (up(f * r.m * r.n) + up(f * r.m * r.nrhs) + 2 * up(f * r.n * r.nrhs) + up(64 * r.nrhs))
    sketch = up(f * r.d * r.n) + up(f * r.d * r.nrhs) + up(8 * r.d) + up(f * r.d * ldg)
    states = up(32 * r.nrhs) + up(f * r.nrhs * r.d) + up(f * r.nrhs * r.n)   # resumable units
    dp, kp = (r.d + 255) // 256 * 256, (r.n + 63) // 64 * 64
    scratch = up(4 * (2 * r.d + 2 * r.m + 2)) + up(4 * dp * kp) + 2048
    return int(core + sketch + states + scratch + 4096)


class Arena:
    """First-fit allocator of 256-byte aligned ranges in one preallocated
    device buffer, with coalescing on release.  The serving loop carves every
    per-request tensor from it, so steady-state serving makes no cudaMalloc /
    cudaFree (which would synchronise the device) and the HBM budget is a
    real reservation.  Plain Python; the buffer itself is any object the
    caller slices (a torch uint8 tensor on the GPU)."""

    ALIGN = 256

    def __init__(self, nbytes: int):
        self.size = int(nbytes) // self.ALIGN * self.ALIGN
        self.free = [(0, self.size)]          # sorted, non-adjacent (offset, length)

    def alloc(self, nbytes: int) -> int | None:
        n = (int(nbytes) + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        for i, (o, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (o + n, ln - n)
                return o
        return None

    def release(self, off: int, nbytes: int):
        n = (int(nbytes) + self.ALIGN - 1) // self.ALIGN * self.ALIGN
        lo, hi = 0, len(self.free)
        while lo < hi:
            mid = (lo + hi) // 2
            if self.free[mid][0] < off:
                lo = mid + 1
            else:
                hi = mid
        self.free.insert(lo, (off, n))
        # merge with the right and the left neighbour
        if lo + 1 < len(self.free) and off + n == self.free[lo + 1][0]:
            self.free[lo] = (off, n + self.free[lo + 1][1])
            self.free.pop(lo + 1)
        if lo > 0 and self.free[lo - 1][0] + self.free[lo - 1][1] == off:
            self.free[lo - 1] = (self.free[lo - 1][0], self.free[lo - 1][1] + self.free[lo][1])
            self.free.pop(lo)

    def in_use(self) -> int:
        return self.size - sum(ln for _, ln in self.free)


class Admission:
    """FIFO admission under a byte budget, in groups of at most ``max_group``."""

    def __init__(self, budget_bytes: float, max_group: int = 64):
        self.budget = float(budget_bytes)
        self.max_group = max_group
        self.used = 0
        self.waiting: collections.deque[Request] = collections.deque()
        self.peak = 0

    def arrive(self, r: Request):
        if request_bytes(r) > self.budget:
            raise ValueError(f"request {r.rid} alone exceeds the HBM budget")
        self.waiting.append(r)

    def admit(self) -> list[Request]:
        group = []
        while self.waiting and len(group) < self.max_group:
            need = request_bytes(self.waiting[0])
            if self.used + need > self.budget:
                break
            r = self.waiting.popleft()
            self.used += need
            group.append(r)
        self.peak = max(self.peak, self.used)
        return group

    def release(self, group: list[Request]):
        for r in group:
            self.used -= request_bytes(r)
        assert self.used >= 0

    def unadmit(self, group: list[Request]):
        """Return an admitted group to the head of the queue, in order."""
        self.release(group)
        self.waiting.extendleft(reversed(group))


def poisson_requests(rate: float, seconds: float, seed: int, m_range=(2000, 100000),
                     n_range=(20, 500), d_factor=8, rhs_range=(1, 16)) -> list[Request]:
    """Poisson arrivals; m log-uniform, n and the RHS count uniform integers, d = d_factor n."""
    g = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += g.exponential(1.0 / rate)
        if t >= seconds:
            break
        m = int(np.exp(g.uniform(np.log(m_range[0]), np.log(m_range[1]))))
        n = int(g.integers(n_range[0], n_range[1] + 1))
        R = int(g.integers(rhs_range[0], rhs_range[1] + 1))
        out.append(Request(len(out), t, m, n, d_factor * n, R, int(g.integers(1 << 62))))
    return out


class Lane:
    """One stream of the server: its admitted requests and its ticks in flight."""

    def __init__(self, torch, dev, size):
        self.stream = torch.cuda.Stream(dev)
        self.mirrors = [torch.empty(size, dtype=torch.uint8).pin_memory() for _ in range(3)]
        self.active = []          # (request, system, held, info offset)
        self.ticks = collections.deque()   # (tick id, event, mirror, snapshot)
        self.deferred = []        # (tick id, request, held, info offset)
        self.next_tick = 0

    def units(self) -> int:
        return sum(a[0].nrhs for a in self.active)


class Server:
    """Continuous batching at step-chunk granularity on one GPU.

    The server runs `lanes` independent lanes, each on a CUDA stream of its
    own.  A lane's tick is one csk_batched_iterate call over the units of the
    requests it holds, each running at most `chunk` more steps (Algorithm 1
    resumes where the previous tick left it: the requests' sketches, Gram
    matrices and unit states stay resident in their arena ranges).  Requests
    that arrived meanwhile are admitted against the HBM budget, their data
    generated and their sketch and Gram matrix formed (csk_batched_prepare)
    on the lane with the fewest units -- preferring a lane with no tick in
    flight -- and join its next tick.  After each tick the lane's info records
    are copied to the host in one transfer; a request whose units have all
    finished is retired, and its memory is returned once the lane's next
    tick, which still names it with nothing left to do, has completed.  Up to
    two ticks per lane are in flight, and the lanes overlap on the GPU.  With
    a fixed CTA shape a request's arithmetic depends neither on the chunking
    nor on the other requests, so its result is the same alone and in the
    mix."""

    def __init__(self, device="cuda:0", budget_bytes: float = 120e9, threads: int = 256,
                 chunk: int = 512, lanes: int = 8, max_group: int = 64, tol: float = 1e-6,
                 keep_x: bool = False, info_bytes: int = 16 << 20, **_):
        import torch

        from . import csk
        self.torch, self.csk = torch, csk
        self.dev = torch.device(device)
        self.adm = Admission(budget_bytes, max_group)
        # the whole budget is reserved once; requests are carved out of it
        self.arena = Arena(int(budget_bytes))
        self.pool = torch.empty(self.arena.size, dtype=torch.uint8, device=self.dev)
        # info records of every admitted request, read back after each tick
        self.info_arena = Arena(int(info_bytes))
        self.info_pool = torch.zeros(self.info_arena.size, dtype=torch.uint8, device=self.dev)
        self.lanes = [Lane(torch, self.dev, self.info_arena.size) for _ in range(max(1, lanes))]
        self.params = csk.csk_params_default(tol=tol, threads=threads)
        self.chunk = int(chunk)
        self.keep_x = keep_x
        self.launches = 0          # admission groups prepared
        self.ticks = 0

    def _take(self, nbytes: int, held: list):
        off = self.arena.alloc(nbytes)
        if off is None:
            return None
        held.append((off, nbytes))
        return self.pool[off:off + ((nbytes + 3) // 4) * 4]

    def _free(self, r, held, ioff):
        for off, nb in held:
            self.arena.release(off, nb)
        self.info_arena.release(ioff, 64 * r.nrhs)
        self.adm.release([r])

    def _materialise(self, r: Request, synth: list):
        """Arena memory for the request's A, B, X*, X and resident area and
        an info range; None (nothing held) if the arena cannot place it now."""
        f32 = self.torch.float32
        held = []
        ioff = self.info_arena.alloc(64 * r.nrhs)
        if ioff is None:
            return None
        area_bytes = self.csk.csk_batched_area_size(r.n, r.d, r.nrhs)
        parts = [r.m * r.n * 4, r.m * r.nrhs * 4, r.n * r.nrhs * 4, r.n * r.nrhs * 4, area_bytes]
        views = []
        for nb in parts:
            v = self._take(nb, held)
            if v is None:
                for off, nb2 in held:
                    self.arena.release(off, nb2)
                self.info_arena.release(ioff, 64 * r.nrhs)
                return None
            views.append(v)
        A = views[0].view(f32).view(r.m, r.n)
        B = views[1].view(f32).view(r.m, r.nrhs)
        X = views[2].view(f32).view(r.n, r.nrhs)
        Xo = views[3].view(f32).view(r.n, r.nrhs)
        info = self.info_pool[ioff:ioff + 64 * r.nrhs].view(r.nrhs, 64)
        synth.append((A, X, B, r.seed))
        y = self.csk.BatchSystem(A=A, B=B, d=r.d, seed=r.seed, Xstar=X, Xout=Xo, info=info,
                                 area=views[4][:area_bytes])
        return y, held, ioff

    def _admit(self, group, lane: Lane):
        """Data, sketch and Gram matrix of a newly admitted group, enqueued on
        the lane's stream; the requests that could not be placed go back to
        the head of the queue."""
        synth, placed = [], []
        for i, r in enumerate(group):
            got = self._materialise(r, synth)
            if got is None:
                self.adm.unadmit(group[i:])
                break
            placed.append((r,) + got)
        if placed:
            with self.torch.cuda.stream(lane.stream):
                self.csk.csk_synth_systems(synth, device=self.dev)
                self.csk.csk_batched_prepare([p[1] for p in placed])
            self.launches += 1
        return placed

    def warm_up(self):
        """One small untimed request: CUDA context, kernels and libraries warm."""
        r = Request(-1, 0.0, 4000, 32, 256, 2, 12345)
        lane = self.lanes[0]
        self.adm.arrive(r)
        placed = self._admit(self.adm.admit(), lane)
        with self.torch.cuda.stream(lane.stream):
            self.csk.csk_batched_iterate([p[1] for p in placed], self.params, 0)
        lane.stream.synchronize()
        for r, y, held, ioff in placed:
            self._free(r, held, ioff)

    def _tick(self, lane: Lane):
        torch = self.torch
        ys = [a[1] for a in lane.active]
        hi = max(a[3] + 64 * a[0].nrhs for a in lane.active)
        mi = lane.next_tick % len(lane.mirrors)
        with torch.cuda.stream(lane.stream):
            self.csk.csk_batched_iterate(ys, self.params, self.chunk)
            lane.mirrors[mi][:hi].copy_(self.info_pool[:hi], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(lane.stream)
        lane.ticks.append((lane.next_tick, ev, mi, list(lane.active)))
        lane.next_tick += 1
        self.ticks += 1

    def _collect(self, lane: Lane, now):
        """Retire the requests the lane's oldest tick finished."""
        tid, ev, mi, snap = lane.ticks.popleft()
        ev.synchronize()
        keep = []
        for d_tid, r, held, ioff in lane.deferred:
            if d_tid <= tid:
                self._free(r, held, ioff)
            else:
                keep.append((d_tid, r, held, ioff))
        lane.deferred = keep
        host = lane.mirrors[mi].numpy()
        done = set()
        for r, y, held, ioff in snap:
            if not np.isnan(r.t_done):
                continue
            rec = host[ioff:ioff + 64 * r.nrhs]
            recs = np.frombuffer(rec.tobytes(), dtype=self.csk.INFO_DTYPE)
            if (recs["status"] != self.csk.CSK_INPROGRESS).all():
                r.status = [int(v) for v in recs["status"]]
                r.rse = [float(v) for v in recs["rse"]]
                r.iters = [int(v) for v in recs["iters"]]
                if self.keep_x:
                    r.x = y.Xout.cpu().numpy()
                r.t_done = now()
                done.add(r.rid)
                lane.deferred.append((tid + 1, r, held, ioff))   # the next tick still names it
        if done:
            lane.active = [a for a in lane.active if a[0].rid not in done]

    def run(self, requests: list[Request]) -> dict:
        self.warm_up()
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        lanes = self.lanes
        while pending or self.adm.waiting or any(l.active or l.ticks for l in lanes):
            t = now()
            while pending and pending[0].arrival <= t:
                self.adm.arrive(pending.popleft())
            for lane in lanes:
                if lane.deferred and not lane.ticks:       # no tick in flight names them
                    for _, r, held, ioff in lane.deferred:
                        self._free(r, held, ioff)
                    lane.deferred = []
            progressed = False
            if self.adm.waiting:
                lane = min(lanes, key=lambda l: (len(l.ticks) > 0, l.units()))
                group = self.adm.admit()
                if group:
                    placed = self._admit(group, lane)
                    for r in group[:len(placed)]:
                        r.t_admit = now()
                    lane.active += placed
                    progressed = bool(placed)
                    if not placed and not any(l.active or l.ticks for l in lanes):
                        raise RuntimeError("a request does not fit the empty arena: "
                                           "request_bytes underestimates it")
            for lane in lanes:
                if lane.active and len(lane.ticks) < 2:
                    self._tick(lane)
                    progressed = True
                if lane.ticks and (len(lane.ticks) >= 2 or not lane.active) and \
                        lane.ticks[0][1].query():
                    self._collect(lane, now)
                    progressed = True
            if progressed:
                continue
            if not any(l.active or l.ticks for l in lanes) and pending:
                time.sleep(max(0.0, min(1e-3, pending[0].arrival - now())))
            else:
                time.sleep(2e-5)
        for lane in lanes:
            lane.stream.synchronize()
            for _, r, held, ioff in lane.deferred:
                self._free(r, held, ioff)
            lane.deferred = []
        wall = now()
        lat = np.array([r.t_done - r.arrival for r in requests])
        solves = sum(r.nrhs for r in requests)
        ok = all(s == 0 for r in requests for s in r.status)
        return {"requests": len(requests), "solves": solves, "wall_s": wall,
                "solves_per_s": solves / wall, "requests_per_s": len(requests) / wall,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "max_ms": float(lat.max() * 1e3), "groups": self.launches, "ticks": self.ticks,
                "chunk_steps": self.chunk, "lanes": len(lanes), "peak_bytes": self.adm.peak,
                "all_converged": bool(ok), "rse_max": max(max(r.rse) for r in requests)}


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="CSK continuous-batching serving run")
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--seconds", type=float, default=60.0)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=512)
    ap.add_argument("--lanes", type=int, default=8)
    args = ap.parse_args()
    reqs = poisson_requests(args.rate, args.seconds, args.seed)
    srv = Server(budget_bytes=args.budget_gb * 1e9, chunk=args.chunk, lanes=args.lanes)
    print(json.dumps({"workload": f"Poisson {args.rate}/s for {args.seconds} s, m log-uniform "
                      "[2000,100000], n [20,500], d=8n, 1-16 RHS, FP32, A generated on device",
                      **srv.run(reqs)}))


if __name__ == "__main__":
    main()
