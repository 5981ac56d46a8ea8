"""Continuous-batching request loop for CSK solves on one GPU.

Requests (one system A x = B with 1..R right-hand sides each, Algorithm 1 per
right-hand side) arrive over time.  Whenever one of several CUDA streams has
no group in flight, the loop admits the arrived requests whose device memory
fits the HBM budget (up to max_group) and launches them as one group -- their
data generated in one call, then one csk_solve_batched call -- on that
stream, so groups overlap on the device and, while every stream is busy,
arrivals accumulate into larger groups.  Finished groups are retired (results
copied to the host, memory returned to the arena) as soon as their completion
event fires.  Latency is measured from a request's arrival to the moment its
result is on the host.

With a fixed CTA shape (``threads``) a request's arithmetic does not depend
on the requests it shares a launch with, so its result is the same alone and
in the mix.

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


class Server:
    """Drives Admission on a GPU: data generation, batched solves, retirement."""

    def __init__(self, device="cuda:0", budget_bytes: float = 120e9, threads: int = 256,
                 max_group: int = 64, streams: int = 8, tol: float = 1e-6, keep_x: bool = False):
        import torch

        from . import csk
        self.torch, self.csk = torch, csk
        self.dev = torch.device(device)
        self.adm = Admission(budget_bytes, max_group)
        # the whole budget is reserved once; requests are carved out of it
        self.arena = Arena(int(budget_bytes))
        self.pool = torch.empty(self.arena.size, dtype=torch.uint8, device=self.dev)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(streams)]
        self.params = csk.csk_params_default(tol=tol, threads=threads)
        self.keep_x = keep_x
        self.launches = 0

    def _take(self, nbytes: int, held: list):
        off = self.arena.alloc(nbytes)
        if off is None:
            return None
        held.append((off, nbytes))
        return self.pool[off:off + ((nbytes + 3) // 4) * 4]

    def _materialise(self, r: Request, held: list, info, synth: list):
        """Arena memory for the request's A, B, X* and X; the request's data
        (a seeded Gaussian system, the stand-in for a request that arrives with
        its matrix) are generated for the whole group in one call."""
        f32 = self.torch.float32
        parts = [r.m * r.n * 4, r.m * r.nrhs * 4, r.n * r.nrhs * 4, r.n * r.nrhs * 4]
        views = []
        for nb in parts:
            v = self._take(nb, held)
            if v is None:
                return None
            views.append(v)
        A = views[0].view(f32).view(r.m, r.n)
        B = views[1].view(f32).view(r.m, r.nrhs)
        X = views[2].view(f32).view(r.n, r.nrhs)
        Xo = views[3].view(f32).view(r.n, r.nrhs)
        synth.append((A, X, B, r.seed))
        return self.csk.BatchSystem(A=A, B=B, d=r.d, seed=r.seed, Xstar=X, Xout=Xo, info=info)

    def solve_group(self, group: list[Request], stream):
        """Launch one group on `stream`; None (nothing held) if the arena is
        too fragmented to place it right now."""
        torch = self.torch
        held = []
        with torch.cuda.stream(stream):
            systems, synth = [], []
            # the group's info records sit together: one copy retires it
            rows = sum(r.nrhs for r in group)
            infos = self._take(64 * rows, held)
            o = 0
            for r in group if infos is not None else ():
                info = infos[64 * o:64 * (o + r.nrhs)].view(r.nrhs, 64)
                o += r.nrhs
                y = self._materialise(r, held, info, synth)
                if y is None:
                    break
                systems.append(y)
            ws = None
            if len(systems) == len(group):
                ws = self._take(max(self.csk.csk_solve_batched_workspace_size(systems), 256), held)
            if ws is None:
                for off, nb in held:
                    self.arena.release(off, nb)
                return None
            self.csk.csk_synth_systems(synth)
            self.csk.csk_solve_batched(systems, self.params, ws=ws, sync=False)
            self.launches += 1
            ev = torch.cuda.Event()
            ev.record(stream)
        return systems, held, ev

    def _retire(self, group, systems, held, now):
        # one device-to-host copy of every info record of the group (the
        # first range taken by solve_group)
        off, nb = held[0]
        recs = np.frombuffer(self.pool[off:off + nb].cpu().numpy().tobytes(),
                             dtype=self.csk.INFO_DTYPE)
        o = 0
        for r, y in zip(group, systems):
            rr = recs[o:o + r.nrhs]
            o += r.nrhs
            r.status = [int(v) for v in rr["status"]]
            r.rse = [float(v) for v in rr["rse"]]
            r.iters = [int(v) for v in rr["iters"]]
            if self.keep_x:
                r.x = y.Xout.cpu().numpy()
        for off, nb in held:
            self.arena.release(off, nb)
        t = now()
        for r in group:
            r.t_done = t

    def warm_up(self):
        """One small untimed group: CUDA context, kernels and libraries warm."""
        r = Request(-1, 0.0, 4000, 32, 256, 2, 12345)
        systems, held, ev = self.solve_group([r], self.streams[0])
        ev.synchronize()
        for off, nb in held:
            self.arena.release(off, nb)

    def run(self, requests: list[Request]) -> dict:
        self.warm_up()
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        # one group in flight per stream: while every stream is busy, arrivals
        # wait in the admission queue and the next free stream takes them as
        # one larger group (batches grow with the load)
        inflight = {}                              # stream index -> group in flight
        while pending or self.adm.waiting or inflight:
            t = now()
            while pending and pending[0].arrival <= t:
                self.adm.arrive(pending.popleft())
            for si in list(inflight):
                group, systems, held, ev = inflight[si]
                if ev.query():
                    self._retire(group, systems, held, now)
                    self.adm.release(group)
                    del inflight[si]
            free = [si for si in range(len(self.streams)) if si not in inflight]
            group = self.adm.admit() if free else []
            launched = None
            if group:
                launched = self.solve_group(group, self.streams[free[0]])
                if launched is None:              # arena fragmented: retry after a retire
                    if not inflight:
                        # nothing will be retired: an empty arena could not place the
                        # group, so waiting would never end
                        raise RuntimeError(f"group of {len(group)} requests does not fit the "
                                           "empty arena: request_bytes underestimates it")
                    self.adm.unadmit(group)
                    group = []
            if group:
                for r in group:
                    r.t_admit = now()
                inflight[free[0]] = (group,) + launched
            elif not inflight and pending:
                time.sleep(max(0.0, min(1e-3, pending[0].arrival - now())))
            else:
                time.sleep(5e-5)
        wall = now()
        lat = np.array([r.t_done - r.arrival for r in requests])
        solves = sum(r.nrhs for r in requests)
        ok = all(s == 0 for r in requests for s in r.status)
        return {"requests": len(requests), "solves": solves, "wall_s": wall,
                "solves_per_s": solves / wall, "requests_per_s": len(requests) / wall,
                "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "max_ms": float(lat.max() * 1e3), "groups": self.launches,
                "peak_bytes": self.adm.peak, "all_converged": bool(ok),
                "rse_max": max(max(r.rse) for r in requests)}


def main():
    import argparse
    import json
    ap = argparse.ArgumentParser(description="CSK continuous-batching serving run")
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--seconds", type=float, default=60.0)
    ap.add_argument("--budget-gb", type=float, default=120.0)
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    reqs = poisson_requests(args.rate, args.seconds, args.seed)
    srv = Server(budget_bytes=args.budget_gb * 1e9)
    print(json.dumps({"workload": f"Poisson {args.rate}/s for {args.seconds} s, m log-uniform "
                      "[2000,100000], n [20,500], d=8n, 1-16 RHS, FP32, A generated on device",
                      **srv.run(reqs)}))


if __name__ == "__main__":
    main()
