"""Continuous-batching request loop for CSK solves on one GPU.

Requests (one system A x = B with 1..R right-hand sides each, Algorithm 1 per
right-hand side) arrive over time.  The loop admits arrived requests while
their device memory fits the HBM budget, launches each admitted group as one
csk_solve_batched call on the next of several CUDA streams -- so work admitted
while earlier groups are still running overlaps with them on the device --
retires finished groups (copying X to the host and freeing their memory) as
soon as their completion event fires, and admits waiting requests as memory
frees up.  Latency is measured from a request's arrival to the moment its
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


def request_bytes(r: Request) -> int:
    """Device bytes a request holds while admitted: A, B, X*, X, info, and its
    part of the batched workspace (sketch, B sketch, norms, Gram matrix, plus
    sort and operand scratch bounded by its own sizes)."""
    f = 4
    ldg = (r.d + 31) // 32 * 32
    core = f * (r.m * r.n + r.m * r.nrhs + 2 * r.n * r.nrhs) + 64 * r.nrhs
    sketch = f * (r.d * r.n + r.d * r.nrhs) + 8 * r.d + f * r.d * ldg
    scratch = 4 * (2 * r.d + 2 * r.m) + 4 * (r.d + 127) // 128 * 128 * ((r.n + 63) // 64 * 64)
    return int(core + sketch + scratch + 4096)


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
                 max_group: int = 64, streams: int = 4, tol: float = 1e-6, keep_x: bool = False):
        import torch

        from . import csk
        self.torch, self.csk = torch, csk
        self.dev = torch.device(device)
        self.adm = Admission(budget_bytes, max_group)
        self.streams = [torch.cuda.Stream(self.dev) for _ in range(streams)]
        self.params = csk.csk_params_default(tol=tol, threads=threads)
        self.keep_x = keep_x
        self.launches = 0

    def _materialise(self, r: Request):
        """The request's data, generated on the device from its seed (stands in
        for a request that arrives with its matrix)."""
        torch = self.torch
        g = torch.Generator(device=self.dev).manual_seed(r.seed & ((1 << 63) - 1))
        A = torch.randn((r.m, r.n), generator=g, device=self.dev, dtype=torch.float32)
        X = torch.randn((r.n, r.nrhs), generator=g, device=self.dev, dtype=torch.float32)
        B = A @ X
        return self.csk.BatchSystem(A=A, B=B, d=r.d, seed=r.seed, Xstar=X)

    def solve_group(self, group: list[Request], stream):
        torch = self.torch
        with torch.cuda.stream(stream):
            systems = [self._materialise(r) for r in group]
            # one info buffer per group, so retiring it is one device-to-host copy
            info = torch.zeros((sum(r.nrhs for r in group), 64), dtype=torch.uint8, device=self.dev)
            o = 0
            for r, y in zip(group, systems):
                y.info = info[o:o + r.nrhs]
                o += r.nrhs
            ws = torch.empty(max(self.csk.csk_solve_batched_workspace_size(systems), 256),
                             dtype=torch.uint8, device=self.dev)
            self.csk.csk_solve_batched(systems, self.params, ws=ws, sync=False)
            self.launches += 1
            ev = torch.cuda.Event()
            ev.record(stream)
        return (systems, info), ws, ev

    def _retire(self, group, systems_info, now):
        systems, info = systems_info
        recs = np.frombuffer(info.cpu().numpy().tobytes(), dtype=self.csk.INFO_DTYPE)
        o = 0
        for r, y in zip(group, systems):
            rr = recs[o:o + r.nrhs]
            o += r.nrhs
            r.status = [int(v) for v in rr["status"]]
            r.rse = [float(v) for v in rr["rse"]]
            r.iters = [int(v) for v in rr["iters"]]
            if self.keep_x:
                r.x = y.Xout.cpu().numpy()
        t = now()
        for r in group:
            r.t_done = t

    def warm_up(self):
        """One small untimed group: CUDA context, kernels and allocator warm."""
        r = Request(-1, 0.0, 4000, 32, 256, 2, 12345)
        (systems, info), ws, ev = self.solve_group([r], self.streams[0])
        ev.synchronize()

    def run(self, requests: list[Request]) -> dict:
        self.warm_up()
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        inflight = []
        k = 0
        while pending or self.adm.waiting or inflight:
            t = now()
            while pending and pending[0].arrival <= t:
                self.adm.arrive(pending.popleft())
            still = []
            for item in inflight:
                group, systems, ws, ev = item
                if ev.query():
                    self._retire(group, systems, now)
                    self.adm.release(group)
                else:
                    still.append(item)
            inflight = still
            group = self.adm.admit()
            if group:
                for r in group:
                    r.t_admit = now()
                systems, ws, ev = self.solve_group(group, self.streams[k % len(self.streams)])
                k += 1
                inflight.append((group, systems, ws, ev))
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
