"""Host-side checks of the serving loop's admission policy and request stream
(no GPU): FIFO order, the HBM budget is never exceeded, memory is returned on
release, and the synthetic arrivals follow the stated distributions."""
import numpy as np
import pytest

from paper_2004_02480_gb300.serve import Admission, Request, poisson_requests, request_bytes


def _req(i, m=10000, n=100, R=4):
    return Request(i, 0.01 * i, m, n, 8 * n, R, i)


def test_fifo_and_budget():
    reqs = [_req(i, m=2000 + 1000 * i) for i in range(20)]
    budget = sum(request_bytes(r) for r in reqs[:5]) + 10
    adm = Admission(budget, max_group=3)
    for r in reqs:
        adm.arrive(r)
    admitted = []
    groups = []
    while adm.waiting:
        g = adm.admit()
        assert adm.used <= budget
        if not g:
            adm.release(groups.pop(0))
            continue
        groups.append(g)
        admitted += g
        assert len(g) <= 3
    assert [r.rid for r in admitted] == list(range(20))
    for g in groups:
        adm.release(g)
    assert adm.used == 0 and adm.peak <= budget


def test_oversize_request_rejected():
    adm = Admission(1000)
    with pytest.raises(ValueError):
        adm.arrive(_req(0))


def test_head_of_line_waits_for_memory():
    big, small = _req(0, m=100000, n=500, R=16), _req(1, m=2000, n=20, R=1)
    adm = Admission(request_bytes(big) + request_bytes(small) // 2)
    first = _req(2, m=50000, n=100, R=2)
    adm.arrive(first)
    assert adm.admit() == [first]
    adm.arrive(big)
    adm.arrive(small)
    assert adm.admit() == []            # big does not fit; FIFO keeps small behind it
    adm.release([first])
    assert adm.admit() == [big]


def test_poisson_stream_statistics():
    rate, T = 2000.0, 5.0
    reqs = poisson_requests(rate, T, seed=1)
    assert abs(len(reqs) - rate * T) < 5 * np.sqrt(rate * T)
    t = np.array([r.arrival for r in reqs])
    assert np.all(np.diff(t) > 0) and t[-1] < T
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / rate) < 0.05 / rate
    m = np.array([r.m for r in reqs]); n = np.array([r.n for r in reqs])
    assert m.min() >= 2000 and m.max() <= 100000 and n.min() >= 20 and n.max() <= 500
    assert all(r.d == 8 * r.n for r in reqs) and all(1 <= r.nrhs <= 16 for r in reqs)
    # log-uniform m: log(m) has the uniform mean
    assert abs(np.log(m).mean() - (np.log(2000) + np.log(100000)) / 2) < 0.05


def test_arena_first_fit_and_coalescing():
    from paper_2004_02480_gb300.serve import Arena
    a = Arena(10 * 256)
    x = a.alloc(256); y = a.alloc(300); z = a.alloc(256)
    assert (x, y, z) == (0, 256, 768) and a.in_use() == 4 * 256
    assert a.alloc(7 * 256) is None                 # only 6 blocks left
    a.release(y, 300)
    assert a.alloc(512) == 256                      # first fit reuses the hole
    a.release(256, 512); a.release(x, 256); a.release(z, 256)
    assert a.free == [(0, 10 * 256)] and a.in_use() == 0
    rng = __import__("numpy").random.default_rng(0)
    live = []
    for _ in range(2000):
        if live and rng.random() < 0.5:
            o, n = live.pop(int(rng.integers(len(live))))
            a.release(o, n)
        else:
            n = int(rng.integers(1, 1000))
            o = a.alloc(n)
            if o is not None:
                live.append((o, n))
        spans = sorted((o, (n + 255) // 256 * 256) for o, n in live)
        for (o1, n1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + n1 <= o2                    # no overlap
        assert a.in_use() == sum(n for _, n in spans)


def test_request_bytes_covers_what_the_arena_carves():
    """request_bytes (the admission estimate) is at least what solve_group
    carves from the arena for the request alone -- its tensors plus the
    library's batched workspace for its one system -- over the serving size
    ranges, so a lone admitted request always fits an empty arena."""
    import ctypes

    from paper_2004_02480_gb300 import csk
    from paper_2004_02480_gb300.serve import arena_bytes
    L = csk.lib()
    rng = np.random.default_rng(5)
    shapes = [(2000, 20, 1), (100000, 500, 16), (2000, 500, 16), (100000, 20, 1), (2001, 21, 3)]
    shapes += [(int(np.exp(rng.uniform(np.log(2000), np.log(100000)))), int(rng.integers(20, 501)),
                int(rng.integers(1, 17))) for _ in range(200)]
    for m, n, R in shapes:
        r = Request(0, 0.0, m, n, 8 * n, R, 1)
        one = csk.csk_system(256, m, n, n, 256, R, R, 0, r.d, 1, None, 256, 256, 256)
        ws = L.csk_solve_batched_workspace_size((csk.csk_system * 1)(one), 1)
        assert ws > 0
        assert request_bytes(r) >= arena_bytes(r, ws), (m, n, R)
