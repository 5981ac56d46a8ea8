"""GPU parity of the host-memory entry points.

csk_solve_host copies the problem in, runs csk_solve and copies x and the
info record back: its results must be bit-identical to csk_solve on the same
device data, for a packed A (one linear copy) and a strided one (a 2-D
copy).  csk_solve_host_many overlaps the next problem's copies with the
current solve; every problem's x and info must be bit-identical to its own
csk_solve_host call, for problems of different shapes, page-locked or not,
and the first problem's iteration count must match the FP64 oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_2004_02480_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def csk():
    from paper_2004_02480_gb300 import build, csk as _csk
    build.build()
    return _csk


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.mark.parametrize("pad", [0, 3])
def test_solve_host_equals_device_solve(csk, pad):
    m, n, d = 20000, 96, 960
    s = synth.gaussian_system(m, n, 5, np.float32)
    Ah = np.zeros((m, n + pad), np.float32)
    Ah[:, :n] = s.A
    Ah = _pinned(Ah)[:, :n] if pad else _pinned(s.A)
    p = csk.csk_params_default(d=d, seed=11)
    xs = s.x_star.astype(np.float32)
    ws = csk._workspace(csk.csk_solve_host_workspace_size(m, n, csk.CSK_F32, p), DEV)
    x1, inf1, rc = csk.csk_solve_host(Ah, _pinned(s.b), p, x_star=_pinned(xs), ws=ws)
    assert rc == 0 and inf1["status"] == 0
    A = torch.from_numpy(np.ascontiguousarray(s.A)).to(DEV)
    x2, inf2 = csk.csk_solve(A, torch.from_numpy(s.b).to(DEV), p, x_star=torch.from_numpy(xs).to(DEV))
    assert np.array_equal(x1, x2.cpu().numpy())
    assert inf1["iters"] == inf2["iters"] and inf1["rse"] == inf2["rse"]


def test_solve_host_many_equals_one_by_one(csk):
    shapes = [(20000, 96, 960), (12000, 40, 400), (30000, 128, 1280), (20000, 96, 960),
              (5000, 20, 200)]
    p = csk.csk_params_default(d=960, seed=5)
    probs, singles, hosts = [], [], []
    for i, (m, n, _) in enumerate(shapes):
        s = synth.gaussian_system(m, n, 40 + i, np.float32)
        xs = s.x_star.astype(np.float32)
        pin = i % 2 == 0                                 # mix page-locked and pageable
        f = _pinned if pin else np.ascontiguousarray
        probs.append(csk.HostProblem(A=f(s.A), b=f(s.b), x_star=f(xs)))
        hosts.append(s)
    ws = csk._workspace(csk.csk_solve_host_many_workspace_size(probs, p), DEV)
    rc = csk.csk_solve_host_many(probs, p, ws=ws)
    assert rc == 0
    for q in probs:
        m, n = q.A.shape
        w1 = csk._workspace(csk.csk_solve_host_workspace_size(m, n, csk.CSK_F32, p), DEV)
        x1, inf1, rc1 = csk.csk_solve_host(q.A, q.b, p, x_star=q.x_star, ws=w1)
        assert rc1 == 0
        inf = csk.info_dict(q.info)
        assert np.array_equal(q.x_out, x1)
        assert inf["iters"] == inf1["iters"] and inf["rse"] == inf1["rse"] and inf["status"] == 0
        singles.append(inf1)
    # the first problem against the FP64 oracle on the same sketch
    s = hosts[0]
    h, sg = oracle.count_sketch_map(p.seed, s.A.shape[0], p.d)
    At, bt = oracle.sketch_f32_same_order(s.A, s.b[:, None], h, sg, p.d)
    ref = oracle.mwrk(At.astype(np.float64), bt[:, 0].astype(np.float64), x_star=s.x_star,
                      nthreads=4)
    assert abs(singles[0]["iters"] - ref.iters) <= max(3, 0.05 * ref.iters)


def test_solve_host_many_reports_first_bad_status(csk):
    m, n = 8000, 32
    p = csk.csk_params_default(d=320, seed=3, max_iter=5)        # the cap ends every solve
    probs = []
    for i in range(3):
        s = synth.gaussian_system(m, n, 70 + i, np.float32)
        probs.append(csk.HostProblem(A=_pinned(s.A), b=_pinned(s.b),
                                     x_star=_pinned(s.x_star.astype(np.float32))))
    ws = csk._workspace(csk.csk_solve_host_many_workspace_size(probs, p), DEV)
    assert csk.csk_solve_host_many(probs, p, ws=ws) == csk.CSK_MAXITER
    assert all(csk.info_dict(q.info)["status"] == csk.CSK_MAXITER for q in probs)
    assert all(csk.info_dict(q.info)["iters"] == 5 for q in probs)
