"""GPU parity of csk_solve_batched (many systems x many right-hand sides in one
persistent launch).

Each (system, right-hand side) pair must reach RES <= 1e-6 with IT close to
the FP64 oracle's on the same (bit-exact) sketch, agree with the single-system
GPU solve at the same accuracy, and -- with the CTA shape fixed -- give the
same bits alone and inside a larger batch (per-pair arithmetic does not depend
on the co-scheduled work).
"""
import numpy as np
import pytest

import oracle
import stepcheck
from paper_2004_02480_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def csk():
    from paper_2004_02480_gb300 import build, csk as _csk
    build.build()
    return _csk


def _batch(csk, shapes, seed0=0):
    batch, host = [], []
    for i, (m, n, d, R) in enumerate(shapes):
        s = synth.gaussian_multi_rhs(m, n, R, seed0 + i, np.float32)
        batch.append(csk.BatchSystem(A=torch.from_numpy(s.A).to(DEV), B=torch.from_numpy(s.b).to(DEV),
                                     d=d, seed=seed0 + 100 + i,
                                     Xstar=torch.from_numpy(s.x_star.astype(np.float32)).to(DEV)))
        host.append(s)
    return batch, host


SHAPES = [(20000, 120, 1200, 3), (5000, 50, 500, 8), (12000, 200, 2000, 2), (3000, 20, 160, 5),
          (2000, 33, 330, 1), (8000, 77, 770, 4)]


def test_batched_matches_oracle(csk):
    batch, host = _batch(csk, SHAPES)
    p = csk.csk_params_default(max_iter=20000)
    out = csk.csk_solve_batched(batch, p)
    for (m, n, d, R), y, s, (X, infos) in zip(SHAPES, batch, host, out):
        h, sg = oracle.count_sketch_map(y.seed, m, d)
        At, Bt = oracle.sketch_f32_same_order(s.A, s.b, h, sg, d)
        Xh = X.cpu().numpy()
        for r in range(R):
            inf = infos[r]
            ref = oracle.mwrk(At.astype(np.float64), Bt[:, r].astype(np.float64),
                              x_star=s.x_star[:, r], nthreads=4)
            assert inf["status"] == 0 and ref.status == 0, (m, n, d, r, inf)
            assert inf["rse"] <= 1e-6
            xs32 = s.x_star[:, r].astype(np.float32).astype(np.float64)
            rse = np.sum((Xh[:, r] - xs32) ** 2) / np.sum(xs32 ** 2)
            assert abs(inf["rse"] - rse) <= 1e-9 * rse
            assert abs(inf["iters"] - ref.iters) <= max(3, 0.1 * ref.iters), (inf["iters"], ref.iters)
            rr, res = oracle.final_check(At.astype(np.float64), Bt[:, r].astype(np.float64), Xh[:, r])
            assert abs(inf["resid"] - res) <= 1e-6 * res + 1e-9


def test_batched_agrees_with_single_solve(csk):
    shapes = SHAPES[:3]
    batch, host = _batch(csk, shapes, seed0=10)
    out = csk.csk_solve_batched(batch, csk.csk_params_default())
    for (m, n, d, R), y, s, (X, infos) in zip(shapes, batch, host, out):
        for r in range(R):
            p = csk.csk_params_default(d=d, seed=y.seed, path=csk.GRAM)
            b = torch.from_numpy(np.ascontiguousarray(s.b[:, r])).to(DEV)
            xs = torch.from_numpy(s.x_star[:, r].astype(np.float32)).to(DEV)
            x1, inf1 = csk.csk_solve(y.A, b, p, x_star=xs)
            assert inf1["status"] == 0 and infos[r]["status"] == 0
            diff = np.sum((x1.cpu().numpy() - X[:, r].cpu().numpy()) ** 2) / np.sum(s.x_star[:, r] ** 2)
            assert diff <= 4e-6


def test_alone_equals_in_the_mix(csk):
    """With the CTA shape fixed, a pair's result does not depend on which
    other pairs share the launch or on which CTA ran it."""
    batch, host = _batch(csk, SHAPES, seed0=20)
    p = csk.csk_params_default(threads=256)
    mix = [(X.cpu().clone(), [i["iters"] for i in infos]) for X, infos in csk.csk_solve_batched(batch, p)]
    for k in (0, 3, 5):
        y = batch[k]
        alone = csk.BatchSystem(A=y.A, B=y.B, d=y.d, seed=y.seed, Xstar=y.Xstar)
        (X1, inf1), = csk.csk_solve_batched([alone], p)
        assert torch.equal(X1.cpu(), mix[k][0])
        assert [i["iters"] for i in inf1] == mix[k][1]


def test_batched_graph_capture_replay(csk):
    """The batched call makes no synchronising call, so it can be captured
    in a CUDA graph and replayed with the same results."""
    batch, host = _batch(csk, SHAPES[:4], seed0=30)
    p = csk.csk_params_default(threads=256)
    ws = torch.empty(csk.csk_solve_batched_workspace_size(batch), dtype=torch.uint8, device=DEV)
    ref = [(X.cpu().clone()) for X, _ in csk.csk_solve_batched(batch, p, ws=ws)]
    for y in batch:
        y.Xout.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        csk.csk_solve_batched(batch, p, ws=ws, sync=False)   # warm-up outside capture
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    with torch.cuda.graph(g):
        csk.csk_solve_batched(batch, p, ws=ws, sync=False)
    for y in batch:
        y.Xout.zero_()
    g.replay()
    torch.cuda.synchronize()
    for y, X in zip(batch, ref):
        assert torch.equal(y.Xout.cpu(), X)


@pytest.mark.parametrize("refresh", [0, 25])
def test_batched_per_step_replay(csk, refresh):
    """A sample of (system, right-hand side) units of one batched launch,
    logged step by step (i_k and x_k of one unit per launch) and replayed in
    FP64 from the GPU's own iterates: i_k admissible and each step the
    projection of Algorithm 1 within the GRAM path's bound (FP32 rounding,
    split-BF16 error of G_s, drift since the last FP64 recomputation), and the
    oracle's selection from the same iterate equal to i_k wherever it is not
    a near-tie within that bound.  The other units of the launch run as usual."""
    batch, host = _batch(csk, SHAPES, seed0=40)
    L = 20000
    for si, rhs in ((0, 2), (2, 1), (5, 3), (4, 0)):
        m, n, d, R = SHAPES[si]
        ik = torch.full((L,), -1, dtype=torch.int32, device=DEV)
        X = torch.zeros((L, n), dtype=torch.float32, device=DEV)
        p = csk.csk_params_default(refresh_every=refresh, ik_log=ik.data_ptr(), ik_log_len=L,
                                   x_log=X.data_ptr(), x_log_len=L, log_system=si, log_rhs=rhs)
        out = csk.csk_solve_batched(batch, p)
        info = out[si][1][rhs]
        assert info["status"] == 0 and info["rse"] <= 1e-6
        y, s = batch[si], host[si]
        h, sg = oracle.count_sketch_map(y.seed, m, d)
        At, Bt = oracle.sketch_f32_same_order(s.A, s.b, h, sg, d)
        steps = info["iters"]
        ikh = ik.cpu().numpy()
        assert np.all(ikh[:steps] >= 0) and np.all(ikh[steps:] == -1)
        # x_0 .. x_{IT-1} from the log, x_IT = the unit's output
        Xh = np.concatenate([X.cpu().numpy()[:steps], y.Xout[:, rhs].cpu().numpy()[None]])
        rep = stepcheck.replay(At, Bt[:, rhs], Xh, ikh, steps, path="gram",
                               refresh=refresh, oracle=oracle,
                               name=f"batched unit ({m}x{n} d={d}, rhs {rhs}) refresh {refresh}")
        ref = oracle.mwrk(At.astype(np.float64), Bt[:, rhs].astype(np.float64),
                          x_star=s.x_star[:, rhs], log_len=L, nthreads=4)
        rep.prefix, _ = stepcheck.trajectory_prefix(ikh, ref, 1e-3)
        stepcheck.record(rep)
        assert rep.steps == steps and rep.oracle_equal >= 0.9 * steps


def test_tuned_plan_is_used_and_changes_no_result(csk):
    """The batched autotuner times the candidate launch shapes on the batch
    and installs the fastest; a call with threads = grid = 0 then runs that
    shape (its CTA count is reported in info.grid), also inside a CUDA graph,
    and gives the bits of an explicit call with the same thread count."""
    from paper_2004_02480_gb300 import autotune
    batch, host = _batch(csk, SHAPES, seed0=50)
    ws = torch.empty(csk.csk_solve_batched_workspace_size(batch), dtype=torch.uint8, device=DEV)
    best = autotune.tune_batched(batch, ws=ws, use_cache=False)
    assert (best["threads"], best["grid"]) in autotune.batched_candidates(
        torch.cuda.get_device_properties(0).multi_processor_count, max(y.d for y in batch),
        max(y.A.shape[1] for y in batch))
    tuned = [(X.cpu().clone(), [i["grid"] for i in inf], [i["iters"] for i in inf])
             for X, inf in csk.csk_solve_batched(batch, csk.csk_params_default(), ws=ws)]
    assert all(g == best["grid"] for _, gs, _ in tuned for g in gs)
    expl = csk.csk_params_default(threads=best["threads"], grid=best["grid"])
    for (X, _, its), (X2, inf2) in zip(tuned, csk.csk_solve_batched(batch, expl, ws=ws)):
        assert torch.equal(X, X2.cpu()) and its == [i["iters"] for i in inf2]
    # the same plan inside a graph capture
    for y in batch:
        y.Xout.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        csk.csk_solve_batched(batch, csk.csk_params_default(), ws=ws, sync=False)
    g.replay()
    torch.cuda.synchronize()
    for y, (X, _, _) in zip(batch, tuned):
        assert torch.equal(y.Xout.cpu(), X)
    csk.csk_solve_batched_set_plan(batch, 0, 0)            # back to the library default


def test_step_chunks_give_the_same_bits(csk):
    """csk_batched_prepare + csk_batched_iterate with a step budget: units
    report CSK_INPROGRESS between calls, and when every unit has finished,
    X and IT are bit for bit those of one csk_solve_batched call with the
    same CTA shape -- the chunking changes no arithmetic."""
    batch, host = _batch(csk, SHAPES, seed0=60)
    p = csk.csk_params_default(threads=256, max_iter=20000)
    ref = [(X.cpu().clone(), [i["iters"] for i in infos], [i["status"] for i in infos])
           for X, infos in csk.csk_solve_batched(batch, p)]
    chunked = [csk.BatchSystem(A=y.A, B=y.B, d=y.d, seed=y.seed, Xstar=y.Xstar) for y in batch]
    csk.csk_batched_prepare(chunked)
    calls, seen_progress = 0, False
    while True:
        csk.csk_batched_iterate(chunked, p, 37)
        torch.cuda.synchronize()
        calls += 1
        st = [np.frombuffer(y.info.cpu().numpy().tobytes(), dtype=csk.INFO_DTYPE)["status"]
              for y in chunked]
        if any((s == csk.CSK_INPROGRESS).any() for s in st):
            seen_progress = True
            assert calls < 2000
            continue
        break
    assert seen_progress and calls > 1
    for y, (X, its, sts) in zip(chunked, ref):
        recs = np.frombuffer(y.info.cpu().numpy().tobytes(), dtype=csk.INFO_DTYPE)
        assert torch.equal(y.Xout.cpu(), X)
        assert list(recs["iters"]) == its and list(recs["status"]) == sts


def test_systems_join_a_running_batch_between_chunks(csk):
    """Continuous batching at step-chunk granularity: systems prepared after
    the first chunks join the next csk_batched_iterate call beside units
    still running; every unit ends with the bits of its solve alone."""
    batch, host = _batch(csk, SHAPES, seed0=70)
    p = csk.csk_params_default(threads=256)
    first = [csk.BatchSystem(A=y.A, B=y.B, d=y.d, seed=y.seed, Xstar=y.Xstar) for y in batch[:3]]
    late = [csk.BatchSystem(A=y.A, B=y.B, d=y.d, seed=y.seed, Xstar=y.Xstar) for y in batch[3:]]
    csk.csk_batched_prepare(first)
    csk.csk_batched_iterate(first, p, 50)
    csk.csk_batched_iterate(first, p, 50)
    csk.csk_batched_prepare(late)
    active = first + late
    for _ in range(400):
        csk.csk_batched_iterate(active, p, 64)
        torch.cuda.synchronize()
        if all((np.frombuffer(y.info.cpu().numpy().tobytes(), dtype=csk.INFO_DTYPE)["status"]
                != csk.CSK_INPROGRESS).all() for y in active):
            break
    for y in active:
        alone = csk.BatchSystem(A=y.A, B=y.B, d=y.d, seed=y.seed, Xstar=y.Xstar)
        (X1, inf1), = csk.csk_solve_batched([alone], p)
        recs = np.frombuffer(y.info.cpu().numpy().tobytes(), dtype=csk.INFO_DTYPE)
        assert torch.equal(y.Xout.cpu(), X1.cpu())
        assert list(recs["iters"]) == [i["iters"] for i in inf1]
        assert all(s == 0 for s in recs["status"]) and float(recs["rse"].max()) <= 1e-6
