"""GPU parity of the split-BF16 Gram matrix (tcgen05) and of the GRAM residual
path of the iteration.

Tolerances (derived, not tuned):
* GPU G against the oracle's split product (the same BF16 operands, summed
  exactly in binary64): the difference is the tensor core's FP32
  accumulation.  Measured on GB300 it rounds toward zero once per
  K = 16 instruction (every GPU value lies on the zero side of the exact
  split sum), so over M = 3 * k_pad / 16 instructions
  |G - G_split| <= (M + 16) 2^-23 (|A||A|^T)_ij, where k_pad = 64 ceil(n/64).
  An RMS check adds sensitivity: a dropped hi*lo segment would leave a
  relative RMS error near 2^-9, the accumulation about 1e-5 or less.
* GPU G against the exact product: the split drops lo*lo and rounds lo
  (2^-16 relative per product) on top of the accumulation above, so
  |G - A A^T| <= (2^-14 + (M + 16) 2^-23) (|A||A|^T)_ij.
* G is exactly symmetric and G_jj = fl32(||A_j||^2).
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


def _check_G(G, At, rows=None, Gs_rows=None):
    A64 = At.astype(np.float64)
    d, n = At.shape
    rows = np.arange(d) if rows is None else np.asarray(rows)
    Gs = oracle.gram_split_bf16(At) if Gs_rows is None else Gs_rows
    if Gs_rows is None:
        Gs = Gs[rows]
    scale = np.abs(A64[rows]) @ np.abs(A64).T
    exact = A64[rows] @ A64.T
    Gr = G[rows].astype(np.float64)
    M = 3 * ((n + 63) // 64 * 64) // 16
    acc = (M + 16) * 2.0 ** -23
    assert np.all(np.abs(Gr - Gs) <= acc * scale)
    assert np.all(np.abs(Gr - exact) <= (2.0 ** -14 + acc) * scale)
    rms = np.sqrt(np.mean((Gr - Gs) ** 2) / max(np.mean(Gs ** 2), 1e-300))
    assert rms <= 3e-5, rms


@pytest.mark.parametrize("d,n", [(1, 1), (5, 3), (300, 70), (1000, 256), (129, 65), (777, 1000)])
def test_gram_matches_split_oracle(csk, d, n):
    rng = np.random.default_rng(d * 1000 + n)
    At = rng.standard_normal((d, n)).astype(np.float32)
    At_t = torch.from_numpy(At).to(DEV)
    N2 = torch.from_numpy(oracle.row_norms2(At)).to(DEV)
    G = csk.csk_gram(At_t, N2).cpu().numpy()
    G_nodiag = csk.csk_gram(At_t).cpu().numpy()
    torch.cuda.synchronize()
    assert np.array_equal(G, G.T)                                   # mirrored tiles
    assert np.array_equal(np.diag(G), oracle.row_norms2(At).astype(np.float32))
    off = ~np.eye(d, dtype=bool)
    assert np.array_equal(G[off], G_nodiag[off])
    _check_G(G_nodiag, At)


def test_gram_full_precision_form_sampled_rows(csk):
    """d = 20000, n = 1000 (the precision-form sketch size): sampled rows."""
    d, n = 20000, 1000
    g = torch.Generator(device=DEV).manual_seed(3)
    At_t = torch.randn((d, n), generator=g, device=DEV, dtype=torch.float32)
    G = csk.csk_gram(At_t)
    torch.cuda.synchronize()
    At = At_t.cpu().numpy()
    rows = np.random.default_rng(0).choice(d, 12, replace=False)
    rows = np.concatenate([rows, [0, d - 1, 127, 128, 19999 - 128]])
    Gs = oracle.gram_split_bf16_rows(At, rows)
    Gh = G[torch.from_numpy(rows).to(DEV)].cpu().numpy()
    full = np.zeros((d, d), np.float32)
    full[rows] = Gh
    _check_G(full, At, rows=rows, Gs_rows=Gs)
    # symmetry on the sampled rows against the matching columns
    Gc = G[:, torch.from_numpy(rows).to(DEV)].cpu().numpy().T
    assert np.array_equal(Gh, Gc)


def _solve(csk, s, d, seed, xlog=0, **kw):
    A, b = torch.from_numpy(s.A).to(DEV), torch.from_numpy(s.b).to(DEV)
    xs = torch.from_numpy(s.x_star.astype(np.float32)).to(DEV)
    ik = torch.full((20000,), -1, dtype=torch.int32, device=DEV)
    n = s.A.shape[1]
    X = torch.zeros((max(xlog, 1), n), dtype=torch.float32, device=DEV)
    p = csk.csk_params_default(d=d, seed=seed, ik_log=ik.data_ptr(), ik_log_len=20000,
                               x_log=X.data_ptr() if xlog else None, x_log_len=xlog, **kw)
    x, info = csk.csk_solve(A, b, p, x_star=xs)
    if xlog:
        return x.cpu().numpy(), info, ik.cpu().numpy(), X.cpu().numpy()
    return x.cpu().numpy(), info, ik.cpu().numpy()


@pytest.mark.parametrize("refresh", [0, 50])
def test_gram_path_converges_like_oracle(csk, refresh):
    """GRAM path on 100000 x 500, d = 5000: RES <= 1e-6, i_k prefix equal to
    the FP64 oracle's up to the first near-tie, IT within 5 %, and every step
    replayed in FP64 from the GPU's own iterate: i_k admissible and the step
    the projection of Algorithm 1 within the GRAM path's bound (FP32 rounding
    + split-BF16 error of G + drift since the last FP64 refresh), and the
    oracle's selection from the same iterate equal to i_k wherever it is not
    a near-tie within that bound."""
    m, n, d, seed = 100000, 500, 5000, 2
    s = synth.gaussian_system(m, n, seed, np.float32)
    x, info, ik, X = _solve(csk, s, d, seed, xlog=20000, path=csk.GRAM, refresh_every=refresh)
    h, sg = oracle.count_sketch_map(seed, m, d)
    At, bt = oracle.sketch_f32_same_order(s.A, s.b, h, sg, d)
    ref = oracle.mwrk(At.astype(np.float64), bt.astype(np.float64), x_star=s.x_star,
                      log_len=20000, nthreads=8)
    assert info["status"] == 0 and info["rse"] <= 1e-6 and info["path"] == csk.GRAM
    name = f"FP32 GRAM 100000x500 d=5000 refresh {refresh}"
    K, k_tau = stepcheck.trajectory_prefix(ik, ref, 1e-3)
    stepcheck.REPORT.append(f"{name}: i_k equal to the oracle's own trajectory for the first {K} "
                            f"steps (first near-tie, gap < 0.001, at step {k_tau})")
    steps = info["iters"]
    Xh = np.concatenate([X[:steps], x[None]])          # x_0 .. x_{IT-1} logged, x_IT returned
    rep = stepcheck.replay(At, bt, Xh, ik, steps, path="gram", refresh=refresh, name=name,
                           oracle=oracle)
    stepcheck.record(rep)
    assert rep.steps == steps and rep.oracle_compared == steps
    # without refresh the drift term grows over the whole solve and the
    # bound forces fewer steps (late steps have small residuals)
    assert rep.forced >= (steps // 2 if refresh else steps // 8)
    assert rep.oracle_equal >= 0.9 * steps
    assert abs(info["iters"] - ref.iters) <= 0.05 * ref.iters


def test_gram_path_small_and_ragged(csk):
    for (m, n, d) in [(5000, 70, 300), (3000, 1, 10), (20000, 129, 1000)]:
        s = synth.gaussian_system(m, n, n, np.float32)
        x, info, _ = _solve(csk, s, d, 4, path=csk.GRAM, refresh_every=25)
        h, sg = oracle.count_sketch_map(4, m, d)
        At, bt = oracle.sketch(s.A.astype(np.float64), s.b.astype(np.float64), h, sg, d)
        ref = oracle.mwrk(At, bt, x_star=s.x_star)
        assert info["status"] == ref.status == 0 and info["rse"] <= 1e-6
        assert abs(info["iters"] - ref.iters) <= max(3, 0.1 * ref.iters)


def test_precision_form_full_size(csk):
    """The precision-form workload: A 1e6 x 1000 = G diag(sigma) Q (sigma
    log-spaced 1..1e3), d = 20000, GRAM path with FP64 refresh every 100
    steps.  With kappa = 1e3 RES <= 1e-6 lies far beyond the 20000-step cap
    of Section 3, so the solve ends at the cap; checked: the status, the FP64
    final RES against a host recomputation, monotone decrease of the error,
    and the first 200 steps against the FP64 oracle on the same sketch."""
    m, n, d, seed = 1_000_000, 1000, 20000, 0
    A, b, xs64 = synth.conditioned_system_device(m, n, seed, 1e3, DEV)
    xs = xs64.float()
    L = 20000
    X = torch.zeros((L, n), dtype=torch.float32, device=DEV)
    ik = torch.full((L,), -1, dtype=torch.int32, device=DEV)
    p = csk.csk_params_default(d=d, seed=seed, path=csk.GRAM, refresh_every=100, max_iter=L,
                               ik_log=ik.data_ptr(), ik_log_len=L, x_log=X.data_ptr(), x_log_len=L)
    x, info = csk.csk_solve(A, b, p, x_star=xs)
    assert info["status"] == 1 and info["iters"] == L
    xs_h = xs.double().cpu().numpy()
    xh = x.double().cpu().numpy()
    rse = np.sum((xh - xs_h) ** 2) / np.sum(xs_h ** 2)
    assert abs(info["rse"] - rse) <= 1e-9 * rse
    Xh = X.double().cpu().numpy()
    e2 = np.sum((Xh - xs_h) ** 2, axis=1)
    assert e2[-1] < 0.5 * e2[0]
    # exact projections never increase the error; allow FP32 noise
    assert np.all(e2[1:] <= e2[:-1] * (1 + 1e-4))
    # first 200 steps against the FP64 oracle on the GPU's (bit-exact) sketch
    sk = csk.csk_sketch(A, d, seed, b)
    At = sk.At.double().cpu().numpy()
    bt = sk.bt.double().cpu().numpy()
    ref = oracle.mwrk(At, bt, x_star=xs_h, tol=0.0, max_iter=200, log_len=201, nthreads=16)
    gap = ref.gap
    k_tau = int(np.argmax(gap < 1e-3)) if np.any(gap < 1e-3) else len(gap)
    K, _ = stepcheck.trajectory_prefix(ik.cpu().numpy()[:200], ref, 1e-3)
    assert K >= min(200, k_tau)
    assert abs(e2[200] - ref.err2[200]) <= 0.1 * ref.err2[200]
    # every step up to 300 (three FP64 refreshes) replayed from the GPU's iterate
    rep = stepcheck.replay(At, bt, Xh, ik.cpu().numpy(), 300, path="gram", refresh=100,
                           name="FP32 GRAM precision form 1e6x1000 d=20000 refresh 100",
                           oracle=oracle, oracle_steps=set(range(0, 300, 10)), nthreads=16)
    rep.prefix = K
    stepcheck.record(rep)
    assert rep.steps == 300


GRAM_CHILD = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_2004_02480_gb300 import csk
out = {}
for d, n in [(300, 70), (1000, 256), (777, 1000), (5000, 130)]:
    g = torch.Generator(device="cuda:0").manual_seed(d + n)
    At = torch.randn((d, n), generator=g, device="cuda:0")
    out[f"{d}x{n}"] = csk.csk_gram(At).cpu().numpy()
np.savez(sys.argv[2], **out)
"""


def test_gram_pair_kernel_equals_single_cta_kernel(csk, tmp_path):
    """The paired-CTA Gram kernel (B panels shared by multicast between the
    two CTAs of a cluster, the default) and the one-CTA kernel
    (CSK_GRAM_PAIR=0) issue the same MMAs on the same operands: G must be the
    same bits, including shapes whose last pair holds a tile below the
    diagonal and ragged d."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    files = {}
    for mode in ("1", "0"):
        f = str(tmp_path / f"g{mode}.npz")
        r = subprocess.run([sys.executable, "-c", GRAM_CHILD, root, f], capture_output=True,
                           text=True, timeout=600, env={**os.environ, "CSK_GRAM_PAIR": mode})
        assert r.returncode == 0, r.stderr[-3000:]
        files[mode] = np.load(f)
    for k in files["1"].files:
        a, b = files["1"][k], files["0"][k]
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32)), k


@pytest.mark.parametrize("d,n", [(777, 100), (2000, 300), (300, 1000), (5002, 130), (4998, 64)])
def test_gram_tensor_store_epilogue_equals_lane_stores(csk, d, n):
    """Tiles above the diagonal band leave the tensor cores through shared
    memory and TMA tensor stores (each 32 x 32 block inside G and its
    transpose) when G's rows are 16-byte aligned; with a row stride that is
    not (ldg % 4 != 0) the same tiles are written by per-lane stores.  Both
    must give the same bits, G exactly symmetric, and nothing written past
    column d (d = 777 and 5000 +- 2 are not multiples of 4: a tensor store
    crossing column d would write the rest of its 16-byte granule)."""
    g = torch.Generator(device=DEV).manual_seed(d * 7 + n)
    At = torch.randn((d, n), generator=g, device=DEV)
    ld_odd = d + (1 if (d + 1) % 4 else 2)
    Ga = csk.csk_gram(At)                        # ldg = round_up(d, 32): tensor stores
    Gb = csk.csk_gram(At, ldg=ld_odd)            # per-lane stores
    torch.cuda.synchronize()
    a, b = Ga.cpu().numpy(), Gb.cpu().numpy()
    assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
    assert np.array_equal(a, a.T)
    _check_G(a, At.cpu().numpy(), rows=np.arange(0, d, max(1, d // 40)))
    # padding columns past d are untouched on both store paths
    L = csk.lib()
    ws = csk._workspace(int(L.csk_gram_workspace_size(d, n)), torch.device(DEV))
    for ld in (ld_odd, (d + 31) // 32 * 32 + 32):
        pad = torch.full((d, ld), 7.0, device=DEV)
        rc = L.csk_gram(At.data_ptr(), d, n, None, pad.data_ptr(), ld, None, ws.data_ptr(),
                        ws.numel(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert rc == 0
        assert bool((pad[:, d:] == 7.0).all()), ld
        assert np.array_equal(pad[:, :d].cpu().numpy().view(np.uint32), b.view(np.uint32)), ld
