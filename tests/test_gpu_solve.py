"""GPU parity of csk_solve (Algorithm 1 end to end) against the CPU oracle.

* FP64 (the 2000 x 50, d = 500 workload): the GPU iterates in FP64 on a sketch
  that is bit-identical to the oracle's, so the row sequence i_k must equal
  the oracle's at every step whose selection gap exceeds 1e-9 (only rounding
  order differs), and IT must match.
* FP32 (the 100000 x 500, d = 5000 workload): the oracle iterates in FP64 on
  the GPU's (bit-exact) FP32 sketch; i_k must match over the first
  min(1000, k_tau) steps, k_tau being the first step whose relative gap
  between the two best weighted residuals is below tau = 1e-3 (FP32 residuals
  carry ~1e-6 relative error at n = 500).
* Every solve must reach RES <= 1e-6 and the final FP64 check must agree with
  the oracle's recomputation.
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


def _to(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _solve(csk, sysm, d, seed, log=0, xlog=0, **kw):
    A, b, xs = _to(sysm.A), _to(sysm.b), _to(sysm.x_star.astype(sysm.A.dtype))
    ik = torch.full((max(log, 1),), -1, dtype=torch.int32, device=DEV)
    n = sysm.A.shape[1]
    X = torch.zeros((max(xlog, 1), n), dtype=A.dtype, device=DEV)
    p = csk.csk_params_default(d=d, seed=seed, ik_log=ik.data_ptr() if log else None,
                               ik_log_len=log, x_log=X.data_ptr() if xlog else None,
                               x_log_len=xlog, **kw)
    x, info = csk.csk_solve(A, b, p, x_star=xs)
    if xlog:
        return x.cpu().numpy(), info, ik.cpu().numpy()[:log], X.cpu().numpy()
    return x.cpu().numpy(), info, ik.cpu().numpy()[:log]


def _check_steps(At, bt, X, ik, steps, u, name="", oracle_check=True):
    """Every GPU step replayed in FP64 from the GPU's own iterate x_k
    (stepcheck.replay, GEMV bound): i_k admissible under the rounding bound,
    the projection exact to it, and the oracle's own selection from x_k equal
    to i_k wherever that choice is not a near-tie within the bound."""
    rep = stepcheck.replay(At, bt, X, ik, steps, path="gemv", u=u, name=name,
                           oracle=oracle if oracle_check else None)
    stepcheck.record(rep)
    if oracle_check:
        assert rep.oracle_equal >= rep.oracle_forced
    return rep.steps


def _compare_prefix(ik_gpu, ref, tau, name=""):
    K, k_tau = stepcheck.trajectory_prefix(ik_gpu, ref, tau)
    stepcheck.REPORT.append(f"{name}: i_k equal to the oracle's own trajectory for the first {K} "
                            f"steps (first near-tie, gap < {tau:g}, at step {k_tau})")
    return K


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_config1_fp64_matches_oracle(csk, seed):
    m, n, d = 2000, 50, 500
    s = synth.gaussian_system(m, n, seed, np.float64)
    x, info, ik = _solve(csk, s, d, seed, log=2000)
    h, sg = oracle.count_sketch_map(seed, m, d)
    At, bt = oracle.sketch(s.A, s.b, h, sg, d)
    ref = oracle.mwrk(At, bt, x_star=s.x_star, tol=1e-6, log_len=2000)
    assert info["status"] == 0 and ref.status == 0
    assert info["rse"] <= 1e-6
    K = _compare_prefix(ik, ref, 1e-9, name=f"FP64 2000x50 d=500 seed {seed}")
    if K == ref.iters:
        assert info["iters"] == ref.iters
    assert np.sum((x - ref.x) ** 2) / np.sum(s.x_star ** 2) <= 1e-6
    rse, res = oracle.final_check(At, bt, x, s.x_star)
    assert abs(info["rse"] - rse) <= 1e-12 * max(rse, 1e-30) + 1e-18
    assert abs(info["resid"] - res) <= 1e-10 * res + 1e-18
    assert info["empty_rows"] == int(np.sum(np.sum(At ** 2, axis=1) == 0))


@pytest.mark.parametrize("grid", [0, 1, 3, 64])
def test_grid_shape_does_not_change_result(csk, grid):
    """Every CTA count gives the same iterates: each row's residual is one
    warp's dot product whichever CTA owns it, and every CTA reduces the same
    candidates, so i_k and x do not depend on the grid."""
    s = synth.gaussian_system(3000, 40, 7, np.float64)
    x0, i0, _ = _solve(csk, s, 400, 7, grid=1)
    x1, i1, _ = _solve(csk, s, 400, 7, grid=grid)
    assert i0["iters"] == i1["iters"]
    np.testing.assert_allclose(x1, x0, rtol=0, atol=1e-12 * np.abs(x0).max())


def test_config2_fp32_gemv_matches_oracle(csk):
    """100000 x 500 FP32, d = 5000: exact i_k prefix up to the first near-tie
    (tau = 1e-3), every step valid within FP32 rounding, RES <= 1e-6, IT
    within 5 % of the FP64 oracle's on the same sketch."""
    m, n, d, seed = 100000, 500, 5000, 0
    s = synth.gaussian_system(m, n, seed, np.float32)
    x, info, ik, X = _solve(csk, s, d, seed, log=20000, xlog=20000, path=csk.GEMV)
    h, sg = oracle.count_sketch_map(seed, m, d)
    At32, bt32 = oracle.sketch_f32_same_order(s.A, s.b, h, sg, d)
    ref = oracle.mwrk(At32.astype(np.float64), bt32.astype(np.float64), x_star=s.x_star,
                      tol=1e-6, log_len=20000, nthreads=8)
    assert info["status"] == 0 and info["rse"] <= 1e-6
    K = _compare_prefix(ik, ref, 1e-3, name="FP32 GEMV 100000x500 d=5000 seed 0")
    assert K >= 1
    Xh = np.concatenate([X[:info["iters"]], x[None]])   # x_0 .. x_{IT-1} logged, x_IT returned
    assert _check_steps(At32, bt32, Xh, ik, info["iters"], 2.0 ** -24,
                        name="FP32 GEMV 100000x500 d=5000 seed 0") == info["iters"]
    assert abs(info["iters"] - ref.iters) <= 0.05 * ref.iters
    assert np.sum((x - ref.x) ** 2) / np.sum(s.x_star ** 2) <= 4e-6


def test_unsketched_mwrk_matches_oracle(csk):
    """Remark 1: d = 0 runs MWRK on A itself."""
    s = synth.gaussian_system(20000, 100, 3, np.float32)
    x, info, ik, X = _solve(csk, s, 0, 0, log=5000, xlog=5000)
    ref = oracle.mwrk(s.A.astype(np.float64), s.b.astype(np.float64), x_star=s.x_star,
                      log_len=5000, nthreads=8)
    assert info["status"] == 0 and info["rse"] <= 1e-6 and info["rows"] == 20000
    _compare_prefix(ik, ref, 1e-3)
    _check_steps(s.A, s.b, X, ik, info["iters"] - 1, 2.0 ** -24)
    assert abs(info["iters"] - ref.iters) <= max(2, 0.05 * ref.iters)


@pytest.mark.parametrize("m,n,d,dt", [(1, 1, 1, np.float64), (5, 1, 3, np.float32),
                                      (50, 3, 200, np.float64), (3000, 50, 500, np.float32),
                                      (2001, 33, 257, np.float32), (4096, 1, 1, np.float64)])
def test_edge_shapes(csk, m, n, d, dt):
    """Tiny, ragged, d > m (empty rows), n = 1 and d = 1 (a single row)."""
    s = synth.gaussian_system(m, n, m + n, dt)
    x, info, _ = _solve(csk, s, d, 1, max_iter=20000)
    h, sg = oracle.count_sketch_map(1, m, d)
    At, bt = oracle.sketch(s.A.astype(np.float64), s.b.astype(np.float64), h, sg, d)
    ref = oracle.mwrk(At, bt, x_star=s.x_star, tol=1e-6, max_iter=20000)
    assert info["status"] == ref.status
    if ref.status == 0:
        assert info["rse"] <= 1e-6
    assert info["empty_rows"] == int(np.sum(np.sum(At ** 2, axis=1) == 0))


def test_max_iter_cap(csk):
    s = synth.gaussian_system(2000, 50, 4, np.float64)
    x, info, _ = _solve(csk, s, 500, 4, max_iter=10)
    assert info["status"] == 1 and info["iters"] == 10


def test_nan_input_is_numeric_failure(csk):
    s = synth.gaussian_system(2000, 50, 5, np.float32)
    s.A[17, 3] = np.nan
    x, info, _ = _solve(csk, s, 500, 5)
    assert info["status"] == -4


def test_wait_timeout_returns_status_and_context_survives(csk):
    """Failure detection without a fault: CTA 0 never publishes, every wait
    runs out of polls, the kernel returns CSK_ETIMEOUT, and the next solve
    on the same context works."""
    s = synth.gaussian_system(3000, 40, 6, np.float32)
    x, info, _ = _solve(csk, s, 400, 6, grid=4, spin_limit=20000, fault_inject=1)
    assert info["status"] == -3
    x, info, _ = _solve(csk, s, 400, 6, grid=4)
    assert info["status"] == 0 and info["rse"] <= 1e-6


def test_determinism(csk):
    s = synth.gaussian_system(100000, 500, 1, np.float32)
    x1, i1, k1 = _solve(csk, s, 5000, 1, log=5000)
    x2, i2, k2 = _solve(csk, s, 5000, 1, log=5000)
    assert i1["iters"] == i2["iters"] and np.array_equal(k1, k2)
    assert np.array_equal(x1.view(np.uint32), x2.view(np.uint32))


def test_no_xstar_residual_stop(csk):
    """Without x*, the loop stops on ||bt - At x||^2 / ||bt||^2 <= tol."""
    s = synth.gaussian_system(2000, 50, 8, np.float64)
    p = csk.csk_params_default(d=500, seed=8, tol=1e-12)
    x, info = csk.csk_solve(_to(s.A), _to(s.b), p)
    h, sg = oracle.count_sketch_map(8, 2000, 500)
    At, bt = oracle.sketch(s.A, s.b, h, sg, 500)
    ref = oracle.mwrk(At, bt, tol=1e-12)
    assert info["status"] == 0 and info["resid"] ** 2 <= 1.0001e-12
    assert abs(info["iters"] - ref.iters) <= 1


def test_gemv_variants_agree(csk):
    """Rows of At in shared memory (variant 1) and in registers (variant 2)
    both follow the oracle's i_k prefix and converge with the same IT +-2 %."""
    m, n, d, seed = 100000, 500, 5000, 3
    s = synth.gaussian_system(m, n, seed, np.float32)
    h, sg = oracle.count_sketch_map(seed, m, d)
    At32, bt32 = oracle.sketch_f32_same_order(s.A, s.b, h, sg, d)
    ref = oracle.mwrk(At32.astype(np.float64), bt32.astype(np.float64), x_star=s.x_star,
                      tol=1e-6, log_len=20000, nthreads=8)
    its = []
    for variant in (1, 2):
        x, info, ik, X = _solve(csk, s, d, seed, log=20000, xlog=20000, gemv_variant=variant)
        assert info["status"] == 0 and info["rse"] <= 1e-6
        _compare_prefix(ik, ref, 1e-3)
        _check_steps(At32, bt32, X, ik, min(info["iters"] - 1, 300), 2.0 ** -24)
        its.append(info["iters"])
    assert abs(its[0] - its[1]) <= 0.02 * ref.iters


@pytest.mark.parametrize("grid", [50, 64, 100])
def test_register_variant_small_and_timeout(csk, grid):
    """Register-resident loop on a small sketch (one row per warp), and its
    bounded wait: CTA 0 never publishes -> CSK_ETIMEOUT, context survives."""
    s = synth.gaussian_system(3000, 40, 9, np.float32)
    x, info, _ = _solve(csk, s, 400, 9, grid=grid, gemv_variant=2)
    ref = oracle.csk(s.A.astype(np.float64), s.b.astype(np.float64), 400, 9, x_star=s.x_star)
    assert info["status"] == 0 and info["rse"] <= 1e-6
    assert abs(info["iters"] - ref.iters) <= max(3, 0.05 * ref.iters)
    x, info, _ = _solve(csk, s, 400, 9, grid=grid, gemv_variant=2, spin_limit=20000,
                        fault_inject=1)
    assert info["status"] == -3


def test_bench_launch_configuration_matches_oracle(csk):
    """The configuration bench.py times (autotuned CTA count and loop variant
    on the 100000 x 500, d = 5000 workload) gives the oracle's row sequence up
    to the first near-tie and valid steps throughout."""
    from paper_2004_02480_gb300 import autotune
    m, n, d, seed = 100000, 500, 5000, 0
    s = synth.gaussian_system(m, n, seed, np.float32)
    A, b = _to(s.A), _to(s.b)
    xs = _to(s.x_star.astype(np.float32))
    p = csk.csk_params_default(d=d, seed=seed, path=csk.GEMV)
    tuned = autotune.tune_solve(A, b, p, x_star=xs, use_cache=False)
    x, info, ik, X = _solve(csk, s, d, seed, log=20000, xlog=20000, path=csk.GEMV,
                            grid=tuned["grid"], gemv_variant=tuned["gemv_variant"])
    h, sg = oracle.count_sketch_map(seed, m, d)
    At32, bt32 = oracle.sketch_f32_same_order(s.A, s.b, h, sg, d)
    ref = oracle.mwrk(At32.astype(np.float64), bt32.astype(np.float64), x_star=s.x_star,
                      tol=1e-6, log_len=20000, nthreads=8)
    assert info["status"] == 0 and info["rse"] <= 1e-6 and info["grid"] == tuned["grid"]
    _compare_prefix(ik, ref, 1e-3)
    _check_steps(At32, bt32, X, ik, info["iters"] - 1, 2.0 ** -24)
    assert abs(info["iters"] - ref.iters) <= 0.05 * ref.iters


@pytest.mark.parametrize("grid", [60, 79, 128])
def test_stream_variant_equals_register_variant(csk, grid):
    """Rows streamed through the bulk-copy ring (variant 3) use the register
    variant's arithmetic in the same order: identical iterates, bit for bit."""
    m, n, d, seed = 40000, 200, 2000, 12
    s = synth.gaussian_system(m, n, seed, np.float32)
    x2, i2, k2 = _solve(csk, s, d, seed, log=3000, grid=grid, gemv_variant=2)
    x3, i3, k3 = _solve(csk, s, d, seed, log=3000, grid=grid, gemv_variant=3)
    assert i2["status"] == 0 and i3["status"] == 0 and i3["rse"] <= 1e-6
    assert i2["iters"] == i3["iters"] and np.array_equal(k2, k3)
    assert np.array_equal(x2.view(np.uint32), x3.view(np.uint32))


@pytest.mark.parametrize("grid", [25, 28])
def test_register_loop_nine_and_ten_rows_per_warp(csk, grid):
    """At d = 2000 with rows of 300 columns (4 float4 per lane), 25 and 28
    CTAs put 10 and 9 rows on each warp of the register loop (the 16-row
    transposed butterfly, lanes paired per row).  Its iterates equal the
    streamed variant's bit for bit, and every step replays in FP64 against
    the oracle's FP32 same-order sketch."""
    m, n, d, seed = 40000, 300, 2000, 12
    s = synth.gaussian_system(m, n, seed, np.float32)
    x2, i2, k2, X = _solve(csk, s, d, seed, log=5000, xlog=5000, grid=grid, gemv_variant=2)
    x3, i3, k3 = _solve(csk, s, d, seed, log=5000, grid=grid, gemv_variant=3)
    assert i2["status"] == 0 and i2["rse"] <= 1e-6 and i2["grid"] == grid
    assert i2["iters"] == i3["iters"] and np.array_equal(k2, k3)
    assert np.array_equal(x2.view(np.uint32), x3.view(np.uint32))
    h, sg = oracle.count_sketch_map(seed, m, d)
    At32, bt32 = oracle.sketch_f32_same_order(s.A, s.b, h, sg, d)
    _check_steps(At32, bt32, X, k2, i2["iters"] - 1, 2.0 ** -24)


@pytest.mark.parametrize("pad", [0, 4])
def test_stream_variant_unsketched_mwrk(csk, pad):
    """MWRK on A itself (Remark 1, d = 0) streams A every step: the oracle's
    row sequence up to the first near-tie, valid steps, RES <= 1e-6, for a
    packed A (one bulk copy per block) and a strided one (one per row)."""
    m, n, seed = 30000, 120, 13
    s = synth.gaussian_system(m, n, seed, np.float32)
    Ad = torch.zeros((m, n + pad), dtype=torch.float32, device=DEV)
    Ad[:, :n] = _to(s.A)
    A = Ad[:, :n]
    ik = torch.full((20000,), -1, dtype=torch.int32, device=DEV)
    X = torch.zeros((20000, n), dtype=torch.float32, device=DEV)
    p = csk.csk_params_default(d=0, path=csk.GEMV, gemv_variant=3, ik_log=ik.data_ptr(),
                               ik_log_len=20000, x_log=X.data_ptr(), x_log_len=20000)
    x, info = csk.csk_solve(A, _to(s.b), p, x_star=_to(s.x_star.astype(np.float32)))
    ref = oracle.mwrk(s.A.astype(np.float64), s.b.astype(np.float64), x_star=s.x_star,
                      tol=1e-6, log_len=20000, nthreads=8)
    assert info["status"] == 0 and info["rse"] <= 1e-6
    ikh = ik.cpu().numpy()[:info["iters"]]
    _compare_prefix(ikh, ref, 1e-3)
    _check_steps(s.A, s.b, X.cpu().numpy(), ikh, min(info["iters"] - 1, 200), 2.0 ** -24)
    assert abs(info["iters"] - ref.iters) <= max(3, 0.05 * ref.iters)


def test_stream_variant_idle_ctas_and_timeout(csk):
    """More CTAs than rows (CTAs with an empty row range stream nothing), and
    the bounded waits: CTA 0 never publishes -> CSK_ETIMEOUT, context
    survives."""
    s = synth.gaussian_system(3000, 40, 14, np.float32)
    x, info, _ = _solve(csk, s, 120, 14, grid=128, gemv_variant=3)     # CTAs 120..127 idle
    ref = oracle.csk(s.A.astype(np.float64), s.b.astype(np.float64), 120, 14, x_star=s.x_star)
    assert info["status"] == ref.status
    if ref.status == 0:
        assert info["rse"] <= 1e-6 and abs(info["iters"] - ref.iters) <= max(3, 0.05 * ref.iters)
    x, info, _ = _solve(csk, s, 400, 14, grid=16, gemv_variant=3, spin_limit=20000,
                        fault_inject=1)
    assert info["status"] == -3
    x, info, _ = _solve(csk, s, 400, 14, grid=16, gemv_variant=3)
    assert info["status"] == 0 and info["rse"] <= 1e-6


@pytest.mark.parametrize("pad", [0, 2])
def test_stream_variant_fp64_unsketched_mwrk(csk, pad):
    """FP64 MWRK on A itself through the streamed loop (16-byte chunks of two
    doubles): the oracle's row sequence wherever the selection gap exceeds
    1e-9, the oracle's IT, and an x within FP64 rounding of the oracle's."""
    m, n, seed = 20000, 50, 17
    s = synth.gaussian_system(m, n, seed, np.float64)
    Ad = torch.zeros((m, n + pad), dtype=torch.float64, device=DEV)
    Ad[:, :n] = _to(s.A)
    A = Ad[:, :n]
    ik = torch.full((20000,), -1, dtype=torch.int32, device=DEV)
    p = csk.csk_params_default(d=0, path=csk.GEMV, gemv_variant=3, ik_log=ik.data_ptr(),
                               ik_log_len=20000)
    x, info = csk.csk_solve(A, _to(s.b), p, x_star=_to(s.x_star))
    ref = oracle.mwrk(s.A, s.b, x_star=s.x_star, tol=1e-6, log_len=20000, nthreads=8)
    assert info["status"] == 0 and ref.status == 0 and info["rse"] <= 1e-6
    assert info["iters"] == ref.iters
    _compare_prefix(ik.cpu().numpy()[:info["iters"]], ref, 1e-9)
    err = np.sum((x.cpu().numpy() - ref.x) ** 2) / np.sum(s.x_star ** 2)
    assert err <= 1e-20


def test_stream_variant_fp64_sketched_matches_shared_memory_variant(csk):
    """FP64 CSK at a Table 1 shape (d = n^2) with the sketch streamed every
    step (variant 3) and resident in shared memory (variant 1): both follow
    the FP64 oracle's rows up to the first near-tie, with its IT, and agree
    with each other to FP64 rounding."""
    m, n, d, seed = 60000, 150, 22500, 18
    s = synth.gaussian_system(m, n, seed, np.float64)
    h, sg = oracle.count_sketch_map(seed, m, d)
    At, bt = oracle.sketch(s.A, s.b, h, sg, d)
    ref = oracle.mwrk(At, bt, x_star=s.x_star, tol=1e-6, log_len=20000, nthreads=8)
    out = []
    for variant in (1, 3):
        x, info, ik = _solve(csk, s, d, seed, log=20000, gemv_variant=variant)
        assert info["status"] == 0 and info["rse"] <= 1e-6
        assert abs(info["iters"] - ref.iters) <= 1
        _compare_prefix(ik[:info["iters"]], ref, 1e-9)
        out.append(x)
    assert np.sum((out[0] - out[1]) ** 2) / np.sum(s.x_star ** 2) <= 1e-20


def test_fp64_check_widens_subnormals_exactly(csk):
    """The FP64 row norms and final check widen FP32 entries to binary64 with
    integer operations; the widening must be exact for subnormal floats and
    signed zeros too.  Unsketched solve (d = 0) stopped before its first step
    (max_iter = 0), so x = x0 and the check reports ||b - A x0|| / ||b||:
    column 0 of A holds signed subnormals k 2^-149, column 1 signed zeros, b
    the smallest normals, x0 = (1, 0.5, 0, 0).  Every product and difference
    is exact in binary64, so the expected value is fixed up to the order of
    the final sums; a subnormal flushed to zero or given a wrong exponent
    moves it by far more than the tolerance, and a flushed row norm would
    count the row as empty."""
    rng = np.random.default_rng(3)
    m, n = 256, 4
    a0 = rng.integers(1, 2 ** 23, size=m) * 2.0 ** -149 * rng.choice([-1.0, 1.0], size=m)
    A = np.zeros((m, n), np.float32)
    A[:, 0] = a0.astype(np.float32)
    A[:, 1] = np.where(rng.random(m) < 0.5, np.float32(-0.0), np.float32(0.0))
    assert np.array_equal(A[:, 0].astype(np.float64), a0)          # representable exactly
    b = (rng.integers(2 ** 23, 2 ** 24, size=m) * 2.0 ** -149).astype(np.float32)
    x0 = np.array([1.0, 0.5, 0.0, 0.0], np.float32)
    p = csk.csk_params_default(d=0, tol=1e-6, max_iter=0)
    x, info = csk.csk_solve(_to(A), _to(b), p, x0=_to(x0))
    assert info["iters"] == 0
    assert np.array_equal(x.cpu().numpy(), x0)
    r = b.astype(np.float64) - A.astype(np.float64) @ x0.astype(np.float64)
    want = np.sqrt(np.sum(r * r) / np.sum(b.astype(np.float64) ** 2))
    assert abs(info["resid"] - want) <= 1e-13 * want
    assert info["empty_rows"] == 0


def _ls_floor(At, bt):
    """||bt - At x_LS||^2 / ||bt||^2: no x reaches a smaller residual."""
    xls = np.linalg.lstsq(At, bt, rcond=None)[0]
    return float(np.sum((bt - At @ xls) ** 2) / np.sum(bt * bt))


def test_inconsistent_system_residual_stop_fp64(csk):
    """Inconsistent b = A x* + e (relative noise 1e-3), no x*: the loop stops
    on ||bt - At x||^2 / ||bt||^2 <= tol.  Above the least-squares floor of
    the sketched system the GPU follows the oracle's row sequence and stops at
    its IT; below the floor neither can stop (no x beats the least-squares
    residual), both run to the cap and end above the floor."""
    m, n, d, seed = 2000, 50, 500, 8
    s = synth.noisy_system(m, n, seed, 1e-3, np.float64)
    h, sg = oracle.count_sketch_map(seed, m, d)
    At, bt = oracle.sketch(s.A, s.b, h, sg, d)
    floor = _ls_floor(At, bt)
    assert 1e-7 < floor < 1e-5
    # reachable: 10 x the floor
    tol = 10 * floor
    ik = torch.full((4000,), -1, dtype=torch.int32, device=DEV)
    p = csk.csk_params_default(d=d, seed=seed, tol=tol, ik_log=ik.data_ptr(), ik_log_len=4000)
    x, info = csk.csk_solve(_to(s.A), _to(s.b), p)
    ref = oracle.mwrk(At, bt, tol=tol, log_len=4000)
    assert info["status"] == 0 and info["resid"] ** 2 <= tol * (1 + 1e-9)
    assert abs(info["iters"] - ref.iters) <= 1
    k = min(info["iters"], ref.iters)
    assert np.array_equal(ik.cpu().numpy()[:k], ref.ik[:k])
    if info["iters"] == ref.iters:
        assert np.linalg.norm(x.cpu().numpy() - ref.x) <= 1e-9 * np.linalg.norm(ref.x)
    # unreachable: a tenth of the floor, 3000-step cap
    p2 = csk.csk_params_default(d=d, seed=seed, tol=floor / 10, max_iter=3000)
    x2, info2 = csk.csk_solve(_to(s.A), _to(s.b), p2)
    ref2 = oracle.mwrk(At, bt, tol=floor / 10, max_iter=3000)
    assert info2["status"] == 1 and info2["iters"] == 3000 and ref2.iters == 3000
    for res in (info2["resid"] ** 2, float(np.sum((bt - At @ ref2.x) ** 2) / np.sum(bt * bt))):
        assert floor * (1 - 1e-9) <= res <= 10 * floor


def test_inconsistent_system_residual_stop_fp32(csk):
    """FP32, 20000 x 200, d = 2000, relative noise 1e-3, no x*, tol ten times
    the least-squares floor: the GPU (register or shared-memory loop) follows
    the oracle's rows on the bit-identical FP32 sketch up to the first
    near-tie (gap 1e-3) and stops within 2 % of its IT, above the floor."""
    m, n, d, seed = 20000, 200, 2000, 4
    s = synth.noisy_system(m, n, seed, 1e-3, np.float32)
    h, sg = oracle.count_sketch_map(seed, m, d)
    At32, bt32 = oracle.sketch_f32_same_order(s.A, s.b, h, sg, d)
    At, bt = At32.astype(np.float64), bt32.astype(np.float64)
    floor = _ls_floor(At, bt)
    tol = 10 * floor
    ik = torch.full((20000,), -1, dtype=torch.int32, device=DEV)
    p = csk.csk_params_default(d=d, seed=seed, tol=tol, ik_log=ik.data_ptr(), ik_log_len=20000)
    x, info = csk.csk_solve(_to(s.A), _to(s.b), p)
    ref = oracle.mwrk(At, bt, tol=tol, log_len=20000, nthreads=8)
    assert info["status"] == 0 and ref.status == 0
    assert floor * (1 - 1e-6) <= info["resid"] ** 2 <= tol * (1 + 1e-3)
    assert abs(info["iters"] - ref.iters) <= max(2, 0.02 * ref.iters)
    _compare_prefix(ik.cpu().numpy(), ref, 1e-3)


@pytest.mark.parametrize("dt,refresh", [(np.float32, 0), (np.float32, 40), (np.float64, 0)])
def test_residual_update_form_unsketched_mwrk(csk, dt, refresh):
    """Remark 1's residual-update form of MWRK on A itself (d = 0): the loop
    keeps r and subtracts alpha A A_{i_k}^T each step (a GEMV of A against
    the chosen row), recomputing bt - A x every `refresh` steps.  RES <= 1e-6
    at the oracle's IT (+-2 %), and every step replayed from the GPU's own
    iterate within the update form's bound (rounding of the dot products
    against the chosen row accumulated since the last recomputation), with
    the oracle's selection from the same iterate."""
    m, n, seed = 30000, 120, 21
    s = synth.gaussian_system(m, n, seed, dt)
    u = 2.0 ** -24 if dt == np.float32 else 2.0 ** -53
    A = _to(s.A)
    ik = torch.full((20000,), -1, dtype=torch.int32, device=DEV)
    X = torch.zeros((20000, n), dtype=A.dtype, device=DEV)
    p = csk.csk_params_default(d=0, path=csk.UPDATE, refresh_every=refresh, ik_log=ik.data_ptr(),
                               ik_log_len=20000, x_log=X.data_ptr(), x_log_len=20000)
    x, info = csk.csk_solve(A, _to(s.b), p, x_star=_to(s.x_star.astype(dt)))
    ref = oracle.mwrk(s.A.astype(np.float64), s.b.astype(np.float64), x_star=s.x_star,
                      tol=1e-6, log_len=20000, nthreads=8)
    assert info["status"] == 0 and info["rse"] <= 1e-6 and info["path"] == csk.UPDATE
    assert abs(info["iters"] - ref.iters) <= max(2, 0.02 * ref.iters)
    steps = info["iters"]
    ikh = ik.cpu().numpy()
    Xh = np.concatenate([X.cpu().numpy()[:steps], x.cpu().numpy()[None]])
    name = f"{'FP32' if dt == np.float32 else 'FP64'} residual-update MWRK {m}x{n} refresh {refresh}"
    rep = stepcheck.replay(s.A, s.b, Xh, ikh, steps, path="update", refresh=refresh, u=u,
                           name=name, oracle=oracle)
    rep.prefix, _ = stepcheck.trajectory_prefix(ikh, ref, 1e-3 if dt == np.float32 else 1e-9)
    stepcheck.record(rep)
    assert rep.steps == steps and rep.oracle_equal >= 0.9 * steps


def test_residual_update_form_sketched_fp32(csk):
    """The residual-update form on a sketch (100000 x 500 FP32, d = 5000):
    the same replay, and the same IT as the GEMV form within 2 %."""
    m, n, d, seed = 100000, 500, 5000, 0
    s = synth.gaussian_system(m, n, seed, np.float32)
    x, info, ik, X = _solve(csk, s, d, seed, log=20000, xlog=20000, path=csk.UPDATE,
                            refresh_every=100)
    assert info["status"] == 0 and info["rse"] <= 1e-6
    _, info_g, _ = _solve(csk, s, d, seed, path=csk.GEMV)
    assert abs(info["iters"] - info_g["iters"]) <= 0.02 * info_g["iters"]
    h, sg = oracle.count_sketch_map(seed, m, d)
    At32, bt32 = oracle.sketch_f32_same_order(s.A, s.b, h, sg, d)
    steps = info["iters"]
    Xh = np.concatenate([X[:steps], x[None]])
    rep = stepcheck.replay(At32, bt32, Xh, ik, steps, path="update", refresh=100,
                           name="FP32 residual-update CSK 100000x500 d=5000 refresh 100",
                           oracle=oracle)
    stepcheck.record(rep)
    assert rep.steps == steps and rep.oracle_equal >= 0.9 * steps


def test_fused_launch_fp32_bench_workload(csk):
    """fused = 1: the sketch (16-bit buckets, each CTA ordering and summing
    the rows it then owns) and the loop in one cooperative kernel, on the
    100000 x 500 FP32, d = 5000 workload.  Every step replayed from the GPU's
    own iterate against the oracle's FP32 same-order sketch (so a sketch
    that differed from it would show as steps outside the bound), the
    oracle's selection from the same iterate, IT within 2 % of the FP64
    oracle's and of the separate-launch solve."""
    m, n, d, seed = 100000, 500, 5000, 0
    s = synth.gaussian_system(m, n, seed, np.float32)
    x, info, ik, X = _solve(csk, s, d, seed, log=20000, xlog=20000, path=csk.GEMV, fused=1)
    assert info["status"] == 0 and info["rse"] <= 1e-6
    _, info_sep, _ = _solve(csk, s, d, seed, path=csk.GEMV, grid=info["grid"])
    h, sg = oracle.count_sketch_map(seed, m, d)
    At32, bt32 = oracle.sketch_f32_same_order(s.A, s.b, h, sg, d)
    ref = oracle.mwrk(At32.astype(np.float64), bt32.astype(np.float64), x_star=s.x_star,
                      tol=1e-6, log_len=20000, nthreads=8)
    assert abs(info["iters"] - ref.iters) <= 0.02 * ref.iters
    assert abs(info["iters"] - info_sep["iters"]) <= 0.02 * info_sep["iters"]
    steps = info["iters"]
    Xh = np.concatenate([X[:steps], x[None]])
    assert _check_steps(At32, bt32, Xh, ik, steps, 2.0 ** -24,
                        name="FP32 fused launch 100000x500 d=5000") == steps
    xs32 = s.x_star.astype(np.float32).astype(np.float64)      # the x* the GPU was given
    rse, res = oracle.final_check(At32.astype(np.float64), bt32.astype(np.float64), x, xs32)
    assert abs(info["rse"] - rse) <= 1e-9 * rse and abs(info["resid"] - res) <= 1e-6 * res


@pytest.mark.parametrize("m,n,d,seed", [(2000, 50, 500, 0), (300000, 50, 2500, 1),
                                        (300000, 100, 10000, 2)])
def test_fused_launch_fp64_matches_oracle(csk, m, n, d, seed):
    """fused = 1 in FP64 (the 2000 x 50 workload and Table 1 shapes, d = n^2,
    shared-memory loop): the sketch is the oracle's bit for bit (same
    ascending-order additions), so the row sequence must equal the oracle's
    wherever the selection gap exceeds 1e-9, with the oracle's IT and an x
    within FP64 rounding of the oracle's."""
    s = synth.gaussian_system(m, n, seed, np.float64)
    x, info, ik = _solve(csk, s, d, seed, log=20000, fused=1)
    h, sg = oracle.count_sketch_map(seed, m, d)
    At, bt = oracle.sketch(s.A, s.b, h, sg, d)
    ref = oracle.mwrk(At, bt, x_star=s.x_star, tol=1e-6, log_len=20000, nthreads=8)
    assert info["status"] == 0 and ref.status == 0 and info["rse"] <= 1e-6
    K = _compare_prefix(ik, ref, 1e-9, name=f"FP64 fused launch {m}x{n} d={d}")
    if K == ref.iters:
        assert info["iters"] == ref.iters
    assert np.sum((x - ref.x) ** 2) / np.sum(s.x_star ** 2) <= 1e-12
    rse, res = oracle.final_check(At, bt, x, s.x_star)
    assert abs(info["rse"] - rse) <= 1e-12 * rse + 1e-18


def test_fused_launch_residual_stop_and_timeout(csk):
    """fused = 1 without x* (the stopping norm ||bt||^2 assembled from the
    CTAs' FP64 partials inside the kernel), and the bounded waits of the
    fused kernel: CTA 0 never publishes -> CSK_ETIMEOUT, the context
    survives and the next fused solve converges."""
    s = synth.gaussian_system(2000, 50, 8, np.float64)
    p = csk.csk_params_default(d=500, seed=8, tol=1e-12, fused=1)
    x, info = csk.csk_solve(_to(s.A), _to(s.b), p)
    h, sg = oracle.count_sketch_map(8, 2000, 500)
    At, bt = oracle.sketch(s.A, s.b, h, sg, 500)
    ref = oracle.mwrk(At, bt, tol=1e-12)
    assert info["status"] == 0 and info["resid"] ** 2 <= 1.0001e-12
    assert abs(info["iters"] - ref.iters) <= 1
    s2 = synth.gaussian_system(3000, 40, 6, np.float32)
    x, info, _ = _solve(csk, s2, 400, 6, grid=4, spin_limit=20000, fault_inject=1, fused=1)
    assert info["status"] == -3
    x, info, _ = _solve(csk, s2, 400, 6, grid=4, fused=1)
    assert info["status"] == 0 and info["rse"] <= 1e-6
