"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: published
generator outputs, a library routine (numpy matmul / stable argsort / SVD,
torch's bfloat16 cast), an identity from the convergence proof, a closed-form
special case, or the iteration counts printed in Table 1.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2004_02480_gb300 import synth


def dense_S(h, sign, d):
    """Definition 1 written as a dense d x m matrix Phi D."""
    m = h.shape[0]
    S = np.zeros((d, m))
    S[h, np.arange(m)] = sign
    return S


# ------------------------------------------------------------ Definition 1

def test_splitmix64_published_outputs(golden):
    for seed, idx, val in golden("splitmix64.txt"):
        assert oracle.splitmix64_at(int(seed), int(idx)) == int(val)


@pytest.mark.parametrize("m,d", [(1, 1), (7, 3), (50, 7), (200, 500), (1000, 1)])
def test_sketch_matrix_structure(m, d):
    """Every column of S has exactly one non-zero entry, equal to +-1,
    so diag(S^T S) = 1 exactly (Definition 1)."""
    h, s = oracle.count_sketch_map(12345 + m, m, d)
    assert h.min() >= 0 and h.max() < d
    assert set(np.unique(s)).issubset({-1, 1})
    S = dense_S(h, s, d)
    assert np.all((S != 0).sum(axis=0) == 1)
    assert np.all(np.abs(S).sum(axis=0) == 1)
    assert np.array_equal(np.diag(S.T @ S), np.ones(m))


def test_sketch_isotropy_over_seeds():
    """E[S^T S] = I: off-diagonal entries D_i D_k [h(i)=h(k)] average to 0."""
    m, d, T = 6, 3, 20000
    acc = np.zeros((m, m))
    for t in range(T):
        h, s = oracle.count_sketch_map(t, m, d)
        S = dense_S(h, s, d)
        acc += S.T @ S
    mean = acc / T
    assert np.allclose(np.diag(mean), 1.0)
    off = mean[~np.eye(m, dtype=bool)]
    sd = np.sqrt(1.0 / d / T)                     # Var of one entry is 1/d
    assert np.max(np.abs(off)) < 5 * sd


def test_sketch_preserves_norm_in_expectation():
    """E ||S y||^2 = ||y||^2 (Definition 1 with independent h and D)."""
    rng = np.random.default_rng(1)
    m, d, T = 40, 8, 6000
    y = rng.standard_normal(m)
    vals = []
    for t in range(T):
        h, s = oracle.count_sketch_map(1000 + t, m, d)
        vals.append(np.sum((dense_S(h, s, d) @ y) ** 2))
    vals = np.array(vals)
    assert abs(vals.mean() - y @ y) < 5 * vals.std() / np.sqrt(T)


def test_bucket_uniformity_and_sign_balance():
    """h(i) is uniform on [d] and the signs are fair (chi-square / binomial)."""
    m, d = 1_000_000, 997
    h, s = oracle.count_sketch_map(2024, m, d)
    cnt = np.bincount(h, minlength=d)
    chi2 = np.sum((cnt - m / d) ** 2 / (m / d))
    assert stats.chi2.sf(chi2, d - 1) > 1e-4
    plus = int(np.sum(s > 0))
    assert stats.binomtest(plus, m, 0.5).pvalue > 1e-4


# ------------------------------------------------------ sort and sketch

@pytest.mark.parametrize("m,d", [(1, 1), (7, 3), (2000, 500), (3000, 3000), (100, 1000), (10000, 1)])
def test_stable_count_sort_matches_library_sort(m, d):
    h, _ = oracle.count_sketch_map(99, m, d)
    cnt, off, perm = oracle.stable_count_sort(h, d)
    assert np.array_equal(cnt, np.bincount(h, minlength=d))
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(cnt)]))
    assert np.array_equal(perm, np.argsort(h, kind="stable"))


@pytest.mark.parametrize("m,n,d,R", [(1, 1, 1, 1), (7, 3, 3, 1), (200, 13, 40, 3),
                                     (50, 9, 80, 2), (500, 21, 1, 1)])
def test_sketch_equals_dense_product(m, n, d, R):
    """Algorithm 1 Initialize: At = S A and bt = S b for the dense S."""
    rng = np.random.default_rng(m * 31 + n)
    A = rng.standard_normal((m, n))
    B = rng.standard_normal((m, R))
    h, s = oracle.count_sketch_map(7, m, d)
    At, bt = oracle.sketch(A, B, h, s, d)
    S = dense_S(h, s, d)
    np.testing.assert_allclose(At, S @ A, rtol=0, atol=1e-12 * max(1, np.abs(A).sum()))
    np.testing.assert_allclose(bt, S @ B, rtol=0, atol=1e-12 * max(1, np.abs(B).sum()))


def test_identity_map_sketch_is_identity():
    """d = m, h = identity, signs +1: S = I, so the sketch returns A itself."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((30, 4))
    b = rng.standard_normal(30)
    At, bt = oracle.sketch(A, b, np.arange(30), np.ones(30, np.int8), 30)
    assert np.array_equal(At, A) and np.array_equal(bt, b)


def test_f32_twin_exact_on_integers_and_ordered():
    """The FP32 twin is exact when every partial sum is representable, and it
    adds in ascending row order (an order-sensitive case proves which)."""
    rng = np.random.default_rng(4)
    m, n, d = 3000, 17, 100
    A = rng.integers(-1000, 1000, (m, n)).astype(np.float32)
    b = rng.integers(-1000, 1000, m).astype(np.float32)
    h, s = oracle.count_sketch_map(5, m, d)
    At, bt = oracle.sketch_f32_same_order(A, b, h, s, d)
    S = dense_S(h, s, d)
    assert np.array_equal(At, (S @ A.astype(np.float64)).astype(np.float32))
    assert np.array_equal(bt, (S @ b.astype(np.float64)).astype(np.float32))
    # rows 0,1,2 in one bucket with sign +1: ((0 + 1e8) + 1) - 1e8 = 0 in FP32
    A3 = np.array([[1e8], [1.0], [-1e8]], np.float32)
    At3, _ = oracle.sketch_f32_same_order(A3, None, np.zeros(3, np.int32), np.ones(3, np.int8), 1)
    assert At3[0, 0] == 0.0
    At3r, _ = oracle.sketch_f32_same_order(A3[[0, 2, 1]], None, np.zeros(3, np.int32),
                                           np.ones(3, np.int8), 1)
    assert At3r[0, 0] == 1.0


def test_f32_twin_within_recursive_summation_bound():
    rng = np.random.default_rng(6)
    m, n, d = 20000, 33, 300
    A = rng.standard_normal((m, n)).astype(np.float32)
    h, s = oracle.count_sketch_map(8, m, d)
    At32, _ = oracle.sketch_f32_same_order(A, None, h, s, d)
    At64, _ = oracle.sketch(A, None, h, s, d)
    cnt = np.bincount(h, minlength=d)
    absum, _ = oracle.sketch(np.abs(A), None, h, np.ones(m, np.int8), d)
    bound = (cnt[:, None] * 2.0 ** -24) * absum
    assert np.all(np.abs(At32 - At64) <= bound + 1e-30)


def test_sketched_system_is_consistent():
    """S(A x*) = (S A) x*, so the sketch of a consistent system is consistent."""
    sysm = synth.gaussian_system(2000, 50, 0)
    h, s = oracle.count_sketch_map(0, 2000, 500)
    At, bt = oracle.sketch(sysm.A, sysm.b, h, s, 500)
    assert np.linalg.norm(bt - At @ sysm.x_star) / np.linalg.norm(bt) < 1e-14


def test_row_norms_match_library():
    rng = np.random.default_rng(9)
    At = rng.standard_normal((40, 17))
    np.testing.assert_allclose(oracle.row_norms2(At), np.einsum("ij,ij->i", At, At), rtol=1e-14)
    At32 = At.astype(np.float32)
    np.testing.assert_allclose(oracle.row_norms2(At32),
                               np.einsum("ij,ij->i", At32.astype(np.float64), At32.astype(np.float64)),
                               rtol=1e-14)


# ------------------------------------------------------------- iteration

def _replay_x(At, x0, res):
    """Iterates x_k rebuilt from the logged rows and step lengths."""
    xs = [x0.copy()]
    for k in range(len(res.ik)):
        xs.append(xs[-1] + (res.r_ik[k] / res.n_ik[k]) * At[res.ik[k]])
    return xs


def test_selection_is_brute_force_argmax_with_ties_and_zero_rows():
    """i_k is the first maximiser of |r_j|/||At_j|| over non-zero rows."""
    # designed first step: row 0 is zero (its large residual must be ignored),
    # rows 1..3 tie exactly, so the smallest index 1 must win
    At = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [2.0, 0.0], [0.5, 0.5]])
    bt = np.array([5.0, 1.0, 1.0, 2.0, 0.25])
    res = oracle.mwrk(At, bt, tol=0.0, max_iter=1, log_len=4)
    assert res.ik[0] == 1
    rng = np.random.default_rng(11)
    for trial in range(30):
        d, n = int(rng.integers(1, 9)), int(rng.integers(1, 5))
        At = rng.integers(-2, 3, (d, n)).astype(float)       # small ints: frequent ties
        At[rng.random(d) < 0.2] = 0.0                         # and zero rows
        if not np.any(np.abs(At).sum(axis=1) > 0):
            continue
        bt = rng.integers(-3, 4, d).astype(float)
        x0 = rng.integers(-1, 2, n).astype(float)
        res = oracle.mwrk(At, bt, x0=x0, tol=0.0, max_iter=6, log_len=8)
        xs = _replay_x(At, x0, res)
        for k, ik in enumerate(res.ik):
            r = bt - At @ xs[k]
            nrm = np.sqrt(np.sum(At ** 2, axis=1))
            key = np.where(nrm > 0, np.abs(r) / np.where(nrm > 0, nrm, 1), -np.inf)
            assert ik == int(np.flatnonzero(key == key.max())[0])


def test_all_zero_rows_is_numeric_failure():
    res = oracle.mwrk(np.zeros((4, 3)), np.ones(4), tol=1e-6)
    assert res.status == oracle.STATUS_ENUMERIC


def test_per_step_error_identity_eqA():
    """Proof of Theorem 2, eq. (eq:A): ||e_{k+1}||^2 = ||e_k||^2 - r_{i_k}^2 / ||At_{i_k}||^2."""
    sysm = synth.gaussian_system(2000, 50, 1)
    h, s = oracle.count_sketch_map(1, 2000, 500)
    At, bt = oracle.sketch(sysm.A, sysm.b, h, s, 500)
    res = oracle.mwrk(At, bt, x_star=sysm.x_star, tol=1e-12, max_iter=200, log_len=201)
    e2 = res.err2
    pred = e2[:-1] - res.r_ik[:len(e2) - 1] ** 2 / res.n_ik[:len(e2) - 1]
    assert np.max(np.abs(e2[1:] - pred)) <= 1e-10 * e2[0]


def test_deterministic_sketched_rate_eq6():
    """Eqs. (eq:5)-(eq:6): ||e_{k+1}||^2 <= (1 - sigma_min^2(At)/||At||_F^2) ||e_k||^2."""
    sysm = synth.gaussian_system(3000, 40, 2)
    h, s = oracle.count_sketch_map(2, 3000, 400)
    At, bt = oracle.sketch(sysm.A, sysm.b, h, s, 400)
    sv = np.linalg.svd(At, compute_uv=False)
    q = 1.0 - sv[-1] ** 2 / np.sum(At ** 2)
    res = oracle.mwrk(At, bt, x_star=sysm.x_star, tol=1e-10, max_iter=500, log_len=501)
    e2 = res.err2
    assert np.all(e2[1:] <= q * e2[:-1] * (1 + 1e-9))


def test_theorem2_rate_with_empirical_epsilon():
    """Theorem 2 with eps measured from Lemma 1's two inequalities on this draw:
    per-step contraction is at most 1 - (1-eps)^3 sigma_r^2(A) / (n ||A||_2^2)."""
    m, n, d = 4000, 20, 400
    sysm = synth.gaussian_system(m, n, 3)
    h, s = oracle.count_sketch_map(3, m, d)
    At, bt = oracle.sketch(sysm.A, sysm.b, h, s, d)
    sA = np.linalg.svd(sysm.A, compute_uv=False)
    sSA = np.linalg.svd(At, compute_uv=False)
    # Lemma 1 (lem11): (1-eps)||Ax||^2 <= ||SAx||^2 for all x  <=> via the
    # generalised eigenvalues of (At^T At, A^T A); (lem12): (1-eps) s_i(SA) <= s_i(A)
    lam = np.linalg.eigvals(np.linalg.solve(sysm.A.T @ sysm.A, At.T @ At)).real
    eps1 = max(1 - lam.min(), lam.max() - 1)
    eps2 = np.max(1 - sA / sSA)
    eps = max(eps1, eps2, 0.0)
    assert eps < 1
    q = 1 - (1 - eps) ** 3 / n * sA[-1] ** 2 / sA[0] ** 2
    res = oracle.mwrk(At, bt, x_star=sysm.x_star, tol=1e-10, max_iter=300, log_len=301)
    e2 = res.err2
    assert np.all(e2[1:] <= q * e2[:-1] * (1 + 1e-9))


def test_orthogonal_rows_converge_in_n_steps():
    """Square At with orthogonal rows: each projection fixes one coordinate
    of the error for good, so x* is reached after exactly n steps, each row
    chosen once."""
    n = 12
    Q = synth.haar_orthogonal(n, np.random.default_rng(5))
    At = Q * np.linspace(1, 3, n)[:, None]
    xs = np.random.default_rng(6).standard_normal(n)
    res = oracle.mwrk(At, At @ xs, x_star=xs, tol=1e-24, max_iter=3 * n, log_len=3 * n)
    assert res.iters == n and res.status == oracle.STATUS_OK
    assert sorted(res.ik.tolist()) == list(range(n))
    assert np.linalg.norm(res.x - xs) < 1e-12 * np.linalg.norm(xs)


def test_single_unknown_converges_in_one_step():
    rng = np.random.default_rng(7)
    At = rng.standard_normal((9, 1))
    res = oracle.mwrk(At, At[:, 0] * 2.5, x_star=np.array([2.5]), tol=1e-24, max_iter=5)
    assert res.iters == 1 and abs(res.x[0] - 2.5) < 1e-14


def test_stopping_rule_and_cap():
    """RES is tested before each step; the cap returns status 1 after max_iter updates."""
    sysm = synth.gaussian_system(2000, 50, 4)
    h, s = oracle.count_sketch_map(4, 2000, 500)
    At, bt = oracle.sketch(sysm.A, sysm.b, h, s, 500)
    full = oracle.mwrk(At, bt, x_star=sysm.x_star, tol=1e-6, log_len=1000)
    assert full.status == oracle.STATUS_OK
    e2 = full.err2 / np.sum(sysm.x_star ** 2)
    assert e2[full.iters] <= 1e-6 < e2[full.iters - 1]
    cap = oracle.mwrk(At, bt, x_star=sysm.x_star, tol=1e-6, max_iter=10)
    assert cap.status == oracle.STATUS_MAXITER and cap.iters == 10
    assert oracle.mwrk(At, bt, x0=sysm.x_star, x_star=sysm.x_star).iters == 0


def test_thread_count_does_not_change_result():
    sysm = synth.gaussian_system(3000, 30, 5)
    a = oracle.csk(sysm.A, sysm.b, 300, 5, x_star=sysm.x_star, nthreads=1)
    b = oracle.csk(sysm.A, sysm.b, 300, 5, x_star=sysm.x_star, nthreads=4)
    assert a.iters == b.iters and np.array_equal(a.x, b.x)


def test_mwrk_mode_is_csk_with_identity_sketch():
    """Remark 1: MWRK is Algorithm 1 with S = I."""
    sysm = synth.gaussian_system(600, 20, 6)
    a = oracle.csk(sysm.A, sysm.b, 0, 0, x_star=sysm.x_star)
    b = oracle.mwrk(sysm.A, sysm.b, x_star=sysm.x_star)
    assert a.iters == b.iters and np.array_equal(a.x, b.x)


def test_final_check_matches_library_norms():
    rng = np.random.default_rng(8)
    At, bt, x, xs = (rng.standard_normal((30, 5)), rng.standard_normal(30),
                     rng.standard_normal(5), rng.standard_normal(5))
    rse, res = oracle.final_check(At, bt, x, xs)
    assert abs(rse - np.sum((x - xs) ** 2) / np.sum(xs ** 2)) < 1e-14
    assert abs(res - np.linalg.norm(bt - At @ x) / np.linalg.norm(bt)) < 1e-14


@pytest.mark.parametrize("seed", range(5))
def test_config1_converges(seed):
    """2000 x 50, d = 500, FP64: RES <= 1e-6 well inside the 20000-step cap."""
    sysm = synth.gaussian_system(2000, 50, seed)
    res = oracle.csk(sysm.A, sysm.b, 500, seed, x_star=sysm.x_star)
    assert res.status == oracle.STATUS_OK and res.iters < 1000
    rse, _ = oracle.final_check(sysm.A, sysm.b, res.x, sysm.x_star)
    assert rse <= 1e-6


@pytest.mark.slow
@pytest.mark.parametrize("n,seeds", [(50, 8), (100, 4), (150, 2)])
def test_table1_iteration_counts(golden, n, seeds):
    """Mean IT of CSK (d = n^2) and MWRK at m = 300000 lands within 15 % of
    Table 1; the random stream differs from MATLAB's, the distribution not."""
    rows = {(int(r[0]), int(r[1])): (float(r[2]), float(r[3])) for r in golden("table1_iterations.txt")}
    csk_paper, mwrk_paper = rows[(300000, n)]
    its, mits = [], []
    for sd in range(seeds):
        sysm = synth.gaussian_system(300000, n, 100 + sd)
        its.append(oracle.csk(sysm.A, sysm.b, n * n, sd, x_star=sysm.x_star, nthreads=8).iters)
        if sd == 0:
            mits.append(oracle.csk(sysm.A, sysm.b, 0, 0, x_star=sysm.x_star, nthreads=8).iters)
    assert abs(np.mean(its) - csk_paper) <= 0.15 * csk_paper
    assert abs(np.mean(mits) - mwrk_paper) <= 0.15 * mwrk_paper


# ------------------------------------------------------------------ Gram

def test_bf16_round_matches_torch_cast():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(10)
    v = np.concatenate([rng.standard_normal(2000).astype(np.float32) * 10.0 ** rng.integers(-5, 5, 2000),
                        np.float32([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -0.0, 0.0, 65504.0])])
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    ours = np.array([oracle.bf16_round(float(t)) for t in v], np.float32)
    assert np.array_equal(ours.view(np.uint32), ref.view(np.uint32))


def test_gram_matches_library_and_split_error_bound():
    rng = np.random.default_rng(12)
    At = rng.standard_normal((37, 29)).astype(np.float32)
    G = oracle.gram(At.astype(np.float64))
    A64 = At.astype(np.float64)
    np.testing.assert_allclose(G, A64 @ A64.T, rtol=0, atol=1e-12 * 29)
    Gs = oracle.gram_split_bf16(At)
    # dropping lo*lo and rounding lo cost at most ~2^-16 relative per product
    absG = np.abs(A64) @ np.abs(A64).T
    assert np.all(np.abs(Gs - G) <= 2.0 ** -15 * absG)
    assert np.max(np.abs(Gs - G) / absG) > 0           # the split is not exact


def test_inconsistent_system_never_beats_least_squares():
    """Inconsistent b = A x* + e: no iterate reaches a residual below the
    least-squares residual of the sketched system (numpy lstsq), so the
    residual stopping rule is met above that floor and never below it.  The
    oracle's steps remain orthogonal projections onto the chosen rows'
    hyperplanes: for z on row i_k's hyperplane (here the projection of the
    least-squares solution onto it), ||x_{k+1} - z||^2 = ||x_k - z||^2 - r^2/N."""
    m, n, d, seed = 2000, 40, 400, 3
    s = synth.noisy_system(m, n, seed, 1e-3, np.float64)
    h, sg = oracle.count_sketch_map(seed, m, d)
    At, bt = oracle.sketch(s.A, s.b, h, sg, d)
    xls = np.linalg.lstsq(At, bt, rcond=None)[0]
    floor = np.sum((bt - At @ xls) ** 2) / np.sum(bt * bt)
    assert floor > 1e-9                                   # really inconsistent
    hi = oracle.mwrk(At, bt, tol=10 * floor, max_iter=5000)
    assert hi.status == 0
    res_hi = np.sum((bt - At @ hi.x) ** 2) / np.sum(bt * bt)
    assert floor <= res_hi <= 10 * floor * (1 + 1e-12)
    lo = oracle.mwrk(At, bt, tol=floor / 10, max_iter=1500, log_len=1501)
    assert lo.status == 1 and lo.iters == 1500
    res_lo = np.sum((bt - At @ lo.x) ** 2) / np.sum(bt * bt)
    assert res_lo >= floor * (1 - 1e-12)
    # projection identity on step k: z = the projection of x_LS onto row i_k's hyperplane
    N = np.sum(At * At, axis=1)
    x = np.zeros(n)
    for k in range(50):
        i = lo.ik[k]
        r = bt[i] - At[i] @ x
        x1 = x + r / N[i] * At[i]
        z = xls + (bt[i] - At[i] @ xls) / N[i] * At[i]
        lhs = np.sum((x1 - z) ** 2)
        rhs = np.sum((x - z) ** 2) - r * r / N[i]
        assert abs(lhs - rhs) <= 1e-9 * np.sum((x - z) ** 2)
        x = x1
    # and the oracle's own iterate after those 50 steps is this replay
    r50 = oracle.mwrk(At, bt, tol=0.0, max_iter=50)
    assert np.allclose(r50.x, x, rtol=1e-12, atol=1e-12 * np.linalg.norm(x))


@pytest.mark.parametrize("d,n", [(1, 1), (9, 7), (70, 65), (130, 64), (257, 130)])
def test_gram_rows_equal_whole_split_product(d, n):
    """or_gram_split_bf16_rows (the comparator of the full-size Gram check):
    each requested row, in the requested order and with repeats, equals the
    same row of or_gram_split_bf16 bit for bit, and both equal the split
    definition hi hi^T + hi lo^T + lo hi^T formed independently here with
    torch's BF16 cast and a numpy product (BF16 products are exact in
    binary64, so only the summation order differs)."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(d * 131 + n)
    At = (rng.standard_normal((d, n)) * 10.0 ** rng.integers(-3, 3, (d, 1))).astype(np.float32)
    rows = np.concatenate([[d - 1, 0], rng.integers(0, d, 6), [d - 1]]).astype(np.int64)
    Gr = oracle.gram_split_bf16_rows(At, rows)
    Gs = oracle.gram_split_bf16(At)
    assert Gr.shape == (len(rows), d)
    assert np.array_equal(Gr.view(np.uint64), Gs[rows].view(np.uint64))
    t = torch.from_numpy(At)
    hi_t = t.to(torch.bfloat16).to(torch.float32)
    lo_t = (t - hi_t).to(torch.bfloat16).to(torch.float32)
    hi, lo = hi_t.double().numpy(), lo_t.double().numpy()
    split = hi[rows] @ hi.T + hi[rows] @ lo.T + lo[rows] @ hi.T
    mag = np.abs(hi[rows]) @ np.abs(hi).T + np.abs(hi[rows]) @ np.abs(lo).T + np.abs(lo[rows]) @ np.abs(hi).T
    assert np.all(np.abs(Gr - split) <= 4 * n * 2.0 ** -53 * mag)
    # a transposed operand or a dropped segment would be far outside that
    wrong = hi[rows] @ hi.T + lo[rows] @ hi.T
    if n > 1:
        assert np.any(np.abs(Gr - wrong) > 4 * n * 2.0 ** -53 * mag)
