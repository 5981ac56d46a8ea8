"""GPU parity of the sketch (Algorithm 1, Initialize) against the CPU oracle.

Integer outputs (bucket offsets, row permutation) must match bit for bit.
The FP32 sketch must equal the oracle's FP32 same-order twin bit for bit and
the FP64 sketch the oracle's FP64 sketch bit for bit (both add the same exact
signed terms in ascending row order); the FP64 row norms agree to 1e-13
relative (accumulation order differs).
"""
import numpy as np
import pytest

import oracle
from paper_2004_02480_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def csk():
    from paper_2004_02480_gb300 import build, csk as _csk
    build.build()
    return _csk


DEV = "cuda:0"


def _gpu_sketch(csk, A, b, d, seed):
    At = torch.from_numpy(np.ascontiguousarray(A)).to(DEV)
    bt = None if b is None else torch.from_numpy(np.ascontiguousarray(b)).to(DEV)
    s = csk.csk_sketch(At, d, seed, bt, norms=True, perm=True, off=True)
    torch.cuda.synchronize()
    return s


@pytest.mark.parametrize("m,d", [(1, 1), (7, 3), (2000, 500), (2000, 2000), (2000, 5000),
                                 (100000, 1), (1_000_000, 500), (1_000_000, 20000), (33, 1000),
                                 # one-block scan up to 32768 buckets, tiled scan above
                                 (100000, 32768), (100000, 32769), (300000, 100000)])
def test_sort_bit_exact(csk, m, d):
    seed = 17 + m + d
    A = np.zeros((m, 4), np.float32)
    s = _gpu_sketch(csk, A, None, d, seed)
    h, _ = oracle.count_sketch_map(seed, m, d)
    cnt, off, perm = oracle.stable_count_sort(h, d)
    assert np.array_equal(s.off.cpu().numpy(), off)
    assert np.array_equal(s.perm.cpu().numpy(), perm)


@pytest.mark.parametrize("d", [3000, 40000])
def test_sort_offsets_into_unaligned_buffer(csk, d):
    """off_out and perm_out may be any int32-aligned caller buffers (here 4
    bytes past a 16-byte boundary): the scans and the scatter must not assume
    vector alignment there."""
    m, n, seed = 50000, 4, 5
    A = torch.zeros((m, n), dtype=torch.float32, device=DEV)
    At = torch.empty((d, n), dtype=torch.float32, device=DEV)
    obuf = torch.zeros(d + 2, dtype=torch.int32, device=DEV)
    pbuf = torch.zeros(m + 1, dtype=torch.int32, device=DEV)
    off_view, perm_view = obuf[1:], pbuf[1:]
    assert off_view.data_ptr() % 16 == 4 and perm_view.data_ptr() % 16 == 4
    ws = csk._workspace(csk.csk_sketch_workspace_size(m, d), A.device)
    rc = csk.lib().csk_sketch(csk._ptr(A), m, n, n, None, 0, 0, csk.CSK_F32, d, seed, csk._ptr(At),
                              None, None, csk._ptr(perm_view), csk._ptr(off_view), csk._ptr(ws),
                              ws.numel(), csk._stream(A.device))
    assert rc == 0
    torch.cuda.synchronize()
    h, _ = oracle.count_sketch_map(seed, m, d)
    _, off, perm = oracle.stable_count_sort(h, d)
    assert np.array_equal(off_view.cpu().numpy(), off)
    assert np.array_equal(perm_view.cpu().numpy(), perm)


@pytest.mark.parametrize("m,n,d,R", [(1, 1, 1, 1), (7, 3, 3, 1), (2000, 50, 500, 1),
                                     (5000, 64, 300, 3), (3000, 257, 1000, 1), (1000, 33, 2000, 2),
                                     (20000, 1000, 700, 0), (40000, 12, 10, 64)])
def test_sketch_fp32_bit_exact(csk, m, n, d, R):
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((m, n)).astype(np.float32)
    b = rng.standard_normal((m, R)).astype(np.float32) if R else None
    seed = 5 * m + d
    s = _gpu_sketch(csk, A, b, d, seed)
    h, sg = oracle.count_sketch_map(seed, m, d)
    At, bt = oracle.sketch_f32_same_order(A, b, h, sg, d)
    assert np.array_equal(s.At.cpu().numpy().view(np.uint32), At.view(np.uint32))
    if R:
        assert np.array_equal(s.bt.cpu().numpy().view(np.uint32), bt.view(np.uint32))
    np.testing.assert_allclose(s.norms2.cpu().numpy(), oracle.row_norms2(At), rtol=1e-13, atol=0)
    # and within the recursive-summation bound of the FP64 sketch
    At64, _ = oracle.sketch(A, None, h, sg, d)
    cnt = np.bincount(h, minlength=d)[:, None]
    absum, _ = oracle.sketch(np.abs(A), None, h, np.ones(m, np.int8), d)
    assert np.all(np.abs(s.At.cpu().numpy() - At64) <= cnt * 2.0 ** -24 * absum + 1e-30)


@pytest.mark.parametrize("m,n,d", [(2000, 50, 500), (999, 7, 100), (4000, 130, 4000),
                                   # FP64 chunk shapes: 64, 128, 192, 256 columns, several warps, scalar
                                   (3000, 64, 700), (3000, 128, 700), (3000, 200, 900), (3000, 256, 900),
                                   (3000, 300, 900), (3000, 65, 800)])
def test_sketch_fp64_bit_exact(csk, m, n, d):
    s_ = synth.gaussian_system(m, n, m, np.float64)
    s = _gpu_sketch(csk, s_.A, s_.b, d, 3)
    h, sg = oracle.count_sketch_map(3, m, d)
    At, bt = oracle.sketch(s_.A, s_.b, h, sg, d)
    assert np.array_equal(s.At.cpu().numpy(), At)
    assert np.array_equal(s.bt.cpu().numpy(), bt)


@pytest.mark.parametrize("m,n,d,R", [(3000, 40, 300, 1), (3000, 40, 300, 3), (5000, 130, 60, 1),
                                     (999, 7, 2000, 1)])
def test_sketch_fp64_rhs_bit_exact(csk, m, n, d, R):
    """FP64 right-hand sides: one column (8 buckets per warp, lane g summing
    bucket g's rows in order) and several (a warp per bucket), including
    buckets of hundreds of rows (d = 60) and many empty ones (d > m)."""
    rng = np.random.default_rng(7 * m + R)
    A = rng.standard_normal((m, n))
    b = rng.standard_normal((m, R)) if R > 1 else rng.standard_normal(m)
    s = _gpu_sketch(csk, A, b, d, 11)
    h, sg = oracle.count_sketch_map(11, m, d)
    At, bt = oracle.sketch(A, b, h, sg, d)
    assert np.array_equal(s.At.cpu().numpy(), At)
    assert np.array_equal(s.bt.cpu().numpy().reshape(bt.shape), bt)


def test_sketch_strided_lda(csk):
    rng = np.random.default_rng(0)
    full = rng.standard_normal((3000, 80)).astype(np.float32)
    At_gpu = csk.csk_sketch(torch.from_numpy(full).to(DEV)[:, :50], 300, 9, norms=False)
    h, sg = oracle.count_sketch_map(9, 3000, 300)
    At, _ = oracle.sketch_f32_same_order(full[:, :50], None, h, sg, 300)
    assert np.array_equal(At_gpu.At.cpu().numpy(), At)


def test_sketch_full_size_precision_form_sampled(csk):
    """1e6 x 1000 FP32 (the precision-form workload): integer parts exact,
    sampled rows of At bit-exact against the twin computed row by row."""
    m, n, d, seed = 1_000_000, 1000, 20000, 11
    g = torch.Generator(device=DEV).manual_seed(5)
    A = torch.randn((m, n), generator=g, device=DEV, dtype=torch.float32)
    s = csk.csk_sketch(A, d, seed, norms=True, perm=True, off=True)
    torch.cuda.synchronize()
    h, sg = oracle.count_sketch_map(seed, m, d)
    cnt, off, perm = oracle.stable_count_sort(h, d)
    assert np.array_equal(s.off.cpu().numpy(), off)
    assert np.array_equal(s.perm.cpu().numpy(), perm)
    rows = np.random.default_rng(1).choice(d, 64, replace=False)
    Atg = s.At.cpu().numpy()
    for j in rows:
        members = perm[off[j]:off[j + 1]]
        Aj = A[torch.from_numpy(members.astype(np.int64)).to(DEV)].cpu().numpy()
        Atj, _ = oracle.sketch_f32_same_order(Aj, None, np.zeros(len(members), np.int32),
                                              sg[members], 1)
        assert np.array_equal(Atg[j], Atj[0])


@pytest.mark.parametrize("env", [{"CSK_SKETCH_PATH": "sort"}, {"CSK_SKETCH_PATH": "cta"},
                                 {"CSK_SKETCH_PATH": "warp"}, {"CSK_SKETCH_PATH": "own"},
                                 {"CSK_SKETCH_PATH": "own", "CSK_SKETCH_OWN_CAP": "256"},
                                 {"CSK_SKETCH_PATH": "own", "CSK_SKETCH_OWN_CAP": "16"}])
def test_sketch_paths_bit_exact(csk, env):
    """The counting-sort path (with the segmented sum the library picks, and
    forced to the CTA-per-bucket kernel for every shape, or to the
    warp-per-bucket kernel wherever buckets hold at most 128 rows on
    average: buckets of 0 to ~130 rows, so the warp kernel's register
    ordering of up to 32 and of 33..64 rows and its global ordering of
    larger buckets all run) and the bucket-owner FP32 path (forced for every
    shape), the latter also with a per-CTA row list of 256 and of 16 rows --
    so its sub-range rescans and its large-bucket ordering by ballot
    compaction run -- give the oracle's offsets, permutation, At and Bt bit
    for bit (child process: the path is read from the environment once)."""
    import os
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    r = subprocess.run([sys.executable, os.path.join(here, "sketch_paths_check.py")],
                       env={**os.environ, **env}, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
