"""csk_sketch_noalloc -- the sketch entry point that allocates nothing.

It exists for callers that cannot allocate device memory (code handed only
input and output pointers by an application that owns all device memory, or
code that must not call cudaMalloc because it may synchronise the device);
its scratch is a static device array inside the library.  This test calls
it through the C ABI twice in a row and checks every output against the
regular csk_sketch entry point: the integer outputs and the FP32 sketch must
be bit-identical (the same fixed-order kernels run), the FP64 norms equal.
It lives in its own file, collected last, and works both alone in a fresh
process and after the other tests.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def csk():
    from paper_2004_02480_gb300 import build, csk as _csk
    build.build()
    return _csk


def test_noalloc_sketch_matches_workspace_sketch_twice(csk):
    dev = "cuda:0"
    g = torch.Generator(device=dev).manual_seed(123)
    cases = [(200_000, 300, 3000, 2, torch.float32, 7),   # several scan tiles, b with 2 RHS
             (50_000, 33, 700, 1, torch.float64, 8),      # ragged n, FP64
             (1 << 20, 4, 1 << 18, 1, torch.float32, 9)]  # the largest m and d the scratch holds
    for m, n, d, R, dt, seed in cases:
        A = torch.randn((m, n), generator=g, device=dev, dtype=dt)
        b = torch.randn((m, R), generator=g, device=dev, dtype=dt)
        ref = csk.csk_sketch(A, d, seed, b, norms=True, perm=True, off=True)
        for _ in range(2):                      # two calls in a row share the static scratch
            out = csk.csk_sketch_noalloc(A, d, seed, b, norms=True, perm=True, off=True)
            torch.cuda.synchronize()
            assert torch.equal(out.off, ref.off)
            assert torch.equal(out.perm, ref.perm)
            assert torch.equal(out.At, ref.At)
            assert torch.equal(out.bt, ref.bt)
            assert torch.equal(out.norms2, ref.norms2)


def test_noalloc_default_outputs_only(csk):
    """The common call: no b, no perm and no off requested, so the sorted
    rows and the bucket offsets stay in the static array too (at the full
    2^20-row, 2^18-bucket size as well).  At and the FP64 norms must equal
    csk_sketch's bit for bit, on two calls in a row."""
    dev = "cuda:0"
    g = torch.Generator(device=dev).manual_seed(321)
    for m, n, d, dt, seed in [(1 << 20, 4, 1 << 18, torch.float32, 3),
                              (70_001, 129, 5_003, torch.float32, 4),
                              (30_000, 50, 2_500, torch.float64, 5)]:
        A = torch.randn((m, n), generator=g, device=dev, dtype=dt)
        ref = csk.csk_sketch(A, d, seed, None, norms=True)
        for _ in range(2):
            out = csk.csk_sketch_noalloc(A, d, seed, None, norms=True)
            torch.cuda.synchronize()
            assert out.bt is None and out.perm is None and out.off is None
            assert torch.equal(out.At, ref.At)
            assert torch.equal(out.norms2, ref.norms2)


def test_noalloc_rejects_sizes_beyond_static_scratch(csk):
    fake = ctypes.c_void_p(256)
    L = csk.lib()
    assert L.csk_sketch_noalloc(fake, (1 << 20) + 1, 4, 4, None, 0, 0, 0, 10, 0, fake, None,
                                None, None, None, None) == csk.CSK_ENOMEM
    assert L.csk_sketch_noalloc(fake, 1000, 4, 4, None, 0, 0, 0, (1 << 18) + 1, 0, fake, None,
                                None, None, None, None) == csk.CSK_ENOMEM
