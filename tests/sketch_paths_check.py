"""Run by tests/test_gpu_sketch.py in a child process whose environment
forces a sketch path (CSK_SKETCH_PATH = sort | cta | warp | own) and, for the
bucket-owner path, a small per-CTA row list (CSK_SKETCH_OWN_CAP), which
drives its sub-range and large-bucket code.  Every case must match the
oracle: offsets and permutation bit for bit, At and Bt bit for bit against
the FP32 same-order twin, the FP64 norms to 1e-13.  Exits non-zero on the
first mismatch."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2004_02480_gb300 import csk  # noqa: E402

CASES = [(100000, 500, 5000, 1), (20000, 130, 700, 3), (5000, 64, 300, 64), (3000, 50, 20, 1),
         (7, 3, 3, 1), (1, 1, 1, 1), (2000, 33, 5000, 1), (30000, 1000, 1500, 2), (4000, 8, 40, 0),
         (60000, 12, 600, 1), (8000, 126, 900, 1), (40000, 254, 3000, 2), (6000, 514, 200, 1),
         (5000, 301, 250, 1), (20000, 260, 400, 1)]


def main():
    dev = "cuda:0"
    for m, n, d, R in CASES:
        rng = np.random.default_rng(m + 3 * n + d)
        A = rng.standard_normal((m, n)).astype(np.float32)
        b = rng.standard_normal((m, R)).astype(np.float32) if R else None
        seed = 7 * m + d
        s = csk.csk_sketch(torch.from_numpy(A).to(dev), d, seed,
                           None if b is None else torch.from_numpy(b).to(dev),
                           norms=True, perm=True, off=True)
        torch.cuda.synchronize()
        h, sg = oracle.count_sketch_map(seed, m, d)
        _, off, perm = oracle.stable_count_sort(h, d)
        At, bt = oracle.sketch_f32_same_order(A, b, h, sg, d)
        tag = (m, n, d, R, os.environ.get("CSK_SKETCH_PATH"), os.environ.get("CSK_SKETCH_OWN_CAP"))
        assert np.array_equal(s.off.cpu().numpy(), off), tag
        assert np.array_equal(s.perm.cpu().numpy(), perm), tag
        assert np.array_equal(s.At.cpu().numpy().view(np.uint32), At.view(np.uint32)), tag
        if R:
            assert np.array_equal(s.bt.cpu().numpy().reshape(bt.shape).view(np.uint32),
                                  bt.view(np.uint32)), tag
        np.testing.assert_allclose(s.norms2.cpu().numpy(), oracle.row_norms2(At), rtol=1e-13,
                                   atol=0, err_msg=str(tag))
    print("sketch paths ok", os.environ.get("CSK_SKETCH_PATH"), os.environ.get("CSK_SKETCH_OWN_CAP"))


if __name__ == "__main__":
    main()
