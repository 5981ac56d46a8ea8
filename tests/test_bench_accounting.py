"""Host-side checks of the benchmark's roofline accounting (no GPU): the
algorithmic byte counts of the sketch and of one GEMV residual evaluation,
and the lookup of the committed DRAM-traffic capture of the register loop
(used only while the loop's sources are unchanged)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_sketch_bytes_at_the_two_sketch_sizes():
    # A read once, b read once, perm written and read, At and bt written, cnt/off
    assert bench.sketch_bytes(100_000, 500, 5_000) == 4 * 100_000 * 500 + 4 * 100_000 + 8 * 100_000 \
        + 4 * 5_000 * 500 + 4 * 5_000 + 8 * 5_000
    assert abs(bench.sketch_bytes(100_000, 500, 5_000) / 1e9 - 0.211) < 0.001
    assert abs(bench.sketch_bytes(1_000_000, 1000, 20_000) / 1e9 - 4.09) < 0.01


def test_gemv_bytes_per_residual_evaluation():
    # At (d x n) plus bt, x and the chosen row: 10 MB at d = 5000, n = 500
    assert bench.gemv_bytes_per_eval(5_000, 500) == 4 * 5_000 * 500 + 4 * (5_000 + 1_000)
    assert abs(bench.gemv_bytes_per_eval(100_000, 500) / 1e6 - 200.4) < 0.1   # MWRK on A


def test_traffic_lookup_follows_the_source_hash():
    tag = "k_iterate_gemv_reg_100000x500_d5000"
    h = bench._source_hash(*(f"paper_2004_02480_gb300/csrc/{f}" for f in bench.LOOP_SOURCES))
    t = bench._traffic(tag, h)
    assert t is None or 1e6 < t < 1e8             # a capture of one solve: ~10 MB
    assert bench._traffic(tag, "0" * 16) is None  # a stale capture is not reported
