"""Host-side check of the loop autotuner's candidate CTA counts (no GPU):
fractions of the SM count, plus small counts for problems that a few dozen
CTAs can hold, never more CTAs than leave 4 rows each."""
import pytest

pytest.importorskip("torch")
from paper_2004_02480_gb300.autotune import candidates  # noqa: E402


def test_candidates_large_problem_adds_small_counts():
    c = candidates(152, rows=5000)
    assert c == sorted(c, reverse=True) and len(set(c)) == len(c)
    assert {152, 137, 128, 114, 100, 91, 76} <= set(c)
    assert {8, 16, 32, 64} <= set(c)
    assert max(c) <= 152
    # the fewest CTAs holding 5000 rows at 10, 9, 8, 7, 6, 5 rows per warp (8 warps)
    assert {63, 70, 79, 90, 105, 125} <= set(c)


def test_candidates_small_problem_keeps_four_rows_per_cta():
    c = candidates(152, rows=200)
    small = [g for g in c if g <= 64]
    assert small and all(4 * g <= 200 for g in small)
    assert 48 in c and 64 not in c


def test_candidates_without_rows_are_fractions_only():
    assert candidates(152) == [152, 137, 128, 114, 100, 91, 76]


def test_batched_candidates_respect_residency():
    """Batched loop shapes: every thread count, 1..k CTAs per SM with k the
    most that shared memory (r, weights: d each; x, x*: n each) and 128
    registers a thread let stay resident."""
    from paper_2004_02480_gb300.autotune import batched_candidates, batched_smem_bytes
    c = batched_candidates(152, 10000, 1000)
    assert batched_smem_bytes(10000, 1000) == (20000 + 2000) * 4
    assert set(c) == {(128, 152), (128, 304), (256, 152), (256, 304), (384, 152), (512, 152)}
    small = batched_candidates(152, 500, 50)
    assert (128, 4 * 152) in small and (512, 152) in small and (512, 304) not in small
    assert all(t in (128, 256, 384, 512) and g % 152 == 0 for t, g in small)


def test_batched_signature_is_a_shape_histogram():
    """Plans are keyed by the histogram of right-hand sides over (log2 d,
    log2 n) bins: independent of the systems' order and of sizes inside a
    bin, sensitive to a system moving bins or gaining right-hand sides."""
    from paper_2004_02480_gb300 import csk
    a = [(5000, 50, 500, 64), (20000, 120, 1200, 64), (8000, 77, 770, 3)]
    s = csk.csk_solve_batched_signature(a)
    assert s == csk.csk_solve_batched_signature(a[::-1])
    assert s == csk.csk_solve_batched_signature([(5100, 51, 510, 64)] + a[1:])
    assert s != csk.csk_solve_batched_signature([(5000, 50, 1100, 64)] + a[1:])
    assert s != csk.csk_solve_batched_signature(a[:2] + [(8000, 77, 770, 4)])
