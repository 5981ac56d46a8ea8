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


def test_candidates_small_problem_keeps_four_rows_per_cta():
    c = candidates(152, rows=200)
    small = [g for g in c if g <= 64]
    assert small and all(4 * g <= 200 for g in small)
    assert 48 in c and 64 not in c


def test_candidates_without_rows_are_fractions_only():
    assert candidates(152) == [152, 137, 128, 114, 100, 91, 76]
