"""Table 1 shape on the GPU: CSK (d = n^2) and MWRK (d = 0) in FP64 reach
RES <= 1e-6 with mean iteration counts near the paper's Table 1 means (the
paper's 50 MATLAB trials; a different random stream, so a band)."""
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_table1_smallest_shape_iterations():
    from paper_2004_02480_gb300 import build, csk, table1
    build.build()
    r = table1.run_shape(csk, torch, 300000, 50, 6, torch.device("cuda", 0))
    p = table1.PAPER[(300000, 50)]
    assert r["all_converged"]
    assert abs(r["csk_it"] - p[0]) <= 0.15 * p[0]
    assert abs(r["mwrk_it"] - p[1]) <= 0.2 * p[1]
    assert r["speedup"] > 1.0
