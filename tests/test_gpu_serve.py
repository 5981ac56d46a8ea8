"""GPU run of the continuous-batching loop: requests arriving while others
are on the GPU are admitted as memory frees up (a deliberately small HBM
budget forces waiting), every solve reaches RES <= 1e-6, and a request's
result is bit-identical alone and in the mix."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def serve():
    from paper_2004_02480_gb300 import build
    build.build()
    from paper_2004_02480_gb300 import serve as _serve
    return _serve


def test_serving_mix_converges_and_matches_alone(serve):
    reqs = serve.poisson_requests(400.0, 0.5, seed=3, m_range=(2000, 20000), n_range=(20, 100),
                                  rhs_range=(1, 4))
    budget = 6 * max(serve.request_bytes(r) for r in reqs)
    srv = serve.Server(budget_bytes=budget, keep_x=True, streams=3, max_group=8)
    stats = srv.run(reqs)
    assert stats["all_converged"] and stats["rse_max"] <= 1e-6
    assert stats["peak_bytes"] <= budget
    assert stats["groups"] > 3                     # admitted in several overlapping groups
    assert all(r.t_admit >= r.arrival for r in reqs)
    for r in reqs[::max(1, len(reqs) // 4)][:4]:
        alone = serve.Request(r.rid, 0.0, r.m, r.n, r.d, r.nrhs, r.seed)
        srv2 = serve.Server(budget_bytes=budget, keep_x=True, streams=1)
        srv2.run([alone])
        assert np.array_equal(alone.x, r.x) and alone.iters == r.iters
