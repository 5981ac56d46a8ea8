"""GPU run of the continuous-batching loop: requests arriving while others
are on the GPU are admitted as memory frees up (a deliberately small HBM
budget forces waiting) and join the running units at the next step chunk,
every solve reaches RES <= 1e-6, and a request's result is bit-identical
alone (in chunks of another size) and in the mix."""
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
    srv = serve.Server(budget_bytes=budget, keep_x=True, max_group=8, chunk=32)
    stats = srv.run(reqs)
    assert stats["all_converged"] and stats["rse_max"] <= 1e-6
    assert stats["peak_bytes"] <= budget
    assert stats["groups"] > 3                     # admitted in several groups
    assert stats["ticks"] > stats["groups"]        # units ran over several step chunks
    assert all(r.t_admit >= r.arrival for r in reqs)
    for r in reqs[::max(1, len(reqs) // 4)][:4]:
        alone = serve.Request(r.rid, 0.0, r.m, r.n, r.d, r.nrhs, r.seed)
        srv2 = serve.Server(budget_bytes=budget, keep_x=True, chunk=1000)
        srv2.run([alone])
        assert np.array_equal(alone.x, r.x) and alone.iters == r.iters


def test_synthetic_systems_are_pure_and_gaussian():
    """The serving harness's data generator: a system's entries depend only on
    its seed (alone and in a group: identical bits), are standard normal, and
    B = A X to FP32 accumulation error."""
    from paper_2004_02480_gb300 import build, csk
    build.build()
    dev = "cuda:0"
    shapes = [(3000, 40, 3, 11), (50000, 200, 16, 12), (777, 33, 1, 13)]
    def alloc(m, n, R):
        return (torch.empty((m, n), device=dev), torch.empty((n, R), device=dev),
                torch.empty((m, R), device=dev))
    group = [alloc(m, n, R) + (seed,) for m, n, R, seed in shapes]
    csk.csk_synth_systems(group)
    for (m, n, R, seed), g in zip(shapes, group):
        alone = alloc(m, n, R) + (seed,)
        csk.csk_synth_systems([alone])
        for a, b in zip(g[:3], alone[:3]):
            assert torch.equal(a, b)
    A, X, B, _ = group[1]
    a = A.double()
    assert abs(a.mean().item()) < 0.01 and abs(a.std().item() - 1.0) < 0.01
    assert abs(a.pow(3).mean().item()) < 0.02 and abs(a.pow(4).mean().item() - 3.0) < 0.05
    ref = a @ X.double()
    err = (B.double() - ref).abs().max().item()
    bound = 2.0 ** -22 * A.shape[1] * (a.abs() @ X.double().abs()).max().item()
    assert err <= bound
    # different seeds give different data
    assert not torch.equal(group[0][0][:20, :20], group[2][0][:20, :20])
