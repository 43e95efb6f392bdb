"""The serving dispatcher (surrogate with MPM fallback) on a short query
stream: every query is answered once, out-of-range queries and failed
checks go to the MPM, sampled checks are measured against the MPM."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def test_stream_is_served_with_fallback_and_checks():
    import paper_2301_08343_gb300 as T
    from paper_2301_08343_gb300 import serving as SV
    from paper_2301_08343_gb300 import surrogate as SG
    specs = W.c3_specs(64, seed_base=500)
    X, Y, _ = SG.generate(specs, W.C3_BLOCK, W.C3_SUBSTEPS, W.C3_DT, size=64, chunk=64)
    net = T.SurrogateNet((32, 64, 128, 256), 2, 3, size=64, max_batch=128, seed=0)
    SG.train(net, X, Y, steps=100, batch=32, lr=2e-3)
    q = W.c4_queries(rate_hz=4096.0, duration_s=0.04, seed=9, out_of_range=0.3)
    assert 100 < len(q) < 250
    srv = SV.PressServer(net, W.C3_BLOCK, W.C3_SUBSTEPS, W.C3_DT, size=64, max_batch=128, check_every=8,
                         mpm_batch=32, pool_sizes=(32, 64))
    r = srv.serve(q)
    n_out = sum(1 for x in q if not SV.in_training_range(x))
    assert n_out > 10
    assert r["queries"] == len(q)
    assert r["mpm_answers"] == n_out + r["checks_over_residual"]
    assert r["surrogate_answers"] + r["mpm_answers"] == len(q)
    assert r["sampled_checks"] == sum(1 for x in q if SV.in_training_range(x) and x["id"] % 8 == 0)
    assert r["sampled_residual_um_mean"] is not None and np.isfinite(r["sampled_residual_um_mean"])
    assert 0 < r["latency_p50_ms"] <= r["latency_p99_ms"]
    plain = SV.PressServer(net, W.C3_BLOCK, W.C3_SUBSTEPS, W.C3_DT, size=64, use_surrogate=False,
                           mpm_batch=64, pool_sizes=(32, 64)).serve(q)
    assert plain["mpm_answers"] == len(q) and plain["surrogate_answers"] == 0


def test_reset_restores_the_initial_lattice():
    import paper_2301_08343_gb300 as T
    bt = T.TacchiBatch([W.Block(6, 6, 2, 0.5e-3, seed=3), W.Block(4, 5, 2, 0.5e-3, seed=4)])
    u0 = [bt.get_state(i)["u"].clone() for i in range(2)]
    bt.set_indenter(0, T.IndenterKind.SPHERE, (1.5e-3,), (1.5e-3, 1.5e-3, 2.2e-3, 1, 0, 0, 0), (0, 0, -0.3, 0, 0, 0))
    bt.step(50, 1e-5)
    assert not torch.equal(bt.get_state(0)["u"], u0[0])
    bt.reset()
    for i in range(2):
        s = bt.get_state(i)
        assert s["status"] == 0 and torch.equal(s["u"], u0[i])
        assert float(s["Fm"].abs().max()) == 0.0 and float(s["v"].abs().max()) == 0.0
