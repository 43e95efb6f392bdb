"""Host logic of the serving dispatcher, with the device lanes replaced by
fakes of fixed cost (virtual clock): every query is answered exactly once,
the network lane keeps answering while an MPM press is running (the press
advances in slices), the MPM lane starts a press on a full batch, on its
oldest query's wait limit or at the end of the stream, and failed checks are
served by the MPM."""
import pytest

import workloads as W

torch = pytest.importorskip("torch")
SV = pytest.importorskip("paper_2301_08343_gb300.serving")

COST = dict(sur=2e-3, sur_per=1e-6, start=1e-3, slice=20e-3, finish=2e-3)  # seconds


class FakeServer(SV.PressServer):
    def __init__(self, bad_ids=(), **kw):
        self.torch = torch
        opts = dict(substeps=500, dt=1e-5, size=4, max_batch=64, check_every=8, residual_um=5.0,
                    use_surrogate=True, mpm_batch=32, mpm_wait_s=0.25, pool_sizes=(32, 64))
        opts.update(kw)
        self._policy(**opts)
        self.bad = set(bad_ids)
        self.calls = []

    def _run(self, fn):
        self._cost = 0.0
        return fn(), self._cost

    def _surrogate(self, qs):
        self._cost = COST["sur"] + COST["sur_per"] * len(qs)
        self.calls.append(("sur", len(qs)))
        return torch.tensor([float(q["id"]) for q in qs]).reshape(-1, 1, 1, 1).expand(-1, 4, 4, 3).clone()

    def _start_press(self, qs):
        self._cost = COST["start"]
        assert len(qs) <= self.pool_sizes[-1]
        self.calls.append(("press", len(qs)))
        return {"handle": None, "left": self.substeps}

    def _advance(self, job, n):
        assert 0 < n <= job["left"]
        self._cost = COST["slice"] * n / 50
        self.calls.append(("slice", n))

    def _finish(self, job):
        self._cost = COST["finish"]
        return [None] * len(job["items"])

    def _residual_um(self, pred, ref):
        return 9.0 if int(pred[0, 0, 0]) in self.bad else 1.0


def queries(duration=0.4, oor=0.3, seed=3):
    return W.c4_queries(rate_hz=2000.0, duration_s=duration, seed=seed, out_of_range=oor)


def test_every_query_answered_once_and_counted():
    q = queries()
    in_range = [x for x in q if SV.in_training_range(x)]
    checked = [x["id"] for x in in_range if x["id"] % 8 == 0]
    bad = checked[::3]
    srv = FakeServer(bad_ids=bad)
    r = srv.serve(q)
    n_out = len(q) - len(in_range)
    assert r["queries"] == len(q)
    assert r["sampled_checks"] == len(checked)
    assert r["checks_over_residual"] == len(bad)
    assert r["mpm_answers"] == n_out + len(bad)
    assert r["surrogate_answers"] == len(in_range) - len(bad)
    assert sum(r["mpm_presses"]) == n_out + len(checked)
    assert sum(n for kind, n in srv.calls if kind == "sur") == len(in_range)
    assert r["sampled_residual_um_mean"] == pytest.approx((9.0 * len(bad) + 1.0 * (len(checked) - len(bad)))
                                                          / len(checked))
    assert 0 <= r["latency_p50_ms"] <= r["latency_p99_ms"]


def test_network_lane_is_not_held_up_by_a_press():
    q = queries(duration=0.6)
    sliced = FakeServer().serve(q, chunk_substeps=50)
    whole = FakeServer().serve(q, chunk_substeps=500)
    press_s = COST["slice"] * 10
    # a surrogate answer waits at most one slice and one network launch behind
    # the press; unsliced, it can wait for the whole press
    bound_ms = (COST["slice"] + COST["start"] + COST["finish"] + 2 * (COST["sur"] + 64 * COST["sur_per"])) * 1e3
    assert sliced["latency_surrogate_p99_ms"] <= bound_ms
    assert whole["latency_surrogate_p99_ms"] > 0.5 * press_s * 1e3
    assert sliced["mpm_answers"] == whole["mpm_answers"]


def test_mpm_lane_triggers():
    # a lone out-of-range query waits the wait limit (the stream goes on),
    # then gets a press of one; at the end of the stream it does not wait
    q = queries(duration=0.4, oor=0.0)
    lone = dict(q[0], kind="heightmap", id=10 ** 6, arrival=0.0)
    later = dict(q[0], id=1, arrival=1.0)
    assert SV.in_training_range(later)
    press = COST["start"] + 10 * COST["slice"] + COST["finish"]
    srv = FakeServer(check_every=10 ** 9, mpm_wait_s=0.1)
    r = srv.serve([lone, later])
    assert r["mpm_presses"] == [1]
    assert r["latency_mpm_p99_ms"] == pytest.approx((0.1 + press) * 1e3)
    r = FakeServer(check_every=10 ** 9, mpm_wait_s=0.1).serve([lone])
    assert r["latency_mpm_p99_ms"] == pytest.approx(press * 1e3)
    # a burst larger than the batch limit starts presses of at most the
    # largest pool size, without waiting
    burst = [dict(lone, id=i, arrival=0.0) for i in range(100)]
    srv = FakeServer(check_every=10 ** 9, mpm_batch=32, mpm_wait_s=10.0)
    r = srv.serve(burst)
    assert r["mpm_presses"] == [64, 36]
    assert r["latency_mpm_p99_ms"] < 10.0 * 1e3
    # plain MPM serving: nothing goes to the network
    srv = FakeServer(use_surrogate=False)
    r = srv.serve(queries(duration=0.2))
    assert r["surrogate_answers"] == 0 and not any(k == "sur" for k, _ in srv.calls)


def test_empty_stream():
    r = FakeServer().serve([])
    assert r["queries"] == 0 and r["mpm_presses"] == [] and r["latency_p50_ms"] is None
