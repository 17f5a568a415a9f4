"""Host-side logic of the served path (no GPU): the trace replay's submission timing and latency
bookkeeping, driven by a synthetic clock and a fake server."""
import numpy as np

from paper_2501_00923_gb300 import serve
from paper_2501_00923_gb300 import workloads as W


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-4)


def test_replay_latency_accounting_with_a_synthetic_clock():
    clk = FakeClock()
    arrivals = np.array([0.0, 0.1, 0.25, 0.26])
    need = {0: 3, 1: 1, 2: 2, 3: 1}           # ticks each request needs
    left = {}
    tick_dt = 0.05

    def submit(k):
        left[k] = need[k]
        return k

    def tick():
        clk.t += tick_dt
        for k in list(left):
            left[k] -= 1

    def done(k):
        return left[k] <= 0

    lat, span = serve.replay(arrivals, submit, tick, done, clock=clk, sleep=clk.sleep)
    # request 0 arrives at 0 and needs 3 ticks of 50 ms; 1 arrives at 0.1 and rides the batch
    assert abs(lat[0] - 0.15) < 1e-9
    assert 0.0 < lat[1] <= 0.1 + 1e-9
    assert np.all(lat > 0)
    assert span >= 0.26
    stats = serve.latency_stats(lat, span)
    assert stats["solves"] == 4 and stats["p99_ms"] >= stats["p50_ms"] > 0


def test_trace_is_seeded_and_spans_the_workload_ranges():
    a = W.request_trace(128, np.random.default_rng(W.SEED_BASE + 3))
    b = W.request_trace(128, np.random.default_rng(W.SEED_BASE + 3))
    assert [r["Kn"] for r in a] == [r["Kn"] for r in b]
    gaps = np.diff([r["t"] for r in a])
    assert abs(gaps.mean() - 0.05) < 0.015                       # Poisson arrivals, mean 20/s
    assert {(r["ni"], r["nj"]) for r in a} == {(64, 32), (128, 64), (192, 96)}
    assert {r["nv"] for r in a} == {24, 32, 48}
    kn = np.log10([r["Kn"] for r in a])
    assert kn.min() < -2.5 and kn.max() > 0.5
    specs = serve.trace_specs(a[:3])
    assert specs[0].mesh.nodes.shape == (a[0]["nj"] + 1, a[0]["ni"], 2)


def test_request_marshalling_carries_the_prediction_options():
    """SolveSpec -> dvm_request: the prediction fields land in the C struct (the layout itself is
    checked against the library in test_abi.py), and a trace asks every request for them."""
    a = W.request_trace(4, np.random.default_rng(W.SEED_BASE + 3))
    specs = serve.trace_specs(a, predict=20)
    assert all(s.predict == 20 for s in specs)
    req = specs[0].to_c()
    assert req.predict_iters == 20 and req.predict_omega == 0.0
    assert req.ni == a[0]["ni"] and req.nv == a[0]["nv"] ** 2
    plain = serve.trace_specs(a[:1])[0].to_c()
    assert plain.predict_iters == 0
