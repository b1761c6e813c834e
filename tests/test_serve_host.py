"""Host logic of the continuous-batching server on CPU: the engine's runs and
batches are replaced by fakes that count steps, so admission (first come,
first served under the HBM budget), re-batching, retirement, rejection and
the statistics are checked without a GPU.  Footprints come from the real
pa_workspace_size (host code of the C ABI)."""
from __future__ import annotations

import pytest

from paper_2006_00561_gb300 import build as B


@pytest.fixture(scope="module")
def S():
    B.build()
    from paper_2006_00561_gb300 import pa, serve
    return pa, serve


class FakeRun:
    live = 0

    def __init__(self, cfg, stream=None):
        self.K, self.R0, self.step = cfg.K, cfg.R0, 0
        FakeRun.live += 1

    def history(self, first, n):
        return [{"step": i, "R": self.R0} for i in range(first, first + n)]

    def observables(self):
        return {"step": self.step, "R": self.R0}

    def spins(self):
        return None

    def close(self):
        FakeRun.live -= 1


class FakeBatch:
    made = []

    def __init__(self, runs, stream=None):
        self.runs = list(runs)
        FakeBatch.made.append(len(self.runs))

    def run_steps(self, n):
        for r in self.runs:
            assert r.step + n <= r.K, "a run was stepped past K"
            r.step += n

    def sync(self):
        return 0

    def close(self):
        pass


@pytest.fixture
def server(S, monkeypatch):
    P, serve = S
    monkeypatch.setattr(serve.P, "Run", FakeRun)
    monkeypatch.setattr(serve.P, "Batch", FakeBatch)
    FakeRun.live = 0
    FakeBatch.made = []
    return P, serve


def spec(L=16, R0=1000, K=10, **kw):
    return dict(dim=2, L=L, R0=R0, K=K, theta=2, seed=1, **kw)


def test_budget_admission_and_retirement(server):
    P, serve = server
    one = P.pa_workspace_size(P.make_config(layout=P.LAYOUT_PACKED, **spec()))
    srv = serve.Server(hbm_budget=2 * one + one // 2, quantum=4, stream=object())
    reqs = [srv.submit(i, spec(K=10 + i), 0.0) for i in range(4)]
    srv.t0 = 0.0
    srv._now = lambda: 0.0
    n = srv.step()
    # two fit the budget; first come, first served
    assert [r.rid for r in srv.resident] == [0, 1] and [r.rid for r in srv.queue] == [2, 3]
    assert n == 4 and srv.used == 2 * one and FakeBatch.made == [2]
    while not srv.idle():
        srv.step()
        assert srv.used <= srv.budget
    assert sorted(r.rid for r in srv.done) == [0, 1, 2, 3]
    assert all(r.result["step"] == r.spec["K"] for r in srv.done)
    assert srv.used == 0 and FakeRun.live == 0 and srv.max_resident == 2
    # membership changes re-form the batch; a full run of K steps ends exactly at K
    assert len(FakeBatch.made) >= 3


def test_oversized_and_invalid_requests_are_rejected(server):
    P, serve = server
    one = P.pa_workspace_size(P.make_config(layout=P.LAYOUT_PACKED, **spec()))
    srv = serve.Server(hbm_budget=one, stream=object())
    big = srv.submit(0, spec(R0=1 << 20), 0.0)
    bad = srv.submit(1, spec(L=7), 0.0)
    ok = srv.submit(2, spec(), 0.0)
    assert big.error.startswith("rejected") and bad.error == "invalid config"
    assert [r.rid for r in srv.queue] == [2] and ok.error is None
    st = srv.stats()
    assert st["rejected"] == 2 and st["waiting"] == 1


def test_trace_statistics(server):
    P, serve = server
    srv = serve.Server(hbm_budget=1 << 34, quantum=8, stream=object())
    trace = [dict(spec(K=5 + 3 * i), arrival=0.0) for i in range(5)]
    st = srv.run_trace(trace)
    assert st["served"] == 5 and st["rejected"] == 0 and st["waiting"] == 0
    assert st["max_resident"] == 5 and st["p99_latency_s"] >= st["p50_latency_s"] >= 0
    want = sum(1000 * 256 * 2 * (5 + 3 * i) for i in range(5))
    assert sum(r.attempts() for r in srv.done) == want
