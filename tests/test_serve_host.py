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


# ---------------------------------------------------------------------------
# pipelined server: quanta in flight, events polled, arena-backed workspaces
# ---------------------------------------------------------------------------
class FakeEvent:
    def __init__(self, polls_until_done=0):
        self.left = polls_until_done
        self.recorded = False

    def query(self):
        if self.left > 0:
            self.left -= 1
            return False
        return True

    def synchronize(self):
        self.left = 0

    def elapsed_time(self, other):
        return 2.0


class FakeRun2(FakeRun):
    def __init__(self, cfg, stream=None, workspace=None):
        super().__init__(cfg, stream)
        assert workspace is not None  # every workspace comes from the arena
        self.workspace = workspace


class FakeBatch2:
    made = []
    closed = 0

    def __init__(self, runs, stream=None, steps_left=None, workspace=None):
        assert steps_left is not None and workspace is not None
        self.runs = list(runs)
        self.left = min(steps_left)
        for r, k in zip(self.runs, steps_left):
            assert k == r.K - r.step_enq
        FakeBatch2.made.append(len(self.runs))

    def run_steps(self, n):
        assert n <= self.left
        self.left -= n
        for r in self.runs:
            r.step_enq += n
            assert r.step_enq <= r.K, "a run was stepped past K"
            r.step = r.step_enq

    def close(self):
        FakeBatch2.closed += 1


class FakeArena:
    def __init__(self, nbytes):
        from paper_2006_00561_gb300.serve import Arena
        self.a = Arena(nbytes, buffer=bytearray(0))
        self.out = 0

    def alloc(self, n):
        off = self.a.alloc(n)
        if off is not None:
            self.out += 1
        return off

    def release(self, off, n):
        self.out -= 1
        self.a.release(off, n)

    def view(self, off, n):
        return (off, n)


@pytest.fixture
def pipelined(S, monkeypatch):
    P, serve = S

    def run_factory(cfg, stream=None, workspace=None):
        r = FakeRun2(cfg, stream, workspace)
        r.step_enq = 0
        return r
    monkeypatch.setattr(serve.P, "Run", run_factory)
    monkeypatch.setattr(serve.P, "Batch", FakeBatch2)
    FakeRun.live = 0
    FakeBatch2.made = []
    FakeBatch2.closed = 0
    return P, serve


def make_pipelined(serve, budget, polls=1, **kw):
    srv = serve.PipelinedServer(hbm_budget=budget, stream=object(), admit_stream=object(),
                                arena=FakeArena(budget + serve.PipelinedServer.BATCH_RESERVE),
                                **kw)
    srv._event = lambda timing=False: FakeEvent(polls)
    srv._record = lambda ev, stream: None
    srv._wait = lambda stream, ev: None
    return srv


def test_pipelined_server_keeps_quanta_in_flight_and_returns_all_memory(pipelined):
    P, serve = pipelined
    one = P.pa_workspace_size(P.make_config(layout=P.LAYOUT_PACKED, **spec()))
    srv = make_pipelined(serve, 2 * one + one // 2, polls=2, quantum=3, depth=2)
    depth_seen = []
    orig = srv._enqueue

    def enqueue():
        ok = orig()
        depth_seen.append(len(srv.inflight))
        return ok
    srv._enqueue = enqueue
    trace = [dict(spec(K=7 + 2 * i), arrival=0.0) for i in range(5)]
    st = srv.run_trace(trace)
    assert st["served"] == 5 and st["waiting"] == 0 and st["resident"] == 0
    assert max(depth_seen) == 2          # two quanta in flight at once
    assert st["max_resident"] == 2       # the budget holds two requests
    assert all(r.result["step"] == r.spec["K"] for r in srv.done)
    assert srv.used == 0 and FakeRun.live == 0
    assert srv.arena.out == 0 and srv.arena.a.free_bytes() == srv.arena.a.size
    assert FakeBatch2.closed == len(FakeBatch2.made)
    assert st["quanta"] >= 5 and 0.0 <= st["gpu_idle_fraction"] <= 1.0
    # first come, first served: admissions in arrival order
    assert sorted(srv.done, key=lambda r: r.admitted)[0].rid == 0


def test_arena_first_fit_and_coalescing():
    from paper_2006_00561_gb300.serve import Arena
    a = Arena(10 * 256, buffer=bytearray(0))
    x = a.alloc(300)     # two blocks
    y = a.alloc(256)
    z = a.alloc(5 * 256)
    assert (x, y, z) == (0, 512, 768)
    assert a.alloc(3 * 256) is None
    a.release(y, 256)
    assert a.alloc(200) == 512          # first fit reuses the hole
    a.release(512, 200)
    a.release(x, 300)
    a.release(z, 5 * 256)
    assert a.free == [(0, 10 * 256)]
