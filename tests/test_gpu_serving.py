"""Serving (continuous batching) on the GPU.

Requests of mixed classes arrive while others are running, wait for HBM,
join the batched device work mid-flight and retire independently.  Each
request's result must be the same as when it runs alone: the whole
observables history and the final population, bit for bit (FP64 included,
since the same kernels compute them), and one request against the oracle.
"""
from __future__ import annotations

import numpy as np
import pytest

from lockstep import compare_obs
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2006_00561_gb300 import build as B
    B.build()
    from paper_2006_00561_gb300 import pa
    return pa


def _trace():
    specs = []
    classes = [(2, 16, 0), (2, 32, 0), (2, 64, 0), (2, 128, 0), (3, 6, 1), (3, 8, 1), (3, 10, 1)]
    rng = np.random.default_rng(55)
    for i in range(12):
        dim, L, model = classes[i % len(classes)]
        specs.append(dict(arrival=0.002 * i, dim=dim, L=L, model=model,
                          R0=int(rng.integers(64, 1500)), K=int(rng.integers(6, 18)), theta=3,
                          beta0=0.0, beta_max=float(rng.choice([1.0, 3.0])),
                          seed=int(rng.integers(1, 2 ** 62)),
                          coupling_seed=int(rng.integers(1, 2 ** 62)), instance_id=100 + i))
    return specs


@pytest.mark.parametrize("kind", ["sync", "pipelined"])
def test_each_result_is_the_same_alone_and_in_the_mix(P, kind):
    """Both servers: the synchronous loop, and the pipelined one that keeps two
    quanta in flight, admits on a second stream and builds the next batch
    while the device runs the current one."""
    from paper_2006_00561_gb300 import serve
    trace = _trace()
    sizes = sorted(P.pa_workspace_size(P.make_config(**{k: v for k, v in s.items()
                                                        if k != "arrival"})) for s in trace)
    budget = sum(sizes[-4:])  # about four requests resident at a time
    if kind == "sync":
        srv = serve.Server(hbm_budget=budget, quantum=3, keep_spins=True)
    else:
        srv = serve.PipelinedServer(hbm_budget=budget, quantum=3, depth=2, keep_spins=True)
    stats = srv.run_trace(trace)
    assert stats["served"] == len(trace) and stats["rejected"] == 0
    assert 2 <= stats["max_resident"] < len(trace)
    assert stats["iterations"] > 4
    if kind == "pipelined":
        assert srv.used == 0 and srv.arena.free_bytes() == srv.arena.size
        assert 0.0 <= stats["gpu_idle_fraction"] < 1.0
    for req in srv.done:
        spec = {k: v for k, v in req.spec.items() if k != "arrival"}
        run = P.Run(P.make_config(**spec))
        for _ in range(spec["K"]):
            run.step()
        alone = run.history(0, spec["K"] + 1)
        assert alone == req.history, req.rid
        assert np.array_equal(run.spins(), req.spins), req.rid
        run.close()
    # one request against the oracle
    req = next(r for r in srv.done if r.spec["dim"] == 3)
    spec = {k: v for k, v in req.spec.items() if k not in ("arrival",)}
    orun = O.Run(O.make_config(**spec))
    for i in range(1, spec["K"] + 1):
        assert orun.step() == 0
        compare_obs(req.history[i], orun.observables(), f"request {req.rid} step {i}")
    assert np.array_equal(req.spins, orun.spins())


def test_admission_respects_the_hbm_budget(P):
    from paper_2006_00561_gb300 import serve
    trace = _trace()[:6]
    big = dict(trace[0], R0=1 << 20, dim=2, L=64, model=0, arrival=0.0)
    need = max(P.pa_workspace_size(P.make_config(**{k: v for k, v in s.items()
                                                    if k != "arrival"})) for s in trace)
    srv = serve.Server(hbm_budget=3 * need, quantum=2)
    r = srv.submit(999, {k: v for k, v in big.items() if k != "arrival"}, 0.0)
    assert r.error and "budget" in r.error
    stats = srv.run_trace(trace)
    assert stats["served"] == 6 and stats["rejected"] == 1
    assert 0 < stats["max_hbm_bytes"] <= 3 * need
    assert srv.used == 0
