"""The seeded synthetic workloads of configs 4 and 5 (paper_2006_00561_gb300/
workloads.py) follow their stated recipes: the 3D +-J ensemble draws L and R0
uniformly from their sets with one coupling and one Metropolis seed per
instance; the serving trace has Poisson arrivals at the stated rate, classes
uniform over the mix, R0 = 2^U with U uniform, K uniform.  Same seed, same
workload."""
from __future__ import annotations

import numpy as np
from scipy import stats

from paper_2006_00561_gb300 import workloads as W


def test_ea_ensemble_recipe():
    specs = W.ea_ensemble(256, seed=4)
    assert specs == W.ea_ensemble(256, seed=4)
    assert specs != W.ea_ensemble(256, seed=5)
    assert len(specs) == 256
    assert [s["instance_id"] for s in specs] == list(range(256))
    for s in specs:
        assert s["dim"] == 3 and s["model"] == 1 and s["L"] in (6, 8, 10)
        assert s["R0"] in (1 << 14, 1 << 15, 1 << 16)
        assert (s["K"], s["theta"], s["beta0"], s["beta_max"]) == (150, 10, 0.0, 3.0)
    assert len({s["seed"] for s in specs}) == 256
    assert len({s["coupling_seed"] for s in specs}) == 256
    # uniform over the sets: chi-square against equal counts
    for key, values in (("L", (6, 8, 10)), ("R0", (1 << 14, 1 << 15, 1 << 16))):
        counts = [sum(s[key] == v for s in specs) for v in values]
        assert stats.chisquare(counts).pvalue > 1e-4


def test_serving_trace_recipe():
    tr = W.serving_trace(256, rate=50.0, seed=5)
    assert tr == W.serving_trace(256, rate=50.0, seed=5)
    t = np.array([r["arrival"] for r in tr])
    assert (np.diff(t) > 0).all()
    gaps = np.diff(np.concatenate([[0.0], t]))
    # exponential inter-arrival times of mean 1/50 s: mean within 4 SE, and a KS test
    assert abs(gaps.mean() - 0.02) < 4 * 0.02 / np.sqrt(len(gaps))
    assert stats.kstest(gaps, "expon", args=(0, 0.02)).pvalue > 1e-4
    classes = [(r["dim"], r["L"]) for r in tr]
    assert set(classes) <= set(W.SERVING_CLASSES)
    assert stats.chisquare([classes.count(c) for c in W.SERVING_CLASSES]).pvalue > 1e-4
    for r in tr:
        assert r["model"] == (0 if r["dim"] == 2 else 1)
        u = int(np.log2(r["R0"]))
        assert r["R0"] == 1 << u and 12 <= u <= 18
        assert 100 <= r["K"] <= 300 and r["theta"] == 10
        assert r["beta_max"] in (1.0, 3.0)
