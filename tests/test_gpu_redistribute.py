"""Replica exchange between virtual GPUs (Sec. 3) executed on the device.

The population's N "GPUs" are consecutive slot ranges.  Every step the engine
computes the copy counts and scan (pa_resample_begin), the host reads the
shards' offspring ranges and plans the exchange (the main block algorithm or
the naive per-replica one), and the engine's gather writes every replica into
its exchanged slot (pa_resample_finish).  The CPU oracle runs the same steps
and applies the same slot order with its own code (or_permute); explicit
per-replica shard labels are carried through the oracle's resamples and
exchanges.  After every step the device population equals the oracle's bit
for bit, and the replicas in shard n's range are exactly those the oracle's
labels place in shard n."""
from __future__ import annotations

import numpy as np
import pytest
from lockstep import compare_state, configs

from oracle import oracle as O
from paper_2006_00561_gb300 import redistribute as RD

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2006_00561_gb300 import build as B
    B.build()
    from paper_2006_00561_gb300 import pa
    return pa


@pytest.mark.parametrize("policy,spec", [
    ("main", dict(dim=2, L=64, layout=1, R0=8 * 512, K=14, theta=1, beta_max=1.0, seed=11)),
    ("naive", dict(dim=2, L=64, layout=1, R0=8 * 512, K=14, theta=1, beta_max=1.0, seed=12)),
    ("main", dict(dim=2, L=16, layout=0, R0=6 * 700, K=12, theta=2, beta_max=1.2, seed=13)),
    ("naive", dict(dim=3, L=8, layout=1, model=1, R0=5 * 600, K=12, theta=2, beta_max=2.0,
                   seed=14, coupling_seed=15, instance_id=3)),
    ("independent", dict(dim=2, L=64, layout=1, R0=4 * 512, K=8, theta=1, beta_max=1.0,
                         seed=16)),
], ids=["main_L64", "naive_L64", "main_int8", "naive_3d_pmj", "independent"])
def test_exchange_on_the_device_follows_the_oracle(P, policy, spec):
    N = {8 * 512: 8, 6 * 700: 6, 5 * 600: 5, 4 * 512: 4}[spec["R0"]]
    block = 16
    ocfg, gcfg = configs(P, **spec)
    orun, grun = O.Run(ocfg), P.Run(gcfg)
    bounds = RD.bounds_from_loads(RD.desired_loads(spec["R0"], N))
    labels = np.repeat(np.arange(N), np.diff(bounds))
    moved_any = False
    for i in range(1, spec["K"] + 1):
        assert orun.resample() == 0
        x = RD.exchange_step(grun, bounds, policy, block=block, maxexc=1)
        # the shards' offspring, read on the device, are the oracle's labels
        labels = np.repeat(labels, orun.counts())
        assert np.array_equal(labels, np.repeat(np.arange(N), np.diff(x["offspring_bounds"])))
        assert orun.permute(x["segments"]) == 0
        perm = np.concatenate([np.arange(a, a + k) for a, k in x["segments"]])
        came = labels[perm]
        new = x["bounds"]
        for n in range(N):
            senders = {s for s, d, _ in x["moves"] if d == n}
            assert set(came[new[n]:new[n + 1]].tolist()) <= {n} | senders, (i, n)
        moved_any |= bool(x["moves"])
        labels = np.repeat(np.arange(N), np.diff(new))
        bounds = new
        assert orun.sweep(spec["theta"]) == 0
        grun.sweep(spec["theta"])
        compare_state(P, grun, orun, i)
    assert moved_any == (policy != "independent")
    grun.close()
    orun.close()


def test_pending_gather_blocks_other_calls_and_one_segment_is_a_plain_step(P):
    """Between pa_resample_begin and pa_resample_finish every other stepping
    call is refused; finishing with the single segment (0, R) gives exactly the
    plain step."""
    spec = dict(dim=2, L=16, layout=1, R0=1500, K=6, theta=2, beta_max=1.0, seed=17)
    _, gcfg = configs(P, **spec)
    a, b = P.Run(gcfg), P.Run(gcfg)
    for _ in range(3):
        a.step()
        b.resample_begin()
        for call in (b.step, b.resample, lambda: b.sweep(1), lambda: b.run_steps(1)):
            with pytest.raises(P.PaError):
                call()
        with pytest.raises(P.PaError):
            b.resample_finish([(0, b.state()["R"] - 1)])  # does not cover R
        b.resample_finish([(0, b.state()["R"])])
        b.sweep(spec["theta"])
        for what in (P.DUMP_SPINS_RAW, P.DUMP_EBIN, P.DUMP_MAG, P.DUMP_HIST, P.DUMP_COUNTS):
            assert np.array_equal(a.dump(what), b.dump(what))
    a.close()
    b.close()


def test_exchange_at_the_paper_workload_every_replica(P):
    """The paper's workload (Sec. 3): 8 GPUs x 20 480 replicas of the 2D Ising
    model at L = 64, beta 0 -> 1 in 200 steps, theta = 1, naive exchange.
    After 90 steps on the device (the critical region, where the naive rule
    moves the most replicas), the oracle recomputes step 91 for every replica
    from the device's state: copy counts, copies, the exchanged slot order and
    the sweep (spread over one spawned process per host core); the device's
    step 91 equals it replica for replica."""
    import multiprocessing as mpc
    import os

    from test_gpu_fullsize import _oracle_sweep_slice
    kw = dict(dim=2, L=64, R0=8 * 20480, K=200, theta=1, seed=2006)
    ocfg = O.make_config(**kw)
    run = P.Run(P.make_config(layout=P.LAYOUT_PACKED, **kw))
    N = 8
    bounds = RD.bounds_from_loads(RD.desired_loads(kw["R0"], N))
    for _ in range(90):
        bounds = RD.exchange_step(run, bounds, "naive")["bounds"]
        run.sweep(kw["theta"])
    st0 = run.state()
    assert st0["status_bits"] == 0 and st0["step"] == 90
    spins0 = run.dump(P.DUMP_SPINS).reshape(st0["R"], -1)
    ebin0 = run.dump(P.DUMP_EBIN)
    hist0 = run.dump(P.DUMP_HIST)
    x = RD.exchange_step(run, bounds, "naive")
    assert x["moves"], "the naive rule moves replicas near the critical point"
    run.sweep(kw["theta"])
    st = run.state()
    step = st["step"]
    Dtab = np.array([O.weight(O.beta(ocfg, step) - O.beta(ocfg, step - 1), j)
                     for j in range(st["bins"])])
    S, kref, n, F = O.tau_table(hist0, Dtab, ocfg.R0)
    assert st["S"] == S and st["kref"] == kref
    counts = O.copy_counts(ocfg, step, ebin0, n, F)
    assert np.array_equal(run.dump(P.DUMP_COUNTS), counts)
    copies = np.repeat(spins0, counts, axis=0)
    del spins0
    perm = np.concatenate([np.arange(a, a + k) for a, k in x["segments"]])
    pre = copies[perm]
    del copies
    T = [O.threshold(O.beta(ocfg, step), 4 * (c + 1)) for c in range(3)]
    g0 = (step - 1) * kw["theta"]
    procs = max(1, min(32, os.cpu_count() or 1))
    cuts = np.linspace(0, pre.shape[0], procs + 1).astype(int)
    jobs = [(kw, pre[a:b], int(a), g0, T) for a, b in zip(cuts[:-1], cuts[1:])]
    with mpc.get_context("spawn").Pool(procs) as pool:
        want = np.concatenate(pool.map(_oracle_sweep_slice, jobs))
    got = run.dump(P.DUMP_SPINS).reshape(st["R"], -1)
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} replicas differ, first {bad[:5]}"
    run.close()


def test_exchange_scan_timeout_is_reported_and_the_context_survives(P):
    """The scan of pa_resample_begin has the resample's bounded lookback wait:
    with tile 0's prefix withheld (test hook) the wait runs out, the sticky
    PA_ERR_TIMEOUT is reported, the pending gather can still be finished (every
    copy stays inside the population buffers), and a fresh run on the same
    context then follows the oracle."""
    import time
    spec = dict(dim=2, L=16, layout=1, R0=5000, K=4, theta=1, seed=3)  # 3 scan tiles
    _, gcfg = configs(P, **spec)
    run = P.Run(gcfg)
    run.step()
    assert run.status() == 0
    P.pa_debug(run.h, P.DEBUG_WITHHOLD_PREFIX)
    t0 = time.perf_counter()
    run.resample_begin()
    assert run.status() == -5  # PA_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 60.0
    run.resample_finish([(0, run.state()["R"])])
    assert run.status() == -5
    run.close()
    ocfg, gcfg = configs(P, **spec)
    orun, grun = O.Run(ocfg), P.Run(gcfg)
    bounds = RD.bounds_from_loads(RD.desired_loads(spec["R0"], 4))
    for i in range(1, 3):
        assert orun.resample() == 0
        x = RD.exchange_step(grun, bounds, "naive")
        assert orun.permute(x["segments"]) == 0
        bounds = x["bounds"]
        assert orun.sweep(1) == 0
        grun.sweep(1)
        compare_state(P, grun, orun, i)
    grun.close()
    orun.close()
