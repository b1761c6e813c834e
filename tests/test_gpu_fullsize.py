"""Parity at the benchmark sizes, in the launch configuration bench.py times.

2D Ising L = 64 bit-packed with R0 = 2^21 (the paper-scale population, two
1 GiB buffers) and R0 = 2^17.  After every checked step:
  * reweight, on the whole population: tau tables (n, F), kref and S of
    Eq. 3 / 4 recomputed by the oracle from the dumped histogram;
  * copy counts and offsets of every replica, recomputed by the oracle from
    the dumped energy levels (bit for bit), and the new population size, for
    the nearest-integer rule and for the Poisson draw;
  * gather: sampled output slots hold exact copies of their source replica;
  * sweep: theta = 10 Metropolis sweeps of sampled replicas recomputed by the
    oracle from their dumped pre-sweep state (each replica's sweep is a pure
    function of its state, slot, sweep index and beta);
  * measurement: histogram == bincount(levels), integer observables == the
    sums over the dumped levels and magnetisations.
Graph-replayed steps (pa_run_steps) run between the checked ones.  The e2e
path's streamed step is checked at 2^21 against the graph step of a twin run,
and the whole 400-step run at 2^21 against Kaufman's exact ln Z and energy.
"""
from __future__ import annotations

import numpy as np
import pytest

from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2006_00561_gb300 import build as B
    B.build()
    from paper_2006_00561_gb300 import pa
    return pa


def check_step(P, run, ocfg, rng, nsample=48):
    N = ocfg.L ** ocfg.dim
    st0 = run.state()
    R_prev = st0["R"]
    ebin = run.dump(P.DUMP_EBIN)
    mag = run.dump(P.DUMP_MAG)
    hist = run.dump(P.DUMP_HIST)
    assert np.array_equal(hist, np.bincount(ebin, minlength=st0["bins"]))
    obs = run.observables()
    par = run.state()["parity"]
    E = 2 * (2 * ebin.astype(np.int64) + par) - ocfg.dim * N
    assert obs["sumE"] == E.sum() and obs["sumE2"] == (E * E).sum()
    assert obs["sumAbsM"] == np.abs(mag.astype(np.int64)).sum()
    assert obs["sumM2"] == (mag.astype(np.int64) ** 2).sum()
    src_sample = rng.choice(R_prev, size=nsample, replace=False)
    pre_src = {int(i): run.dump_range(P.DUMP_SPINS_RAW, int(i), 1)[0] for i in src_sample}

    run.resample()
    st = run.state()
    assert st["status_bits"] == 0
    step = st["step"]
    Dtab = np.array([O.weight(O.beta(ocfg, step) - O.beta(ocfg, step - 1), j)
                     for j in range(st["bins"])])
    S, kref, n, F = O.tau_table(hist, Dtab, ocfg.R0)
    assert st["kref"] == kref and st["S"] == S
    assert np.array_equal(run.dump(P.DUMP_TAB_N), n)
    assert np.array_equal(run.dump(P.DUMP_TAB_F), F)
    counts = run.dump(P.DUMP_COUNTS)
    draw = {O.RESAMPLE_POISSON: O.copy_counts_poisson,
            O.RESAMPLE_MULTINOMIAL: O.copy_counts_multinomial}.get(ocfg.resample, O.copy_counts)
    assert np.array_equal(counts, draw(ocfg, step, ebin, n, F))
    offsets = run.dump(P.DUMP_OFFSETS)
    csum = np.cumsum(counts.astype(np.int64))
    assert np.array_equal(offsets.astype(np.int64), csum - counts)
    assert st["R"] == csum[-1]
    # gather: output slots copy their sources
    for i in src_sample:
        i = int(i)
        for k in range(int(counts[i])):
            got = run.dump_range(P.DUMP_SPINS_RAW, int(offsets[i]) + k, 1)[0]
            assert np.array_equal(got, pre_src[i])
    # sweep of sampled replicas
    R = st["R"]
    slots = rng.choice(R, size=nsample, replace=False)
    pre = {int(s): run.dump_range(P.DUMP_SPINS, int(s), 1)[0].copy() for s in slots}
    g0 = st["sweeps_done"]
    run.sweep(ocfg.theta)
    T = [O.threshold(O.beta(ocfg, step), 4 * (c + 1)) for c in range(3)]
    J = O.couplings(ocfg)
    for s, spins in pre.items():
        O.sweep_replica(ocfg, J, spins, s, g0, ocfg.theta, T)
        assert np.array_equal(run.dump_range(P.DUMP_SPINS, s, 1)[0], spins), (step, s)
    assert run.status() == 0


@pytest.mark.parametrize("R0,seed,checks,resample", [(1 << 21, 3, 3, 0), (1 << 17, 2, 4, 0),
                                                     (1 << 21, 3, 3, 1), (1 << 21, 3, 3, 2)],
                         ids=["2p21", "2p17", "2p21_poisson", "2p21_multinomial"])
def test_fullsize_parity(P, R0, seed, checks, resample):
    K = 400 if R0 == 1 << 21 else 200
    ocfg = O.make_config(dim=2, L=64, R0=R0, K=K, theta=10, seed=seed, resample=resample)
    run = P.Run(P.make_config(dim=2, L=64, layout=P.LAYOUT_PACKED, R0=R0, K=K, theta=10,
                              seed=seed, resample=resample))
    rng = np.random.default_rng(R0)
    # initial population: sampled replicas equal the oracle's uniform init
    for s in rng.choice(R0, size=16, replace=False):
        assert np.array_equal(run.dump_range(P.DUMP_SPINS, int(s), 1)[0],
                              O.init_replica(ocfg, int(s)))
    for c in range(checks):
        check_step(P, run, ocfg, rng)
        run.run_steps(2 + 3 * c)
        assert run.status() == 0
    st = run.state()
    assert abs(st["R"] - R0) < 5 * np.sqrt(R0)
    run.close()


@pytest.mark.parametrize("L,R0", [(10, 1 << 16), (16, (1 << 14) + 77)])
def test_fullsize_parity_3d_pm_j(P, L, R0):
    """The replica-sliced kernel at scale: a 3D +-J run with 2^11 or more
    32-replica chunks (and a partial last chunk), checked like the 2D runs
    above."""
    ocfg = O.make_config(dim=3, L=L, model=O.MODEL_PMJ, R0=R0, K=150, theta=10, beta_max=3.0,
                         seed=40 + L, coupling_seed=50 + L, instance_id=7)
    run = P.Run(P.make_config(dim=3, L=L, model=P.MODEL_PMJ, layout=P.LAYOUT_PACKED, R0=R0,
                              K=150, theta=10, beta_max=3.0, seed=40 + L, coupling_seed=50 + L,
                              instance_id=7))
    rng = np.random.default_rng(L)
    for s in rng.choice(R0, size=8, replace=False):
        assert np.array_equal(run.dump_range(P.DUMP_SPINS, int(s), 1)[0],
                              O.init_replica(ocfg, int(s)))
    for c in range(3):
        check_step(P, run, ocfg, rng, nsample=16)
        run.run_steps(5 + 10 * c)
        assert run.status() == 0
    run.close()


def test_fullsize_streamed_step_equals_the_graph_step(P):
    """The e2e path at the bench size: pa_step_stream (8 slot ranges, each copied
    to pinned host memory on a second stream while the next range sweeps)
    gives the same run, bit for bit, as pa_run_steps on a twin run, and the
    host copy is the whole new population."""
    import torch
    cfg = P.make_config(dim=2, L=64, layout=P.LAYOUT_PACKED, R0=1 << 21, K=400, theta=10,
                        seed=3)
    a, b = P.Run(cfg), P.Run(cfg)
    try:
        st = a.state()
        host = torch.zeros(st["capacity"] * st["stride"], dtype=torch.uint8, pin_memory=True)
        cs = torch.cuda.Stream()
        for _ in range(2):
            R = a.step_stream(host, 8, cs)
            b.run_steps(1)
            oa, ob = a.observables(), b.observables()
            assert R == oa["R"] == ob["R"]
            for k in ("sumE", "sumE2", "sumAbsM", "sumM2", "lnZ"):
                assert oa[k] == ob[k], k
            raw_a = a.dump(P.DUMP_SPINS_RAW).reshape(-1)
            assert np.array_equal(raw_a[: R * st["stride"]], b.dump(P.DUMP_SPINS_RAW).reshape(-1)[: R * st["stride"]])
            assert np.array_equal(host.numpy()[: R * st["stride"]], raw_a[: R * st["stride"]])
    finally:
        a.close()
        b.close()


def test_config3_whole_run_matches_kaufman(P):
    """The whole paper-scale run (2D Ising L = 64, 2^21 replicas, beta 0 -> 1 in
    400 steps, theta = 10, graph-replayed) ends at Kaufman's exact ln Z(1) and
    <E>/N of the 64 x 64 torus.  Two seeds gave deviations of 0.009 / 0.003 in
    ln Z and 8e-7 / 5e-7 in <E>/N; the bounds are about six times those."""
    pytest.importorskip("mpmath")
    import exact
    cfg = P.make_config(dim=2, L=64, layout=P.LAYOUT_PACKED, R0=1 << 21, K=400, theta=10, seed=3)
    run = P.Run(cfg)
    try:
        run.run_steps(400)
        o = run.observables()
    finally:
        run.close()
    assert o["step"] == 400 and o["beta"] == 1.0
    assert abs(o["R"] - (1 << 21)) <= 5 * np.sqrt(1 << 21)
    assert abs(o["lnZ"] - float(exact.kaufman_lnZ(64, 1.0))) < 0.05
    assert abs(o["e"] - exact.kaufman_energy_per_site(64, 1.0)) < 5e-6


def _oracle_sweep_slice(job):
    """The oracle's theta sweeps of consecutive replicas (slots slot0 ..) from
    their pre-sweep states; runs in a spawned worker process."""
    import os
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    from oracle import oracle as Ow
    cfg_kw, spins, slot0, g0, T = job
    cfg = Ow.make_config(**cfg_kw)
    J = Ow.couplings(cfg)
    out = np.ascontiguousarray(spins)
    for k in range(out.shape[0]):
        row = out[k]
        Ow.sweep_replica(cfg, J, row, slot0 + k, g0, cfg.theta, T)
    return out


def test_config2_whole_step_every_replica_matches_the_oracle(P):
    """Config 2 (2D L = 64 packed, R0 = 2^17, 200 steps, theta = 10, seed 2)
    checked whole: from the device population after step 100, the oracle
    recomputes step 101 for all ~131 000 replicas -- tau tables, every copy
    count, the copies, and theta = 10 sweeps of every replica (spread over one
    spawned process per host core) -- and the device's step 101 equals it
    replica for replica."""
    import multiprocessing as mpc
    import os
    kw = dict(dim=2, L=64, R0=1 << 17, K=200, theta=10, seed=2)
    ocfg = O.make_config(**kw)
    run = P.Run(P.make_config(layout=P.LAYOUT_PACKED, **kw))
    run.run_steps(100)
    st0 = run.state()
    assert st0["status_bits"] == 0 and st0["step"] == 100
    spins0 = run.dump(P.DUMP_SPINS).reshape(st0["R"], -1)
    ebin0 = run.dump(P.DUMP_EBIN)
    hist0 = run.dump(P.DUMP_HIST)
    run.step()
    st = run.state()
    step = st["step"]
    Dtab = np.array([O.weight(O.beta(ocfg, step) - O.beta(ocfg, step - 1), j)
                     for j in range(st["bins"])])
    S, kref, n, F = O.tau_table(hist0, Dtab, ocfg.R0)
    assert st["S"] == S and st["kref"] == kref
    counts = O.copy_counts(ocfg, step, ebin0, n, F)
    assert np.array_equal(run.dump(P.DUMP_COUNTS), counts)
    pre = np.repeat(spins0, counts, axis=0)  # the copies, in slot order
    del spins0
    assert pre.shape[0] == st["R"]
    T = [O.threshold(O.beta(ocfg, step), 4 * (c + 1)) for c in range(3)]
    g0 = (step - 1) * ocfg.theta
    procs = max(1, min(32, os.cpu_count() or 1))
    bounds = np.linspace(0, pre.shape[0], procs + 1).astype(int)
    jobs = [(kw, pre[a:b], int(a), g0, T) for a, b in zip(bounds[:-1], bounds[1:])]
    with mpc.get_context("spawn").Pool(procs) as pool:
        want = np.concatenate(pool.map(_oracle_sweep_slice, jobs))
    got = run.dump(P.DUMP_SPINS).reshape(st["R"], -1)
    bad = np.nonzero((got != want).any(axis=1))[0]
    assert bad.size == 0, f"{bad.size} replicas differ, first {bad[:5]}"
    run.close()
