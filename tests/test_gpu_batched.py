"""The batched form (pa_batch_*) against the plain path and the oracle.

Every run of a batch must produce exactly the bits it produces when stepped
alone with pa_step (spins, levels, magnetisations, histograms, copy counts,
offsets, observables), whatever the mix of classes, the launch shape chosen
for a class, or whether steps are replayed from a CUDA graph.
"""
from __future__ import annotations

import numpy as np
import pytest

from lockstep import compare_obs, compare_state
from oracle import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2006_00561_gb300 import build as B
    B.build()
    from paper_2006_00561_gb300 import pa
    return pa


MIX = [
    dict(dim=3, L=6, model=1, layout=1, R0=700, seed=11, coupling_seed=101, instance_id=1),
    dict(dim=3, L=8, model=1, layout=1, R0=2500, seed=12, coupling_seed=102, instance_id=2),
    dict(dim=3, L=10, model=1, layout=1, R0=333, seed=13, coupling_seed=103, instance_id=3),
    dict(dim=3, L=8, model=1, layout=1, R0=64, seed=14, coupling_seed=104, instance_id=4),
    dict(dim=2, L=16, model=0, layout=0, R0=1000, seed=15, instance_id=5),
    dict(dim=2, L=64, model=0, layout=1, R0=300, seed=16, instance_id=6),
    dict(dim=3, L=4, model=1, layout=0, R0=5001, seed=17, coupling_seed=107, instance_id=7),
    dict(dim=2, L=128, model=0, layout=1, R0=40, seed=18, instance_id=8),
    dict(dim=2, L=64, model=1, layout=1, R0=200, seed=19, coupling_seed=109, instance_id=9),
]
COMMON = dict(K=12, theta=3, beta_max=2.0)


def _runs(P, specs):
    return [P.Run(P.make_config(**dict(COMMON, **s))) for s in specs]


def _same(P, a, b, where):
    sa, sb = a.state(), b.state()
    for k in ("step", "R", "R_prev", "kref", "sweeps_done", "status_bits", "S", "lnZ"):
        assert sa[k] == sb[k], (where, k, sa[k], sb[k])
    for what in (P.DUMP_SPINS_RAW, P.DUMP_EBIN, P.DUMP_MAG, P.DUMP_HIST, P.DUMP_COUNTS,
                 P.DUMP_OFFSETS, P.DUMP_TAB_N, P.DUMP_TAB_F):
        assert np.array_equal(a.dump(what), b.dump(what)), (where, what)
    assert a.history(0, sa["step"] + 1) == b.history(0, sb["step"] + 1), where


def test_batched_steps_equal_plain_steps(P):
    plain = _runs(P, MIX)
    batched = _runs(P, MIX)
    batch = P.Batch(batched)
    cls = batch.classes()
    assert len(cls) == 8 and sum(c["runs"] for c in cls) == len(MIX)
    for step in range(1, 7):
        for r in plain:
            r.step()
        if step % 2:
            batch.step()
        else:
            batch.run_steps(1)
        assert batch.sync() == 0
        for i, (a, b) in enumerate(zip(plain, batched)):
            _same(P, a, b, f"step {step} run {i}")
    batch.close()


def test_launch_shape_does_not_change_results(P):
    specs = MIX[:4]
    plain = _runs(P, specs)
    batched = _runs(P, specs)
    batch = P.Batch(batched)
    shapes = [(2, 1), (8, 32), (4, 4), (8, 2), (2, 0)]
    for step, (w, chunk) in enumerate(shapes, start=1):
        for c, info in enumerate(batch.classes()):
            if info["warps"] != 16:
                batch.set_shape(c, w, chunk)
                assert batch.classes()[c]["warps"] == w
                if chunk:
                    assert batch.classes()[c]["chunk"] == chunk
        batch.run_steps(1)
        for r in plain:
            r.step()
        assert batch.sync() == 0
        for i, (a, b) in enumerate(zip(plain, batched)):
            _same(P, a, b, f"step {step} run {i} warps {w}")
    batch.close()


def test_batched_run_matches_oracle(P):
    spec = dict(COMMON, **MIX[1])
    orun = O.Run(O.make_config(**{k: v for k, v in spec.items() if k != "layout"}))
    runs = _runs(P, MIX[:3])
    batch = P.Batch(runs)
    for step in range(1, 6):
        assert orun.step() == 0
        batch.step()
        assert batch.sync() == 0
        compare_state(P, runs[1], orun, step)
    batch.close()


@pytest.mark.parametrize("rules", [(0, 1, 0, 1), (2, 1, 0, 2)], ids=["poisson", "all_three"])
def test_batch_mixing_resampling_rules(P, rules):
    """Runs on the nearest-integer, Poisson and multinomial rules in one batch:
    each run equals its plain twin, and the second run equals the oracle."""
    specs = [dict(MIX[i], resample=rule) for i, rule in zip((1, 4, 5, 6), rules)]
    plain = _runs(P, specs)
    batched = _runs(P, specs)
    spec = dict(COMMON, **specs[1])
    orun = O.Run(O.make_config(**{k: v for k, v in spec.items() if k != "layout"}))
    batch = P.Batch(batched)
    for step in range(1, 6):
        for r in plain:
            r.step()
        assert orun.step() == 0
        batch.run_steps(1)
        assert batch.sync() == 0
        for i, (a, b) in enumerate(zip(plain, batched)):
            _same(P, a, b, f"step {step} run {i}")
        compare_state(P, batched[1], orun, step)
    batch.close()


def test_batch_refuses_to_pass_K(P):
    runs = _runs(P, [dict(dict(COMMON, K=2), **MIX[0])])
    batch = P.Batch(runs)
    batch.run_steps(2)
    with pytest.raises(P.PaError) as e:
        batch.step()
    assert e.value.code == -8
    assert batch.sync() == 0
    batch.close()


def test_config4_ensemble_batched_equals_plain(P):
    """The 256-instance +-J ensemble (L in {6,8,10}, R0 in {2^14,2^15,2^16}):
    two batched graph steps against plain steps, levels, histograms, counts
    and offsets of every instance, spins of a sample of instances."""
    from paper_2006_00561_gb300 import workloads
    specs = workloads.ea_ensemble(256, seed=4)
    rng = np.random.default_rng(0)
    plain = [P.Run(P.make_config(layout=1, **s)) for s in specs]
    batched = [P.Run(P.make_config(layout=1, **s)) for s in specs]
    batch = P.Batch(batched)
    assert len(batch.classes()) == 3
    for step in (1, 2):
        for r in plain:
            r.step()
        batch.run_steps(1)
        assert batch.sync() == 0
        for i, (a, b) in enumerate(zip(plain, batched)):
            assert a.state()["R"] == b.state()["R"]
            for what in (P.DUMP_EBIN, P.DUMP_HIST, P.DUMP_COUNTS, P.DUMP_OFFSETS):
                assert np.array_equal(a.dump(what), b.dump(what)), (step, i, what)
            compare_obs(a.observables(), b.observables(), f"step {step} inst {i}")
        for i in rng.choice(256, size=8, replace=False):
            assert np.array_equal(plain[i].dump(P.DUMP_SPINS_RAW),
                                  batched[i].dump(P.DUMP_SPINS_RAW))
    batch.close()
    for r in plain + batched:
        r.close()


def test_async_batch_and_phase_profile(P):
    """pa_batch_init_async (remaining steps from the caller, nothing waited
    for) steps every run to the bits of pa_batch_init's batch; its phase
    profile counts every non-graph step and times every phase; a wrong
    remaining-step count is refused."""
    import torch
    a_runs, b_runs = _runs(P, MIX[:5]), _runs(P, MIX[:5])
    a = P.Batch(a_runs)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())  # the runs' init, ordered before the batch
    b = P.Batch(b_runs, stream=s, steps_left=[COMMON["K"]] * 5)
    b.profile(True)
    for _ in range(3):
        a.step()
        b.step()
    b.run_steps(2)  # graph replays are not profiled
    a.run_steps(2)
    prof = b.profile_read(reset=True)
    assert a.sync() == 0 and b.sync() == 0
    assert prof["steps"] == 3
    assert all(prof[k] > 0.0 for k in ("reweight", "resample", "sweep", "obs"))
    for ra, rb in zip(a_runs, b_runs):
        _same(P, ra, rb, "async batch")
    with pytest.raises(P.PaError):
        P.Batch(_runs(P, MIX[:1]), steps_left=[COMMON["K"] + 1])
    a.close()
    b.close()
    for r in a_runs + b_runs:
        r.close()
