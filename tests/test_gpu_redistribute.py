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
