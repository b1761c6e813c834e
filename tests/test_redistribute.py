"""Host logic of the virtual-shard redistribution (Sec. 3 of the paper):
interval bookkeeping, the block ("main") plan and the proportional ("naive")
plan, checked on synthetic loads and on the oracle's real resamples against an
explicit per-replica shard label array."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2006_00561_gb300 import redistribute as RD
from oracle import oracle as O


def test_intervals_follow_the_offspring():
    offsets = np.array([0, 2, 2, 5, 6], dtype=np.uint32)  # counts 2,0,3,1,1 -> R_new 7
    assert RD.map_intervals([(0, 2)], offsets, 7) == [(0, 2)]
    assert RD.map_intervals([(1, 3)], offsets, 7) == [(2, 5)]
    assert RD.map_intervals([(3, 5)], offsets, 7) == [(5, 7)]
    assert RD.map_intervals([(1, 2)], offsets, 7) == []      # no offspring
    assert RD.map_intervals([(0, 2), (2, 4)], offsets, 7) == [(0, 6)]  # merged


def test_take_from_end_and_loads():
    kept, taken = RD.take_from_end([(0, 5), (10, 13)], 4)
    assert kept == [(0, 4)] and taken == [(4, 5), (10, 13)]
    assert RD.load(kept) + RD.load(taken) == 8


@pytest.mark.parametrize("match", ["order", "largest"])
@pytest.mark.parametrize("maxexc", [1, 2])
def test_main_plan_conserves_and_balances(maxexc, match):
    rng = np.random.default_rng(maxexc)
    B = 1024
    for _ in range(200):
        loads = [int(x) for x in rng.integers(5_000, 60_000, size=8)]
        moves = RD.plan_main(loads, block=B, maxexc=maxexc, match=match)
        if match == "order":
            # surplus and deficit shards are paired in shard order
            assert moves == sorted(moves)
        cur = list(loads)
        for s, d in moves:
            assert s != d
            cur[s] -= B
            cur[d] += B
        assert sum(cur) == sum(loads)
        want = RD.desired_loads(sum(loads), 8)
        exc = [c - w for c, w in zip(cur, want)]
        # no shard pair qualifies any more: either nobody has maxexc blocks of
        # excess, or nobody maxexc blocks of shortage
        assert max(exc) < maxexc * B or -min(exc) < maxexc * B
        # blocks only leave shards that were above the desired load
        for s, _ in moves:
            assert loads[s] > want[s]


def test_main_order_matching_small_case():
    """Four shards at desired load 10 (block 2, maxexc 1): shard 0 (+4) fills
    shard 1 (-4) before shard 2 (+2) gives to shard 3 (-2)."""
    loads = [14, 6, 12, 8]
    assert RD.plan_main(loads, block=2, maxexc=1) == [(0, 1), (0, 1), (2, 3)]
    assert RD.plan_main(loads, block=2, maxexc=2) == [(0, 1)]
    with pytest.raises(ValueError):
        RD.plan_main(loads, block=2, match="nearest")


def test_naive_plan_moves_half_the_surplus():
    loads = [40_000, 20_000, 20_000, 0 + 10_000]
    moves = RD.plan_naive(loads, alpha=0.5)
    want = RD.desired_loads(sum(loads), 4)
    cur = list(loads)
    for s, d, k in moves:
        assert loads[s] > want[s] and loads[d] < want[d] and k > 0
        cur[s] -= k
        cur[d] += k
    assert sum(cur) == sum(loads)
    assert loads[0] - cur[0] == int(0.5 * (loads[0] - want[0]))
    assert RD.plan_naive([5, 5, 5, 5]) == []


def test_shard_loads_match_explicit_labels_on_oracle_resamples():
    """Propagate an explicit shard label per replica through real resamples of
    the oracle (labels copied with the replicas, blocks relabelled by the plan)
    and compare with the interval bookkeeping."""
    cfg = O.make_config(dim=2, L=8, R0=4000, K=30, theta=2, beta_max=2.0, seed=77)
    run = O.Run(cfg)
    N, B = 4, 64
    for policy in ("independent", "naive", "main"):
        run = O.Run(cfg)
        sh = RD.Shards(run.R, N)
        labels = np.concatenate([np.full(w, n) for n, w in enumerate(RD.desired_loads(run.R, N))])
        for _ in range(cfg.K):
            assert run.resample() == 0
            counts, offsets = run.counts(), run.offsets()
            labels = np.repeat(labels, counts)
            sh.after_resample(offsets, run.R)
            assert sh.loads() == [int((labels == n).sum()) for n in range(N)]
            sh.redistribute(policy, block=B, maxexc=1)
            for n, iv in enumerate(sh.intervals):
                for a, b in iv:
                    labels[a:b] = n
            assert sum(sh.loads()) == run.R
            assert run.sweep(cfg.theta) == 0
        if policy == "main":
            want = RD.desired_loads(run.R, N)
            exc = [l - w for l, w in zip(sh.loads(), want)]
            assert max(exc) < B or -min(exc) < B
