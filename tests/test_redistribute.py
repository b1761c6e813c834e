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


# ---------------------------------------------------------------------------
# the exchange as a slot order (shards = consecutive slot ranges)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("policy", ["main", "naive", "independent", "main_largest"])
def test_exchange_segments_permute_the_slots_into_the_planned_loads(policy):
    rng = np.random.default_rng(5)
    for _ in range(100):
        N = int(rng.integers(2, 12))
        loads = [int(x) for x in rng.integers(0, 3000, size=N)]
        bounds = RD.bounds_from_loads(loads)
        moves = RD.plan_moves(loads, policy, block=64, maxexc=1)
        segs, newb = RD.exchange_segments(bounds, moves)
        perm = np.concatenate([np.arange(a, a + k) for a, k in segs]) if segs else np.zeros(0, int)
        assert np.array_equal(np.sort(perm), np.arange(bounds[-1]))  # a permutation
        cur = list(loads)
        for s, d, k in moves:
            cur[s] -= k
            cur[d] += k
        assert np.diff(newb).tolist() == cur
        # a slot of shard n's new range came from shard n or from a shard that
        # sent to n; replicas that stayed keep their order, in front
        old_shard = np.repeat(np.arange(N), loads)
        senders = {n: {s for s, d, _ in moves if d == n} for n in range(N)}
        for n in range(N):
            got = old_shard[perm[newb[n]:newb[n + 1]]]
            assert set(got.tolist()) <= {n} | senders[n]
            own = perm[newb[n]:newb[n + 1]][got == n]
            assert np.all(np.diff(own) == 1) and (own.size == 0 or own[0] == bounds[n])


def test_oracle_permute_moves_whole_replicas():
    """or_permute (the oracle's exchange) against numpy indexing: states,
    levels and magnetisations move with their slot; the tracked energies move
    too (the from-scratch check after the next measurement stays clean), and
    the histogram is that of the resampled population."""
    cfg = O.make_config(dim=2, L=8, R0=300, K=10, theta=2, beta_max=1.0, seed=5)
    run = O.Run(cfg)
    for _ in range(2):
        assert run.step() == 0
    assert run.resample() == 0
    R = run.R
    s0, e0, m0 = run.spins(), run.ebin(), run.mag()
    cuts = sorted({0, R, *np.random.default_rng(1).integers(1, R, size=6).tolist()})
    pieces = [(a, b - a) for a, b in zip(cuts[:-1], cuts[1:])]
    segs = pieces[::-1]
    perm = np.concatenate([np.arange(a, a + k) for a, k in segs])
    assert run.permute(segs) == 0
    assert np.array_equal(run.spins(), s0[perm])
    assert np.array_equal(run.ebin(), e0[perm]) and np.array_equal(run.mag(), m0[perm])
    assert run.sweep(0) == 0
    assert np.array_equal(run.hist(), np.bincount(e0, minlength=run.bins))
    assert run.check_failures == 0
    assert run.permute([(0, R - 1)]) == -1 and run.permute([(1, R)]) == -1


@pytest.mark.parametrize("policy", ["main", "naive"])
def test_oracle_exchange_keeps_every_replica_in_its_planned_shard(policy):
    """Explicit per-replica shard labels carried through the oracle's real
    resamples and exchanges: after every exchange the labels are shard-major
    (shard n holds slots [bounds[n], bounds[n+1])), every replica that changed
    shard came from a sender of the plan, and the population is the oracle's
    own (no replica lost or duplicated beyond the resample's copies)."""
    cfg = O.make_config(dim=2, L=8, R0=4000, K=30, theta=2, beta_max=2.0, seed=78)
    run = O.Run(cfg)
    N, B = 4, 64
    bounds = RD.bounds_from_loads(RD.desired_loads(run.R, N))
    labels = np.repeat(np.arange(N), np.diff(bounds))
    for _ in range(cfg.K):
        assert run.resample() == 0
        labels = np.repeat(labels, run.counts())
        after = [int(run.offsets()[b]) if b < run.R_prev else run.R for b in bounds]
        assert np.array_equal(labels, np.repeat(np.arange(N), np.diff(after)))
        loads = np.diff(after).tolist()
        moves = RD.plan_moves(loads, policy, block=B)
        segs, bounds = RD.exchange_segments(after, moves)
        perm = np.concatenate([np.arange(a, a + k) for a, k in segs])
        assert run.permute(segs) == 0
        moved = labels[perm]
        for n in range(N):
            came = set(moved[bounds[n]:bounds[n + 1]].tolist())
            assert came <= {n} | {s for s, d, _ in moves if d == n}
        labels = np.repeat(np.arange(N), np.diff(bounds))
        assert run.sweep(cfg.theta) == 0 and run.check_failures == 0
    if policy == "main":
        want = RD.desired_loads(run.R, N)
        exc = [b - a - w for a, b, w in zip(bounds[:-1], bounds[1:], want)]
        assert max(exc) < B or -min(exc) < B
