"""Replica redistribution between GPUs (Sec. 3 of the paper), on virtual shards.

The paper splits the population over N GPUs.  After every resampling step each
GPU holds the offspring of its own replicas, and an exchange restores a
balanced load before the Metropolis sweeps.  Here the population lives on one
GPU, so the N GPUs are virtual shards: each shard owns a set of slots of the
population.  After a resample, slot interval [a, b) of the old population maps
to [o_a, o_b) of the new one (copies of contiguous replicas are contiguous), so
the per-shard offspring counts are exact.  A policy then moves replicas between
shards.  The physics does not change (the sweeps touch every replica
whichever shard owns it); what is measured is the load of each shard, the
largest one per step (the slowest GPU sets a step's time), and the replicas
moved.

Policies:
  * independent -- no exchange; only the global normaliser is shared (the
    first variant of Sec. 3, which the paper rejects for load imbalance);
  * main        -- the paper's block algorithm: blocks of `block` replicas
    (1024 in the paper), desired load r_n = R / N, a shard with excess
    maxg_n = load - r_n of at least `maxexc` blocks gives blocks to shards
    with a shortage minl_n = r_n - load of at least `maxexc` blocks;
  * naive       -- per-replica exchange in proportion to the offspring
    surplus: every shard above the desired load gives a fraction `alpha` of
    its surplus, shards below it take in proportion to their shortage.
Readings (the paper leaves them open): the main algorithm matches surplus
blocks to deficit blocks greedily in shard order (the lowest-indexed shard with
a qualifying excess gives to the lowest-indexed shard with a qualifying
shortage, a block at a time); `main_largest` is the alternative reading that
always moves from the largest excess to the largest shortage.  The naive rule
is the proportional partial exchange above with alpha = 1/2.
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------------------
# interval bookkeeping (pure host logic)
# ---------------------------------------------------------------------------
def map_intervals(intervals: list, offsets: np.ndarray, R_new: int) -> list:
    """New slot intervals of a shard's offspring: [a, b) -> [o_a, o_b)."""
    out = []
    R_old = offsets.size
    for a, b in intervals:
        oa = int(offsets[a]) if a < R_old else R_new
        ob = int(offsets[b]) if b < R_old else R_new
        if ob > oa:
            if out and out[-1][1] == oa:
                out[-1] = (out[-1][0], ob)
            else:
                out.append((oa, ob))
    return out


def load(intervals: list) -> int:
    return sum(b - a for a, b in intervals)


def take_from_end(intervals: list, n: int):
    """Removes n slots from the end of a shard's intervals; returns (kept, taken)."""
    kept = list(intervals)
    taken = []
    while n > 0 and kept:
        a, b = kept[-1]
        k = min(n, b - a)
        kept[-1] = (a, b - k)
        taken.append((b - k, b))
        if kept[-1][0] == kept[-1][1]:
            kept.pop()
        n -= k
    taken.reverse()
    return kept, taken


def desired_loads(R: int, N: int) -> list:
    base, rem = divmod(R, N)
    return [base + (1 if n < rem else 0) for n in range(N)]


def plan_main(loads: list, block: int = 1024, maxexc: int = 1, match: str = "order") -> list:
    """Block moves (src, dst) of the main algorithm for the given loads.  A shard
    gives while its excess maxg_n is at least `maxexc` blocks (and it holds a
    block), and takes while its shortage minl_n is at least `maxexc` blocks.
    match = "order": surplus and deficit shards are paired in shard order;
    match = "largest": each block goes from the largest excess to the largest
    shortage."""
    N = len(loads)
    cur = list(loads)
    want = desired_loads(sum(loads), N)
    moves = []
    if match == "order":
        src, dst = 0, 0
        while src < N and dst < N:
            if cur[src] - want[src] < maxexc * block or cur[src] < block:
                src += 1
            elif want[dst] - cur[dst] < maxexc * block:
                dst += 1
            else:
                cur[src] -= block
                cur[dst] += block
                moves.append((src, dst))
        return moves
    if match != "largest":
        raise ValueError(match)
    while True:
        exc = [cur[n] - want[n] for n in range(N)]
        src = max(range(N), key=lambda n: (exc[n], -n))
        dst = min(range(N), key=lambda n: (exc[n], n))
        if exc[src] < maxexc * block or -exc[dst] < maxexc * block or cur[src] < block:
            break
        cur[src] -= block
        cur[dst] += block
        moves.append((src, dst))
    return moves


def plan_naive(loads: list, alpha: float = 0.5) -> list:
    """Per-replica transfers (src, dst, count) of the naive reading."""
    N = len(loads)
    want = desired_loads(sum(loads), N)
    give = [int(alpha * (loads[n] - want[n])) if loads[n] > want[n] else 0 for n in range(N)]
    short = [want[n] - loads[n] if loads[n] < want[n] else 0 for n in range(N)]
    pool, need = sum(give), sum(short)
    if pool == 0 or need == 0:
        return []
    # shortages take the pool in proportion, largest remainders first
    share = [pool * s // need for s in short]
    rest = pool - sum(share)
    for n in sorted(range(N), key=lambda n: (-(pool * short[n] % need), n))[:rest]:
        share[n] += 1
    moves = []
    si = [n for n in range(N) if give[n] > 0]
    di = [n for n in range(N) if share[n] > 0]
    gi, dj = 0, 0
    g = [give[n] for n in range(N)]
    h = [share[n] for n in range(N)]
    while gi < len(si) and dj < len(di):
        s, t = si[gi], di[dj]
        k = min(g[s], h[t])
        moves.append((s, t, k))
        g[s] -= k
        h[t] -= k
        if g[s] == 0:
            gi += 1
        if h[t] == 0:
            dj += 1
    return moves


class Shards:
    """Shard membership of a population, as slot intervals."""

    def __init__(self, R: int, N: int):
        self.N = N
        self.intervals = []
        start = 0
        for n, w in enumerate(desired_loads(R, N)):
            self.intervals.append([(start, start + w)] if w else [])
            start += w

    def loads(self) -> list:
        return [load(iv) for iv in self.intervals]

    def after_resample(self, offsets: np.ndarray, R_new: int):
        self.intervals = [map_intervals(iv, offsets, R_new) for iv in self.intervals]

    def move(self, src: int, dst: int, n: int):
        kept, taken = take_from_end(self.intervals[src], n)
        self.intervals[src] = kept
        self.intervals[dst] = sorted(self.intervals[dst] + taken)

    def redistribute(self, policy: str, block: int = 1024, maxexc: int = 1,
                     alpha: float = 0.5) -> int:
        """Applies a policy; returns the replicas moved."""
        moved = 0
        if policy in ("main", "main_largest"):
            match = "order" if policy == "main" else "largest"
            for s, d in plan_main(self.loads(), block, maxexc, match):
                self.move(s, d, block)
                moved += block
        elif policy == "naive":
            for s, d, k in plan_naive(self.loads(), alpha):
                self.move(s, d, k)
                moved += k
        elif policy != "independent":
            raise ValueError(policy)
        return moved


def run_sharded(run, K: int, N: int, policies=("independent", "naive", "main", "main_largest"),
                block=1024,
                maxexc=1, alpha=0.5, theta=None) -> dict:
    """Anneals `run` for K steps and follows every policy on the same sequence
    of resamples (the redistribution does not change the physics).  Returns
    per-step loads, the largest load per step and moved replicas, per policy."""
    from . import pa as P
    R = run.state()["R"]
    shards = {p: Shards(R, N) for p in policies}
    rec = {p: {"loads": [], "max": [], "moved": []} for p in policies}
    theta = run.cfg.theta if theta is None else theta
    for _ in range(K):
        run.resample()
        st = run.state()
        offsets = run.dump(P.DUMP_OFFSETS)
        for p in policies:
            sh = shards[p]
            sh.after_resample(offsets, st["R"])
            moved = sh.redistribute(p, block, maxexc, alpha)
            loads = sh.loads()
            assert sum(loads) == st["R"]
            rec[p]["loads"].append(loads)
            rec[p]["max"].append(max(loads))
            rec[p]["moved"].append(moved)
        run.sweep(theta)
    for p in policies:
        m = np.array(rec[p]["max"], dtype=np.float64)
        rec[p]["peak"] = int(m.max())
        rec[p]["sum_max"] = float(m.sum())
    return rec


def main(argv=None):
    """python -m paper_2006_00561_gb300.redistribute --shards 8 --per-shard 20480 ...
    The paper's workload (Sec. 3): 8 GPUs x 20 480 replicas of the 2D Ising
    model at L = 64, beta 0 -> 1 in 200 steps."""
    import argparse
    import json

    from . import pa as P
    ap = argparse.ArgumentParser()
    ap.add_argument("--shards", type=int, default=8)
    ap.add_argument("--per-shard", type=int, default=20480)
    ap.add_argument("--K", type=int, default=200)
    ap.add_argument("--theta", type=int, default=10)
    ap.add_argument("--L", type=int, default=64)
    ap.add_argument("--seed", type=int, default=2006)
    ap.add_argument("--maxexc", type=int, default=1)
    ap.add_argument("--block", type=int, default=1024)
    ap.add_argument("--alpha", type=float, default=0.5)
    ap.add_argument("--loads", action="store_true", help="include every step's shard loads")
    a = ap.parse_args(argv)
    R0 = a.shards * a.per_shard
    run = P.Run(P.make_config(dim=2, L=a.L, layout=P.LAYOUT_PACKED, R0=R0, K=a.K,
                              theta=a.theta, beta_max=1.0, seed=a.seed))
    rec = run_sharded(run, a.K, a.shards, block=a.block, maxexc=a.maxexc, alpha=a.alpha)
    ideal = sum(h["R"] for h in run.history(1, a.K)) / a.shards
    out = {"shards": a.shards, "per_shard": a.per_shard, "L": a.L, "K": a.K, "theta": a.theta,
           "block": a.block, "maxexc": a.maxexc, "alpha": a.alpha, "seed": a.seed}
    for p, r in rec.items():
        m = np.array(r["max"])
        out[p] = {"peak_load": int(m.max()), "peak_step": int(m.argmax()) + 1,
                  "peak_over_desired": float(m.max() / a.per_shard),
                  "time_vs_balanced": float(m.sum() / ideal),
                  "replicas_moved": int(sum(r["moved"]))}
        if a.loads:
            out[p]["max_per_step"] = [int(x) for x in m]
    for p in ("independent", "naive"):
        out[f"{p}_over_main_time"] = out[p]["time_vs_balanced"] / out["main"]["time_vs_balanced"]
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
