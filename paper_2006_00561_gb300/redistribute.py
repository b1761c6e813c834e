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


# ---------------------------------------------------------------------------
# physical exchange: shards as consecutive slot ranges of the device population
# ---------------------------------------------------------------------------
def bounds_from_loads(loads: list) -> list:
    b = [0]
    for w in loads:
        b.append(b[-1] + int(w))
    return b


def exchange_segments(bounds: list, moves: list) -> tuple:
    """Slot order after an exchange between shards that are consecutive slot
    ranges (shard n = [bounds[n], bounds[n+1])).  moves: (src, dst, count)
    transfers (a block move of the main algorithm is (s, d, block)).  Every
    shard keeps the head of its range and gives away its tail, split among its
    destinations in increasing destination order; a shard's new range is its
    kept head followed by what it receives, in increasing source order.
    Returns (segments [(first old slot, length)] in new slot order, adjacent
    ones merged; new bounds)."""
    N = len(bounds) - 1
    flow = {}
    for s, d, k in moves:
        if k:
            flow[(s, d)] = flow.get((s, d), 0) + int(k)
    out = [sum(k for (a, _), k in flow.items() if a == n) for n in range(N)]
    tail = {}
    for s in range(N):
        at = bounds[s + 1] - out[s]
        if at < bounds[s]:
            raise ValueError(f"shard {s} gives more than it holds")
        for d in sorted(d for (a, d) in flow if a == s):
            tail[(s, d)] = at
            at += flow[(s, d)]
    segs, newb = [], [0]
    for n in range(N):
        parts = [(bounds[n], bounds[n + 1] - out[n] - bounds[n])]
        parts += [(tail[(s, n)], flow[(s, n)]) for s in sorted(a for (a, d) in flow if d == n)]
        for a, k in parts:
            if k <= 0:
                continue
            if segs and segs[-1][0] + segs[-1][1] == a:
                segs[-1] = (segs[-1][0], segs[-1][1] + k)
            else:
                segs.append((a, k))
        newb.append(newb[-1] + sum(k for _, k in parts))
    return segs, newb


def plan_moves(loads: list, policy: str, block: int = 1024, maxexc: int = 1,
               alpha: float = 0.5) -> list:
    """(src, dst, count) transfers of a policy for the given shard loads."""
    if policy in ("main", "main_largest"):
        match = "order" if policy == "main" else "largest"
        return [(s, d, block) for s, d in plan_main(loads, block, maxexc, match)]
    if policy == "naive":
        return plan_naive(loads, alpha)
    if policy == "independent":
        return []
    raise ValueError(policy)


def exchange_step(run, bounds: list, policy: str, block: int = 1024, maxexc: int = 1,
                  alpha: float = 0.5) -> dict:
    """One resample of `run` with the exchange executed on the device: the
    counts and scan (pa_resample_begin), the shards' offspring ranges read
    back, the policy's plan, then the gather into the exchanged slot order
    (pa_resample_finish), which moves every replica to its new shard.  Shard n
    holds slots [bounds[n], bounds[n+1]) before and the returned "bounds"
    after.  The sweeps are left to the caller."""
    from . import pa as P
    run.resample_begin()
    st = run.state()
    offsets = run.dump(P.DUMP_OFFSETS)
    R_prev, R_new = offsets.size, st["R"]
    after = [int(offsets[b]) if b < R_prev else R_new for b in bounds]
    loads = [after[n + 1] - after[n] for n in range(len(bounds) - 1)]
    moves = plan_moves(loads, policy, block, maxexc, alpha)
    segs, newb = exchange_segments(after, moves)
    run.resample_finish(segs)
    return {"bounds": newb, "loads_before": loads, "moves": moves, "segments": segs,
            "offspring_bounds": after}


def run_physical(run, K: int, N: int, policy: str, block: int = 1024, maxexc: int = 1,
                 alpha: float = 0.5, theta: int | None = None) -> dict:
    """Anneals `run` for K steps with the replicas exchanged on the device
    after every resample.  Per step: the largest shard load, the replicas and
    messages moved (a main block is one message, a naive replica one), and the
    messages and replicas each shard sends or receives."""
    theta = run.cfg.theta if theta is None else theta
    bounds = bounds_from_loads(desired_loads(run.state()["R"], N))
    rec = {"max": [], "moved": [], "shard_msgs": [], "shard_replicas": []}
    for _ in range(K):
        x = exchange_step(run, bounds, policy, block, maxexc, alpha)
        bounds = x["bounds"]
        loads = [bounds[n + 1] - bounds[n] for n in range(N)]
        msgs, reps = [0] * N, [0] * N
        for s, d, k in x["moves"]:
            m = 1 if policy.startswith("main") else k
            for n in (s, d):
                msgs[n] += m
                reps[n] += k
        rec["max"].append(max(loads))
        rec["moved"].append(sum(k for _, _, k in x["moves"]))
        rec["shard_msgs"].append(max(msgs) if msgs else 0)
        rec["shard_replicas"].append(max(reps) if reps else 0)
        run.sweep(theta)
    rec["bounds"] = bounds
    return rec


# Time model of the paper's setting (Sec. 3 and 4, one V100 per GPU): per step
# the slowest GPU's sweeps, plus the exchange, costed per shard as messages x
# latency + bytes / bandwidth (the busiest shard sets the time).  Constants:
#   sweep of one L = 64 replica: 5.3 us, from the paper's one-V100 runs at
#     theta = 1 and 10 (the difference of their run times over the extra
#     sweeps);
#   message latency: 70 us per MPI message of GPU memory between nodes (not
#     printed in the paper; fitted: on the paper's workload, 8 shards x 20 480
#     replicas, seed 2006, the modeled naive / main ratio at theta = 1 equals
#     the paper's 1.45 at 68 us, see exchange_latency_for_ratio);
#   bandwidth: 10 GB/s between nodes; 4096 bytes per replica (one byte per spin
#     of the single-spin coding at L = 64).
SWEEP_S_PER_REPLICA = 5.3e-6
LATENCY_S = 70e-6
BANDWIDTH_BPS = 10e9
BYTES_PER_REPLICA = 4096


def modeled_time(rec: dict, theta: int, latency_s: float = LATENCY_S,
                 sweep_s: float = SWEEP_S_PER_REPLICA, bandwidth: float = BANDWIDTH_BPS,
                 replica_bytes: int = BYTES_PER_REPLICA) -> float:
    """Seconds of a run in the time model above, from run_physical's record."""
    t = 0.0
    for mx, msgs, reps in zip(rec["max"], rec["shard_msgs"], rec["shard_replicas"]):
        t += mx * theta * sweep_s + msgs * latency_s + reps * replica_bytes / bandwidth
    return t


def exchange_latency_for_ratio(naive: dict, main: dict, theta: int, ratio: float) -> float:
    """The message latency at which the modeled naive / main run-time ratio
    equals `ratio` (the model is linear in the latency)."""
    a0 = modeled_time(naive, theta, 0.0)
    b0 = modeled_time(main, theta, 0.0)
    a1 = sum(naive["shard_msgs"])
    b1 = sum(main["shard_msgs"])
    den = a1 - ratio * b1
    return (ratio * b0 - a0) / den if den else float("nan")


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
    ap.add_argument("--physical", action="store_true",
                    help="move the replicas on the device (one fresh run per policy) and "
                         "report the time model of the paper's setting")
    a = ap.parse_args(argv)
    R0 = a.shards * a.per_shard
    if a.physical:
        return main_physical(a, R0)
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


def main_physical(a, R0: int) -> dict:
    """Each policy on its own fresh run (same seed), replicas exchanged on the
    device after every resample.  Reports per policy the peak shard load, the
    replicas and messages moved, the device time of the resamples with their
    exchanges, and the modeled run time of the paper's setting; then the
    modeled naive / main ratio and the message latency at which it equals the
    paper's 1.45 (Sec. 3, Fig. 2, theta = 1)."""
    import json
    import time

    import torch

    from . import pa as P
    out = {"shards": a.shards, "per_shard": a.per_shard, "L": a.L, "K": a.K, "theta": a.theta,
           "block": a.block, "maxexc": a.maxexc, "alpha": a.alpha, "seed": a.seed,
           "model": {"sweep_s_per_replica": SWEEP_S_PER_REPLICA, "latency_s": LATENCY_S,
                     "bandwidth_Bps": BANDWIDTH_BPS, "bytes_per_replica": BYTES_PER_REPLICA}}
    recs = {}
    for policy in ("independent", "naive", "main"):
        run = P.Run(P.make_config(dim=2, L=a.L, layout=P.LAYOUT_PACKED, R0=R0, K=a.K,
                                  theta=a.theta, beta_max=1.0, seed=a.seed))
        P.pa_profile(run.h, True)
        P.pa_profile_read(run.h, reset=True)
        t0 = time.perf_counter()
        rec = run_physical(run, a.K, a.shards, policy, a.block, a.maxexc, a.alpha)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        prof = P.pa_profile_read(run.h, reset=True)
        lnZ = run.observables()["lnZ"]
        run.close()
        recs[policy] = rec
        m = np.array(rec["max"])
        out[policy] = {"peak_load": int(m.max()), "peak_step": int(m.argmax()) + 1,
                       "peak_over_desired": float(m.max() / a.per_shard),
                       "replicas_moved": int(sum(rec["moved"])),
                       "device_resample_exchange_ms_per_step": prof["resample"][1] / a.K,
                       "wall_s": wall, "lnZ_final": lnZ,
                       "modeled_s": {"theta_1": modeled_time(rec, 1),
                                     f"theta_{a.theta}": modeled_time(rec, a.theta)}}
    for t in (1, a.theta):
        k = f"theta_{t}"
        out[f"naive_over_main_{k}"] = modeled_time(recs["naive"], t) / modeled_time(recs["main"], t)
        out[f"independent_over_main_{k}"] = (modeled_time(recs["independent"], t) /
                                              modeled_time(recs["main"], t))
    out["latency_for_paper_ratio_1p45_theta_1_s"] = exchange_latency_for_ratio(
        recs["naive"], recs["main"], 1, 1.45)
    out["messages"] = {p: int(sum(recs[p]["shard_msgs"])) for p in recs}
    print(json.dumps(out))
    return out


if __name__ == "__main__":
    main()
