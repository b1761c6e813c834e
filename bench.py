"""Benchmark of the population-annealing step on one GB300 (or N independent
replicas under torchrun).

One "step" is one full PA step over the whole population: reweight (Eq. 3/4
tau table), resample (nearest-integer copy counts, lookback scan, gather of
exact copies), theta = 10 checkerboard Metropolis sweeps, measurement.
Workload: 2D Ising L = 64 (bit-packed), R0 = 2^21 replicas (two 1 GiB
population buffers, far above the 129 MB L2), beta 0 -> 1 in 400 steps.
The timed steps are steps W+1 .. W+K of that schedule.

value     = spin-flip attempts per ns over the whole step (device time, CUDA
            events on the run's stream, graph-replayed steps).
e2e       = the same metric through the C ABI with host buffers: every step
            uploads the population from pinned host memory (pa_load), steps,
            and downloads it again (pa_dump_range) with the observables.
roofline  = the sweep kernel (dominant), integer-ALU bound.
cpu_baseline = the CPU oracle (single thread) on a bounded slice.
--impl reference: the CPU oracle alone, as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("spin-flip attempts/ns + resampled replicas/s at R0=2^21; batched vs plain, 1 GB300")
UNIT = "spin-flip attempts/ns"
WORKLOAD = dict(dim=2, L=64, R0=1 << 21, K=400, theta=10, beta0=0.0, beta_max=1.0, seed=3)
# Algorithmic integer work of one Metropolis attempt, in 32-bit integer
# operations (a three-input logic op counts one, a 32x32 -> 64 multiply two:
# its high and low products):
#   Philox4x32-10, 10 rounds x (2 multiplies = 4 + 2 three-input xors = 2)
#     = 60 per block of 4 uniforms                                    -> 15.0
#   acceptance: select the class threshold, compare, merge the bit     ->  3.0
#   lattice: bit-sliced unsatisfied-bond count and class masks, ~48 word
#     operations per 32 sites of one colour in a 64-site row          ->  1.5
OPS_PER_ATTEMPT = 19.5
# Integer issue peak: per SM and clock, 64 lanes on the ALU pipe plus 64 on
# the FMA-heavy pipe (integer multiply-add), 152 SMs, 2070 MHz maximum clock.
ALU_PEAK_TOPS = 152 * 128 * 2.070e9 / 1e12
# DRAM bytes of one sweep launch, from the ncu capture of the same kernel at
# 2^18 replicas (profiles/k_sweep_l64_ising2d_L64_R2p18.md: 210.2 MB), scaled
# by the replica count to 2^21.  None whenever the kernel changes.
SWEEP_TRAFFIC_BYTES_2P21 = 210.2e6 * 8


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampler running while the timed region runs."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.result = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        if not self.proc:
            return
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], [], set()
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                "sw_power_cap"), f[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if sm:
            self.result = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                           "reasons": sorted(reasons), "samples": len(sm)}


def oracle_rate(seconds: float, L=64, R0=512, theta=10):
    """Single-threaded oracle on a slice of the workload: attempts/ns and
    resampled replicas/s (one thread)."""
    from oracle import oracle as O
    cfg = O.make_config(dim=2, L=L, R0=R0, K=WORKLOAD["K"], theta=theta, seed=WORKLOAD["seed"])
    run = O.Run(cfg)
    attempts, t_sweep, t_res, resampled, steps = 0, 0.0, 0.0, 0, 0
    t_end = time.perf_counter() + seconds
    while time.perf_counter() < t_end and steps < cfg.K:
        R_prev = run.R
        t0 = time.perf_counter()
        assert run.resample() == 0
        t1 = time.perf_counter()
        assert run.sweep(theta) == 0
        t2 = time.perf_counter()
        attempts += run.R * L * L * theta
        resampled += R_prev
        t_res += t1 - t0
        t_sweep += t2 - t1
        steps += 1
    total = t_res + t_sweep
    return {"attempts_per_ns": attempts / total / 1e9, "steps": steps, "R0": R0,
            "seconds": total, "resampled_replicas_per_s": resampled / t_res if t_res else None}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    L, R0, theta = WORKLOAD["L"], 256, WORKLOAD["theta"]
    cfg = O.make_config(dim=2, L=L, R0=R0, K=WORKLOAD["K"], theta=theta, seed=WORKLOAD["seed"])
    run = O.Run(cfg)
    for _ in range(args.warmup):
        assert run.step() == 0
    attempts = 0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        assert run.step() == 0
        attempts += run.R * L * L * theta
    dt = time.perf_counter() - t0
    v = attempts / dt / 1e9
    sample = (f"oracle PA steps of L=64, R0={R0} (the 2^21-replica workload scaled down), "
              f"theta={theta}, steps {args.warmup + 1}..{args.warmup + args.steps} of K=400")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
            "data": "synthetic", "config": {"workload": sample},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--R0", type=int, default=WORKLOAD["R0"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2006_00561_gb300 import pa as P

    wl = dict(WORKLOAD, R0=args.R0)
    # replicas only: every rank runs its own independent population
    cfg = P.make_config(layout=P.LAYOUT_PACKED, instance_id=rank, **wl)
    stream = torch.cuda.Stream()
    run = P.Run(cfg, stream=stream)
    N = wl["L"] ** 2
    theta = wl["theta"]
    assert args.warmup + 2 * args.steps + (0 if args.no_e2e else args.steps) <= wl["K"]

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # warm-up (also captures the graph of one step)
    run.run_steps(args.warmup)
    run.observables()

    # ---- timed region 1: graph-replayed steps (the headline) --------------
    first = run.state()["step"] + 1
    barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        run.run_steps(args.steps)
        ev1.record(stream)
        barrier()
    ms_graph = ev0.elapsed_time(ev1)
    hist = run.history(first - 1, args.steps + 1)
    Rs = [h["R"] for h in hist]
    attempts = sum(Rs[1:]) * N * theta
    resampled = sum(Rs[:-1])
    if dist is not None:
        t = torch.tensor([ms_graph, attempts], dtype=torch.float64, device="cuda")
        ts = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(ts, t)
        ms_graph = max(float(x[0]) for x in ts)
        attempts_all = sum(float(x[1]) for x in ts)
    else:
        attempts_all = attempts
    value = attempts_all / (ms_graph * 1e6)
    run.observables()  # raises on a sticky device error

    # ---- timed region 2: plain launches with per-kernel events -------------
    P.pa_profile(run.h, True)
    P.pa_profile_read(run.h, reset=True)
    first2 = run.state()["step"] + 1
    barrier()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        run.step()
    e3.record(stream)
    barrier()
    ms_plain = e2.elapsed_time(e3)
    prof = P.pa_profile_read(run.h, reset=True)
    P.pa_profile(run.h, False)
    hist2 = run.history(first2 - 1, args.steps + 1)
    Rs2 = [h["R"] for h in hist2]
    attempts2 = sum(Rs2[1:]) * N * theta
    resampled2 = sum(Rs2[:-1])
    value_plain = attempts2 / (ms_plain * 1e6)
    n_sw, ms_sw = prof["sweep"]
    sweep_ms = ms_sw / max(n_sw, 1)
    res_ms = (prof["tau"][1] + prof["resample"][1]) / max(prof["resample"][0], 1)
    sweep_attempts_per_launch = attempts2 / max(n_sw, 1)
    achieved_tops = OPS_PER_ATTEMPT * sweep_attempts_per_launch / (sweep_ms * 1e-3) / 1e12
    resampled_per_s = resampled2 / ((prof["tau"][1] + prof["resample"][1]) * 1e-3)
    # resample traffic per input replica (bytes): ebin read 4, counts/offsets
    # write 8, source spins+ebin+mag read once per surviving replica, output
    # spins + ebin + mag written once per slot
    stride = run.state()["stride"]
    R_in = resampled2 / args.steps
    R_out = sum(Rs2[1:]) / args.steps
    res_bytes = R_in * 12 + R_in * (stride + 8) * 0.75 + R_out * (stride + 8)
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6778.0)
    res_gbs = res_bytes / (res_ms * 1e-3) / 1e9

    # ---- e2e: host buffers through the C ABI -------------------------------
    e2e = None
    if not args.no_e2e:
        R_now = run.state()["R"]
        cap = run.state()["capacity"]
        host = torch.empty(cap * stride, dtype=torch.uint8, pin_memory=True)
        hv = host.numpy()
        got = run.dump_range(P.DUMP_SPINS_RAW, 0, R_now)
        hv[: got.size] = got.reshape(-1)
        barrier()
        t0 = time.perf_counter()
        h2d = d2h = 0
        e2e_attempts = 0
        for _ in range(args.steps):
            P.pa_load_ptr(run.h, P.DUMP_SPINS_RAW, host.data_ptr(), R_now, R_now * stride)
            h2d += R_now * stride
            run.step()
            o = run.observables()
            R_now = o["R"]
            e2e_attempts += R_now * N * theta
            buf = P.lib()
            rc = buf.pa_dump_range(P.C.c_void_p(run.h), P.DUMP_SPINS_RAW, 0, R_now,
                                   P.C.c_void_p(host.data_ptr()), host.numel())
            assert rc == 0
            d2h += R_now * stride + 104
        barrier()
        dt = time.perf_counter() - t0
        if dist is not None:
            t = torch.tensor([dt, e2e_attempts], dtype=torch.float64, device="cuda")
            ts = [torch.zeros_like(t) for _ in range(world)]
            dist.all_gather(ts, t)
            dt = max(float(x[0]) for x in ts)
            e2e_attempts = sum(float(x[1]) for x in ts)
        e2e = {"value": e2e_attempts / (dt * 1e9), "unit": UNIT,
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
               "path": "pa_load(pinned host population) + pa_step + pa_observables + "
                       "pa_dump_range(pinned host) every step"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    cpu = None
    if world == 1 and args.cpu_seconds > 0:
        r = oracle_rate(args.cpu_seconds)
        cpu = {"value": r["attempts_per_ns"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{r['steps']} full PA steps of the oracle at L=64, R0={r['R0']} "
                         f"(theta=10), {r['seconds']:.1f} s, one thread",
               "resampled_replicas_per_s": r["resampled_replicas_per_s"]}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_graph / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": f"2D Ising L=64 bit-packed, R0=2^21 ({wl['R0']}), beta 0->1 in "
                               f"K=400 steps, theta=10, steps {first}..{first + args.steps - 1}",
                   "l2": "population 2 x 1 GiB, larger than L2 (no flush needed)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "resampled_replicas_per_s": resampled_per_s,
        "plain": {"value": value_plain, "ms_per_step": ms_plain / args.steps,
                  "note": "one launch per kernel per step, kernel events on"},
        "batched": {"value": value, "ms_per_step": ms_graph / args.steps,
                    "note": "one CUDA graph per step (pa_run_steps)"},
        "kernels_ms_per_step": {k: (v[1] / max(v[0], 1)) for k, v in prof.items()},
        "sweep_attempts_per_ns_kernel": sweep_attempts_per_launch / (sweep_ms * 1e6),
        "roofline": {"bound": "alu", "achieved": achieved_tops, "peak": ALU_PEAK_TOPS,
                     "unit": "Tops/s (32-bit int)", "frac": achieved_tops / ALU_PEAK_TOPS,
                     "traffic": SWEEP_TRAFFIC_BYTES_2P21 if wl["R0"] == 1 << 21 else None,
                     "traffic_note": "ncu dram bytes at 2^18 replicas x 8 (profiles/)",
                     "kernel": "k_sweep_l64 (theta=10 sweeps + measurement)",
                     "ops_per_attempt": OPS_PER_ATTEMPT,
                     "peak_note": "152 SMs x (64 ALU + 64 FMA-heavy) int32 lanes x 2070 MHz "
                                  "(derived from unit counts and the maximum clock)"},
        "resample_roofline": {"bound": "hbm", "achieved": res_gbs, "peak": hbm, "unit": "GB/s",
                              "frac": res_gbs / hbm, "traffic": None,
                              "bytes_per_step": res_bytes,
                              "peak_note": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
        "gpu_launches": 4 * args.steps * (3 if e2e else 2) + (args.steps if e2e else 0),
        "clocks": clk.result,
    }
    if e2e:
        line["e2e"] = e2e
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
