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
            uploads the population from pinned host memory (pa_load), steps
            with the new population copied back to that memory range by range
            while the later ranges sweep (pa_step_stream), and reads the
            observables.
roofline  = the sweep kernel (dominant), integer-ALU bound.
cpu_baseline = the CPU oracle (single thread) on a bounded slice.
next_items = Poisson resampling, adaptive temperature steps and checkpoints
            measured on the same workload (outside the headline timed region).
--impl reference: the CPU oracle alone, as the reference arm.
"""
from __future__ import annotations

import argparse
import gc
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
# 2^20 replicas, four times L2 (profiles/k_sweep_l64_ising2d_L64_R2p18.md:
# 538.5 MB read + 483.2 MB written), scaled by the replica count to 2^21.
# None whenever the kernel changes, until the next capture.
SWEEP_TRAFFIC_BYTES_2P21 = (538.521344e6 + 483.193344e6) * 2
# Slot ranges of the e2e step: each range's copy to the host (~0.7 ms at 1/8 of
# 1 GiB) runs while the next range sweeps (~7 ms).
E2E_CHUNKS = 8


def rank_workload(rank: int, R0: int) -> dict:
    """Replicas only: every rank runs an independent population of the same
    workload, separated by its instance id (the Philox counter's instance
    field), so no data-path collective is needed."""
    return dict(WORKLOAD, R0=R0, instance_id=rank)


def aggregate(dist, ms: float, work: float, device) -> tuple:
    """(max time over ranks, total work over ranks); plain values without a
    process group."""
    if dist is None:
        return ms, work
    import torch
    t = torch.tensor([ms, work], dtype=torch.float64, device=device)
    ts = [torch.zeros_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(ts, t)
    return max(float(x[0]) for x in ts), sum(float(x[1]) for x in ts)


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


def _oracle_worker(job):
    """One oracle process: full PA steps of the L = 64 workload at a small R0,
    for `seconds` or for warmup + steps steps.  Returns its counts and times."""
    seconds, warmup, steps, R0, seed = job
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    L, theta = WORKLOAD["L"], WORKLOAD["theta"]
    cfg = O.make_config(dim=2, L=L, R0=R0, K=WORKLOAD["K"], theta=theta, seed=seed)
    run = O.Run(cfg)
    for _ in range(warmup):
        assert run.step() == 0
    attempts, t_sweep, t_res, resampled, n = 0, 0.0, 0.0, 0, 0
    t_start = time.perf_counter()
    while n < cfg.K - warmup:
        if steps is not None and n >= steps:
            break
        if seconds is not None and time.perf_counter() - t_start >= seconds:
            break
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
        n += 1
    return {"attempts": attempts, "resampled": resampled, "t_res": t_res, "t_sweep": t_sweep,
            "steps": n, "wall": time.perf_counter() - t_start}


def oracle_rate(seconds: float = None, R0=512, procs: int = 1, warmup: int = 0, steps=None):
    """The oracle on a slice of the workload (L = 64, R0 small, theta = 10):
    `procs` independent single-threaded processes (spawned, different seeds),
    each for `seconds` or `steps` steps.  Returns attempts/ns and resampled
    replicas/s over the slowest process's wall time."""
    jobs = [(seconds, warmup, steps, R0, WORKLOAD["seed"] + 1000 * p) for p in range(procs)]
    if procs == 1:
        res = [_oracle_worker(jobs[0])]
        wall = res[0]["t_res"] + res[0]["t_sweep"]
    else:
        import multiprocessing as mp
        t0 = time.perf_counter()
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_oracle_worker, jobs)
        wall = max(r["wall"] for r in res)
        del t0
    att = sum(r["attempts"] for r in res)
    rs = sum(r["resampled"] for r in res)
    t_res = max(r["t_res"] for r in res)
    return {"attempts_per_ns": att / wall / 1e9, "steps": sum(r["steps"] for r in res),
            "R0": R0, "seconds": wall, "procs": procs,
            "resampled_replicas_per_s": rs / t_res if t_res else None}


def _ensemble_oracle_worker(job):
    """One oracle process on one config-4 instance (its L, couplings, seeds and
    schedule) at a small R0: full PA steps for `seconds`.  Returns (attempts,
    seconds)."""
    spec, seconds, R0 = job
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    sp = dict(spec)
    sp["R0"] = R0
    run = O.Run(O.make_config(**sp))
    attempts, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds and run.step_index < sp["K"]:
        assert run.step() == 0
        attempts += run.R * sp["L"] ** 3 * sp["theta"]
    return attempts, time.perf_counter() - t0


def ensemble_oracle_rate(procs: int, seconds: float = 4.0, R0: int = 256) -> dict:
    """The oracle on config 4: the first `procs` instances of the 256, one
    single-threaded process each (spawned), each running full PA steps at
    R0 = 256 for `seconds`; attempts/ns over the slowest process's wall time."""
    import multiprocessing as mp
    from paper_2006_00561_gb300 import workloads
    specs = workloads.ea_ensemble(256, seed=4)[:procs]
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_ensemble_oracle_worker, [(sp, seconds, R0) for sp in specs])
    wall = max(r[1] for r in res)
    return {"kind": "oracle", "cores": procs, "attempts_per_ns": sum(r[0] for r in res) / wall / 1e9,
            "sample": f"the first {procs} of the 256 instances (their L, couplings, seeds and "
                      f"schedule), one process each, full PA steps at R0={R0} for {seconds:.0f} s",
            "seconds": wall}


CONFIG1 = dict(dim=2, L=16, R0=1000, K=100, theta=10, beta0=0.0, beta_max=1.0, seed=1)


def _config1_oracle(seed):
    """One whole config-1 run of the oracle (2D L = 16 int8, R0 = 1000, beta
    0 -> 1 in 100 steps, theta = 10); returns (attempts, seconds, lnZ)."""
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    run = O.Run(O.make_config(**dict(CONFIG1, seed=seed)))
    t0 = time.perf_counter()
    att = 0
    for _ in range(CONFIG1["K"]):
        assert run.step() == 0
        att += run.R * 256 * CONFIG1["theta"]
    return att, time.perf_counter() - t0, run.lnZ


def config1_measure(P, procs: int) -> dict:
    """Config 1 in full: the whole run on the GPU (int8 layout, graph-replayed
    steps, device time) and on the oracle, one process and one per host core
    (different seeds; the seed-1 process is the GPU run's twin)."""
    import multiprocessing as mp

    import torch
    stream = torch.cuda.Stream()
    run = P.Run(P.make_config(layout=P.LAYOUT_INT8, **CONFIG1), stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    run.run_steps(CONFIG1["K"])  # one CUDA graph per step
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    hist = run.history(1, CONFIG1["K"])
    att = sum(h["R"] for h in hist) * 256 * CONFIG1["theta"]
    gpu_lnZ = run.observables()["lnZ"]
    run.close()
    a1, s1, o_lnZ = _config1_oracle(CONFIG1["seed"])
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_config1_oracle, [CONFIG1["seed"] + 1000 * k for k in range(procs)])
    wall = max(r[1] for r in res)
    return {"workload": "2D Ising L=16 int8, R0=1000, beta 0->1 in K=100 steps, theta=10, seed 1",
            "gpu_attempts_per_ns": att / (ms * 1e6), "gpu_run_ms": ms,
            "oracle_attempts_per_ns": a1 / s1 / 1e9, "oracle_run_s": s1,
            "oracle_procs": procs, "oracle_procs_attempts_per_ns": sum(r[0] for r in res) / wall / 1e9,
            "lnZ_gpu": gpu_lnZ, "lnZ_oracle": o_lnZ}


def config2_measure(P) -> dict:
    """Config 2 in full: 2D Ising L = 64 packed, R0 = 2^17, beta 0 -> 1 in 200
    steps, theta = 10, seed 2, every step graph-replayed; device time of the
    whole run (the paper's task at 6.4 times its per-GPU replica count)."""
    import torch
    stream = torch.cuda.Stream()
    run = P.Run(P.make_config(dim=2, L=64, layout=P.LAYOUT_PACKED, R0=1 << 17, K=200, theta=10,
                              beta_max=1.0, seed=2), stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    run.run_steps(200)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    hist = run.history(1, 200)
    att = sum(h["R"] for h in hist) * 4096 * 10
    o = run.observables()
    run.close()
    return {"workload": "2D Ising L=64 packed, R0=2^17, beta 0->1 in K=200 steps, theta=10, seed 2",
            "run_s": ms / 1e3, "attempts_per_ns": att / (ms * 1e6), "lnZ": o["lnZ"], "e": o["e"],
            "R_final": o["R"]}


def host_info() -> dict:
    import platform
    info = {"nproc": os.cpu_count(), "machine": platform.machine()}
    try:
        for line in open("/proc/cpuinfo"):
            k = line.split(":")[0].strip().lower()
            if k in ("model name", "cpu part", "cpu implementer"):
                info.setdefault(k.replace(" ", "_"), line.split(":", 1)[1].strip())
    except OSError:
        pass
    return info


def _ensemble_oracle_twin(job):
    """The oracle's run of one config-4 instance at its full size, for the
    steps the GPU arms take; returns its observables and a hash of its spins
    after the last step."""
    spec, steps = job
    sys.path.insert(0, ROOT)
    import hashlib
    from oracle import oracle as O
    run = O.Run(O.make_config(**spec))
    for _ in range(steps):
        assert run.step() == 0
    o = run.observables()
    return {"step": run.step_index, "R": o["R"], "sumE": o["sumE"], "lnZ": o["lnZ"],
            "spins_sha": hashlib.sha256(run.spins().tobytes()).hexdigest()[:16]}


def _spins_sha(run) -> str:
    import hashlib
    return hashlib.sha256(run.spins().tobytes()).hexdigest()[:16]


def ensemble_compare(P, steps: int, tune_cache=None, oracle_pool=None) -> dict:
    """Config 4: 256 +-J instances (L in {6,8,10}, R0 in {2^14..2^16}, beta
    0 -> 3, K = 150, theta = 10) stepped plain (four launches per run per step)
    and batched (one CUDA graph per step, autotuned sweep shapes).  Both arms
    start from fresh runs of the same seeds, take one untimed step, and time
    the same steps 2 .. steps + 1; throughput = attempts / device time.  The
    autotuner runs first on a throwaway copy of the ensemble, so its timed
    steps do not shift the batched arm's step range.  Parity: after the timed
    steps the sampled instances hold the same spins in both arms, and the
    smallest instance equals the oracle's run (started in `oracle_pool` before
    the GPU work).  Breakdown: device time per phase of two more batched steps
    (reweight, resample, sweep classes, observables)."""
    import torch
    from paper_2006_00561_gb300 import autotune, workloads
    specs = workloads.ea_ensemble(256, seed=4)
    stream = torch.cuda.Stream()
    out = {"workload": "256 3D +-J EA instances, L in {6,8,10}, R0 in {2^14,2^15,2^16}, "
                       "beta 0->3, K=150, theta=10 (numpy PCG64 seed 4)",
           "timed_steps": f"2..{steps + 1} in both arms"}
    sample = sorted({0, 37, 101, 163, 255} | {min(range(len(specs)),
                    key=lambda i: (specs[i]["L"] ** 3 * specs[i]["R0"], i))})
    twin = min(range(len(specs)), key=lambda i: (specs[i]["L"] ** 3 * specs[i]["R0"], i))
    twin_job = oracle_pool.apply_async(_ensemble_oracle_twin, ((specs[twin], steps + 1),)) \
        if oracle_pool is not None else None

    def attempts(runs, first, n):
        tot = 0
        for r, sp in zip(runs, specs):
            h = r.history(first, n)
            tot += sum(x["R"] for x in h) * sp["L"] ** 3 * sp["theta"]
        return tot

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # autotuner on a throwaway copy of the ensemble
    tmp = [P.Run(P.make_config(layout=P.LAYOUT_PACKED, **sp), stream=stream) for sp in specs]
    tb = P.Batch(tmp, stream=stream)
    tuned = autotune.tune(tb, steps_left=specs[0]["K"], cache_path=tune_cache)
    tb.close()
    for r in tmp:
        r.close()
    del tmp, tb
    torch.cuda.empty_cache()

    # plain arm
    plain = [P.Run(P.make_config(layout=P.LAYOUT_PACKED, **sp), stream=stream) for sp in specs]
    for r in plain:
        r.step()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        for r in plain:
            r.step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1)
    a_plain = attempts(plain, 2, steps)
    plain_sha = {i: _spins_sha(plain[i]) for i in sample}
    plain_obs = {i: plain[i].observables() for i in sample}
    for r in plain:
        r.close()
    del plain
    torch.cuda.empty_cache()

    # batched arm, with the tuned shapes
    runs = [P.Run(P.make_config(layout=P.LAYOUT_PACKED, **sp), stream=stream) for sp in specs]
    batch = P.Batch(runs, stream=stream)
    for ci, shape in tuned["shapes"].items():
        batch.set_shape(ci, shape[0], shape[1])
    batch.run_steps(1)  # also captures the step's graph
    assert batch.sync() == 0
    torch.cuda.synchronize()
    e0.record(stream)
    batch.run_steps(steps)
    e1.record(stream)
    assert batch.sync() == 0
    ms_b = e0.elapsed_time(e1)
    a_b = attempts(runs, 2, steps)
    same = all(_spins_sha(runs[i]) == plain_sha[i] and
               runs[i].observables()["lnZ"] == plain_obs[i]["lnZ"] for i in sample)
    twin_gpu = {"step": runs[twin].observables()["step"], "sha": _spins_sha(runs[twin]),
                "obs": runs[twin].observables()}
    # phase breakdown of two more (non-graph) batched steps
    batch.profile(True)
    batch.profile_read(reset=True)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(2):
        batch.step()
    t1.record(stream)
    prof = batch.profile_read(reset=True)
    batch.profile(False)
    assert batch.sync() == 0
    ms_two = t0.elapsed_time(t1)
    phases = {k: prof[k] / max(prof["steps"], 1) for k in ("reweight", "resample", "sweep", "obs")}
    step_ms = ms_two / 2
    out.update({
        "plain_attempts_per_ns": a_plain / (ms_plain * 1e6),
        "batched_attempts_per_ns": a_b / (ms_b * 1e6),
        "speedup": (a_b / ms_b) / (a_plain / ms_plain),
        "plain_ms_per_step": ms_plain / steps, "batched_ms_per_step": ms_b / steps,
        "launches_per_step": {"plain": 4 * len(specs), "batched": 3 + len(batch.classes())},
        "phase_ms_per_step": phases,
        "non_sweep_share": 1.0 - phases["sweep"] / step_ms,
        "autotune": {"shapes": {str(k): v for k, v in tuned["shapes"].items()},
                     "steps_used": tuned["steps_used"]},
        "parity": {"sampled_instances": sample, "batched_equals_plain": bool(same)},
        "replicas": sum(r.state()["R"] for r in runs),
    })
    if twin_job is not None:
        out["parity"]["oracle_instance"] = twin
        try:
            o = twin_job.get(timeout=600)
        except Exception as e:  # the comparison is reported, not allowed to end the bench
            out["parity"]["batched_equals_oracle"] = None
            out["parity"]["oracle_error"] = repr(e)[:200]
        else:
            g = twin_gpu["obs"]
            out["parity"]["batched_equals_oracle"] = bool(
                o["spins_sha"] == twin_gpu["sha"] and o["step"] == twin_gpu["step"] and
                o["R"] == g["R"] and o["sumE"] == g["sumE"] and
                abs(o["lnZ"] - g["lnZ"]) <= 1e-12 * abs(o["lnZ"]))
    batch.close()
    for r in runs:
        r.close()
    return out


def serving_measure(P, prefix: int = 24) -> dict:
    """Config 5: the first `prefix` requests of the 256-request trace (Poisson
    arrivals at 50 req/s, seed 5; the 7 (dim, L) classes, R0 = 2^12..2^18, K =
    100..300, beta_max in {1, 3}, theta = 10), served in real time under a
    64 GiB HBM budget twice: by the pipelined server (two quanta in flight,
    admission and batch building while the device runs) and by the
    synchronous one (the device idles during every host phase).  Then the
    miniature mix (R0 = 2^8..2^14, K = 25..75): at 400 req/s by both servers
    (short requests, so admissions and retirements come every few quanta) and
    at a sub-saturating 40 req/s by the pipelined one.  Reported per run:
    latency p50 / p99, offered and served attempts/ns, the GPU-idle fraction
    (device events between the first quantum's start and the last one's end
    for the pipelined server; one minus the host's waiting share of the wall
    time for the synchronous one)."""
    from paper_2006_00561_gb300 import serve, workloads
    full = workloads.serving_trace(256, rate=50.0, seed=5)
    trace = full[:prefix]
    offered = sum(t["R0"] * t["L"] ** t["dim"] * t["theta"] * t["K"] for t in trace)
    span = trace[-1]["arrival"]
    out = {"workload": f"the first {prefix} requests of the 256-request trace (50 req/s, seed "
                       "5; R0 2^12..2^18, K 100..300, theta 10), 64 GiB budget",
           "offered_attempts_per_ns": offered / (span * 1e9), "arrival_span_s": span}

    def summary(st):
        return {k: st.get(k) for k in ("served", "served_attempts_per_ns", "p50_latency_s",
                                       "p99_latency_s", "max_resident", "iterations", "wall_s",
                                       "gpu_idle_fraction", "gpu_idle_fraction_host_estimate",
                                       "device_busy_s", "device_attempts_per_ns") if k in st}
    for name, cls in (("pipelined", serve.PipelinedServer), ("sync", serve.Server)):
        srv = cls(hbm_budget=64 << 30, quantum=8)
        st = srv.run_trace([dict(t) for t in trace])
        out[name] = summary(st)
        if name == "sync":
            out[name]["host_phase_s"] = st["host_phase_s"]
        del srv
    # the miniature mix: many short requests, so admissions and retirements
    # come every few quanta; above capacity (400 req/s) both servers, below it
    # (40 req/s) the pipelined one
    for rate, kinds in ((400.0, (("pipelined", serve.PipelinedServer), ("sync", serve.Server))),
                        (40.0, (("pipelined", serve.PipelinedServer),))):
        mini = workloads.serving_trace(48, rate=rate, seed=5, R0_exp=(8, 14), K_range=(25, 75))
        off_mini = sum(t["R0"] * t["L"] ** t["dim"] * t["theta"] * t["K"] for t in mini)
        entry = {"offered_attempts_per_ns": off_mini / (mini[-1]["arrival"] * 1e9)}
        for name, cls in kinds:
            srv = cls(hbm_budget=8 << 30, quantum=4)
            entry[name] = summary(srv.run_trace([dict(t) for t in mini]))
            del srv
        out[f"miniature_{int(rate)}_per_s"] = entry
    return out


def next_items_measure(P, steps: int = 5, R0: int = WORKLOAD["R0"]) -> dict:
    """The extensions of the fixed-schedule path, each on the headline workload
    (2D Ising L = 64 packed, theta = 10, beta 0 -> 1 in 400 steps):
      poisson    -- Poisson copy counts (Sec. 2's draw): graph-replayed step rate
                    and resample time per step (kernel events);
      multinomial -- the same for multinomial resampling (cumulative-weight scan,
                    R0 draws, then the scan and gather);
      adaptive   -- adaptive temperature steps (overlap target 0.9): host time of
                    the decision (histogram read + bisection) and wall time of a
                    whole adaptive step (decision, resample, sweeps, synchronise);
      checkpoint -- pa_checkpoint / pa_restore of the whole run to and from
                    pageable host memory;
      host_link  -- pinned host <-> HBM copy bandwidth (the link e2e crosses)."""
    import torch
    wl = dict(WORKLOAD, R0=R0)
    N, theta = wl["L"] ** 2, wl["theta"]
    stream = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"workload": f"2D Ising L=64 packed, R0={R0}, theta=10, beta 0->1 in K=400"}

    for name, rule in (("multinomial", P.RESAMPLE_MULTINOMIAL), ("poisson", P.RESAMPLE_POISSON)):
        run = P.Run(P.make_config(layout=P.LAYOUT_PACKED, resample=rule, **wl), stream=stream)
        run.run_steps(3)
        run.observables()
        first = run.state()["step"] + 1
        torch.cuda.synchronize()
        e0.record(stream)
        run.run_steps(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        h = run.history(first - 1, steps + 1)
        att = sum(x["R"] for x in h[1:]) * N * theta
        P.pa_profile(run.h, True)
        P.pa_profile_read(run.h, reset=True)
        for _ in range(steps):
            run.step()
        prof = P.pa_profile_read(run.h, reset=True)
        P.pa_profile(run.h, False)
        run.observables()
        out[name] = {
            "attempts_per_ns": att / (ms * 1e6), "ms_per_step": ms / steps,
            "resample_ms": prof["resample"][1] / max(prof["resample"][0], 1),
            "k_tau_ms": prof["tau"][1] / max(prof["tau"][0], 1),
            "R_min_max": [min(x["R"] for x in h[1:]), max(x["R"] for x in h[1:])]}
        if name == "multinomial":
            run.close()

    t0 = time.perf_counter()
    blob = run.checkpoint()
    t1 = time.perf_counter()
    run.restore(blob)
    t2 = time.perf_counter()
    out["checkpoint"] = {"bytes": len(blob), "checkpoint_s": t1 - t0, "restore_s": t2 - t1,
                         "checkpoint_gbs": len(blob) / (t1 - t0) / 1e9,
                         "restore_gbs": len(blob) / (t2 - t1) / 1e9}
    del blob
    run.close()

    # the host link the e2e copies cross: 1 GiB each way between pinned host
    # memory and HBM, timed with events on one stream
    nbytes = 1 << 30
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    dev = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    link = {}
    for name, dst, src in (("h2d_gbs", dev, host), ("d2h_gbs", host, dev)):
        with torch.cuda.stream(stream):
            dst.copy_(src, non_blocking=True)  # warm-up
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(3):
                dst.copy_(src, non_blocking=True)
            e1.record(stream)
        torch.cuda.synchronize()
        link[name] = 3 * nbytes / (e0.elapsed_time(e1) * 1e-3) / 1e9
    out["host_link"] = link
    del host, dev

    run = P.Run(P.make_config(layout=P.LAYOUT_PACKED, **wl), stream=stream)
    run.run_steps(3)
    run.observables()
    dec, wall, betas = [], [], []
    for _ in range(steps):
        t0 = time.perf_counter()
        b = run.adaptive_beta(0.9, 1.0)
        t1 = time.perf_counter()
        run.resample_to(b)
        run.sweep(theta)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        dec.append((t1 - t0) * 1e3)
        wall.append((t2 - t0) * 1e3)
        betas.append(b)
    run.observables()
    out["adaptive"] = {"target": 0.9, "decision_ms": statistics.median(dec),
                       "step_wall_ms": statistics.median(wall),
                       "beta_first_last": [betas[0], betas[-1]],
                       "bins": P.pa_num_bins(2, 64)}
    run.close()
    return out


def arm_config(R0: int, first: int, steps: int, world: int) -> dict:
    """The workload both arms report (the reference arm runs a bounded slice of
    it, described in its cpu_baseline)."""
    return {"workload": f"2D Ising L=64 bit-packed, R0=2^21 ({R0}), beta 0->1 in K=400 steps, "
                        f"theta=10, steps {first}..{first + steps - 1}",
            "l2": "population 2 x 1 GiB, larger than L2 (no flush needed)",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}


def run_reference(args):
    """The reference arm: the oracle as it stands, one single-threaded process
    per host core, each running W + K full PA steps of the L = 64 workload at
    R0 = 256 (a bounded slice of the 2^21-replica run, different seeds)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    R0 = 256
    procs = os.cpu_count() or 1
    r = oracle_rate(R0=R0, procs=procs, warmup=args.warmup, steps=args.steps)
    v = r["attempts_per_ns"]
    sample = (f"{procs} oracle processes, each PA steps {args.warmup + 1}..{args.warmup + args.steps}"
              f" of the L=64 workload at R0={R0} (the 2^21-replica run scaled down), theta=10, "
              f"K=400, seeds 3 + 1000 p")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["seconds"] * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int8",
            "data": "synthetic",
            "config": arm_config(WORKLOAD["R0"], args.warmup + 1, args.steps,
                                 int(os.environ.get("WORLD_SIZE", "1"))),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
                             "sample": sample, "host": host_info()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def philox_ceiling(P, sweep_attempts_per_ns: float) -> dict:
    """The register kernels' generator alone (pa_bench_philox): the same
    Philox blocks with no acceptance tests and no lattice work, one 16-warp
    block per SM (its fastest shape; the sweep kernel runs 12 warps).  A sweep attempt consumes one uniform, so the sweep
    kernel's attempts/ns over this kernel's uniforms/ns is the fraction of the
    generator's own ceiling that the sweep reaches."""
    import torch
    n = P.pa_bench_philox_threads()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    halfsweeps, reps = 4000, 5
    for _ in range(2):
        P.pa_bench_philox(7, halfsweeps, out.data_ptr(), n, s.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    for _ in range(reps):
        P.pa_bench_philox(7, halfsweeps, out.data_ptr(), n, s.cuda_stream)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    uniforms = n * halfsweeps * 64
    rate = uniforms / (ms * 1e6)
    return {"kernel": "k_philox_rate", "uniforms_per_ns": rate, "ms_per_launch": ms,
            "uniforms_per_launch": uniforms, "sweep_fraction": sweep_attempts_per_ns / rate,
            "note": "Philox4x32-10 blocks of k_sweep_l64 (14 multiplies each), 1 block of "
                    "16 warps per SM, outputs xor-folded: the generator's ceiling"}


# (name, kind, 32-bit int ops per chain step, instructions per chain step):
# a three-input logic op or a 32-bit multiply-add counts one op, a 32 x 32 ->
# 64 multiply two (its high and low products)
INTOPS_KINDS = (("lop3", 0, 1, 1), ("imad", 1, 1, 1), ("mad_wide", 2, 2, 1),
                ("lop3+imad", 3, 1, 1), ("lop3+mad_wide", 4, 1.5, 1),
                ("mul_wide+xor", 5, 3, 2))
# Philox4x32-10 multiplies per attempt in the L = 64 sweep kernel: 14 of a
# block's 20 products are formed per block (the rest are shared by every
# block of a half-sweep, or formed once per run or per launch), and a block
# serves 4 attempts
MULTIPLIES_PER_ATTEMPT = 3.5


def int_peaks(P, iters: int = 20000, reps: int = 3) -> dict:
    """Integer throughput of this GPU, measured (pa_bench_intops): independent
    chains of one instruction kind on every resident thread of every SM, CUDA
    events on the launching stream.  Per kind: thread-instructions per second
    and 32-bit integer ops per second in the sweep's own counting (a
    three-input logic op or a 32-bit multiply-add is one op, a 32 x 32 -> 64
    multiply two).  The interleaved lop3 + mad.wide stream is the instruction
    mix of a Philox round, the bulk of the sweep kernel's work; its op rate is
    the peak the sweep roofline is reported against."""
    import torch
    n = P.pa_bench_intops_threads()
    per = P.pa_bench_intops_per_iter()
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = {}
    for name, kind, ops_per_step, inst_per_step in INTOPS_KINDS:
        P.pa_bench_intops(kind, iters // 10, out.data_ptr(), n, s.cuda_stream)  # warm-up
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(reps):
            P.pa_bench_intops(kind, iters, out.data_ptr(), n, s.cuda_stream)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        steps = n * iters * per
        res[name] = {"tinst_per_s": steps * inst_per_step / (ms * 1e-3) / 1e12,
                     "tops": steps * ops_per_step / (ms * 1e-3) / 1e12, "ms": ms}
    res["threads"] = n
    res["unit"] = "T per s (thread-instructions, 32-bit int ops)"
    best = max((k for k, *_ in INTOPS_KINDS), key=lambda k: res[k]["tops"])
    res["peak_kind"] = best
    res["peak_tops"] = res[best]["tops"]
    # 32 x 32 -> 64 products per second: one per mul_wide+xor step
    res["multiply_peak_t_per_s"] = res["mul_wide+xor"]["tops"] / 3.0
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--R0", type=int, default=WORKLOAD["R0"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-next", action="store_true",
                    help="skip the Poisson / adaptive / checkpoint measurements")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    ens_pool = None
    if not args.no_ensemble and world == 1:
        # the oracle's twin of one config-4 instance runs beside the GPU work
        import multiprocessing as mp
        ens_pool = mp.get_context("spawn").Pool(1)

    import torch

    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2006_00561_gb300 import pa as P

    wl = rank_workload(rank, args.R0)
    cfg = P.make_config(layout=P.LAYOUT_PACKED, **wl)
    stream = torch.cuda.Stream()
    run = P.Run(cfg, stream=stream)
    N = wl["L"] ** 2
    theta = wl["theta"]
    e2e_warm = max(1, min(args.warmup, 3))
    assert args.warmup + 2 * args.steps + (0 if args.no_e2e else args.steps + e2e_warm) <= wl["K"]

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
    ms_graph, attempts_all = aggregate(dist, ms_graph, attempts, "cuda")
    value = attempts_all / (ms_graph * 1e6)
    run.observables()  # raises on a sticky device error

    # ---- timed region 2: plain launches with per-kernel events -------------
    P.pa_profile(run.h, True)
    P.pa_profile_read(run.h, reset=True)
    sources0 = run.state()["sources"]
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
    res_ms = prof["resample"][1] / max(prof["resample"][0], 1)  # k_resample alone
    sweep_attempts_per_launch = attempts2 / max(n_sw, 1)
    achieved_tops = OPS_PER_ATTEMPT * sweep_attempts_per_launch / (sweep_ms * 1e-3) / 1e12
    resampled_per_s = resampled2 / ((prof["tau"][1] + prof["resample"][1]) * 1e-3)
    # resample traffic (bytes per launch): per input replica the level read (4)
    # and the count and offset writes (8); per surviving source (copy count >
    # 0, counted on the device) its spins, level and magnetisation read once;
    # per output slot spins, level and magnetisation written once
    st_after = run.state()
    stride = st_after["stride"]
    sources = (st_after["sources"] - sources0) / args.steps
    R_in = resampled2 / args.steps
    R_out = sum(Rs2[1:]) / args.steps
    res_bytes = R_in * 12 + sources * (stride + 8) + R_out * (stride + 8)
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
        copy_stream = torch.cuda.Stream()
        # untimed warm-up steps of the same path (the first streamed step pays
        # one-time costs of the copy stream and the pinned buffer)
        for _ in range(e2e_warm):
            P.pa_load_ptr(run.h, P.DUMP_SPINS_RAW, host.data_ptr(), R_now, R_now * stride)
            run.step_stream(host, E2E_CHUNKS, copy_stream)
            R_now = run.observables()["R"]
        # device-side split of every timed step: the upload (copy + measurement
        # pass) and the streamed step with its copies out, by events on the
        # run's stream (they add no synchronisation)
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)]
               for _ in range(args.steps)]
        barrier()
        gc.collect()
        gc.disable()  # no collector pause inside the host-timed loop
        t0 = time.perf_counter()
        h2d = d2h = 0
        e2e_attempts = 0
        for i in range(args.steps):
            evs[i][0].record(stream)
            P.pa_load_ptr(run.h, P.DUMP_SPINS_RAW, host.data_ptr(), R_now, R_now * stride)
            h2d += R_now * stride
            evs[i][1].record(stream)
            # the step, with the new population copied back range by range
            # while the later ranges sweep
            run.step_stream(host, E2E_CHUNKS, copy_stream)
            evs[i][2].record(stream)
            o = run.observables()  # returns once the copies are done
            R_now = o["R"]
            e2e_attempts += R_now * N * theta
            d2h += R_now * stride + 104
        barrier()
        dt = time.perf_counter() - t0
        gc.enable()
        up_steps = [e[0].elapsed_time(e[1]) for e in evs]
        up = sorted(up_steps)
        st_ms = sorted(e[1].elapsed_time(e[2]) for e in evs)
        # device idle between a step's end and the next upload: the host's
        # read of the observables and its next calls
        gaps = sorted(evs[i][2].elapsed_time(evs[i + 1][0]) for i in range(args.steps - 1))
        dt, e2e_attempts = aggregate(dist, dt, e2e_attempts, "cuda")
        e2e = {"value": e2e_attempts / (dt * 1e9), "unit": UNIT,
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
               "wall_ms_per_step": dt * 1e3 / args.steps,
               "device_ms_per_step_median": {"upload": up[len(up) // 2],
                                             "streamed_step": st_ms[len(st_ms) // 2]},
               "upload_ms_per_step": [round(x, 3) for x in up_steps],
               "gap_ms_median_max": [gaps[len(gaps) // 2], gaps[-1]] if gaps else None,
               "path": "pa_load(pinned host population) + pa_step_stream(population back "
                       f"to pinned host in {E2E_CHUNKS} ranges, copies overlapping the sweeps) + "
                       "pa_observables every step"}

    run.close()
    del run
    torch.cuda.empty_cache()
    rng_ceiling = philox_ceiling(P, sweep_attempts_per_launch / (sweep_ms * 1e6))
    ipk = int_peaks(P)
    int_peak = ipk["peak_tops"]
    sweep_rate = sweep_attempts_per_launch / (sweep_ms * 1e6)  # attempts/ns
    mult_rate = sweep_rate * MULTIPLIES_PER_ATTEMPT / 1e3  # T products/s
    # the generator alone forms MULTIPLIES_PER_ATTEMPT products per uniform
    mult_peak = max(ipk["multiply_peak_t_per_s"],
                    rng_ceiling["uniforms_per_ns"] * MULTIPLIES_PER_ATTEMPT / 1e3)
    ens = srv = nxt = None
    if not args.no_ensemble and world == 1:
        ens = ensemble_compare(P, steps=20, oracle_pool=ens_pool)
        ens_pool.close()
        ens_pool.join()
    if not args.no_serving and world == 1:
        srv = serving_measure(P)
    if not args.no_next and world == 1:
        nxt = next_items_measure(P, R0=args.R0)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    cpu = None
    if world == 1 and args.cpu_seconds > 0:
        procs = os.cpu_count() or 1
        r1 = oracle_rate(args.cpu_seconds / 2)
        rp = oracle_rate(args.cpu_seconds / 2, procs=procs)
        cpu = {"value": rp["attempts_per_ns"], "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"{procs} independent oracle processes (different seeds), "
                         f"{rp['steps']} full PA steps in all of the L=64 workload at "
                         f"R0={rp['R0']} (theta=10), {rp['seconds']:.1f} s",
               "resampled_replicas_per_s": rp["resampled_replicas_per_s"],
               "single_thread": {"value": r1["attempts_per_ns"], "cores": 1,
                                 "steps": r1["steps"], "seconds": r1["seconds"],
                                 "resampled_replicas_per_s": r1["resampled_replicas_per_s"]},
               "host": host_info()}
        cfg1 = config1_measure(P, procs)
        if ens:
            ens["oracle"] = ensemble_oracle_rate(procs)
    else:
        cfg1 = None
    cfg2 = config2_measure(P) if world == 1 else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_graph / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": arm_config(wl["R0"], first, args.steps, world),
        "resampled_replicas_per_s": resampled_per_s,
        "plain": {"value": value_plain, "ms_per_step": ms_plain / args.steps,
                  "note": "one launch per kernel per step, kernel events on"},
        "batched": {"value": value, "ms_per_step": ms_graph / args.steps,
                    "note": "one CUDA graph per step (pa_run_steps)"},
        "kernels_ms_per_step": {k: (v[1] / max(v[0], 1)) for k, v in prof.items()},
        "sweep_attempts_per_ns_kernel": sweep_attempts_per_launch / (sweep_ms * 1e6),
        "roofline": {"bound": "alu", "achieved": achieved_tops, "peak": int_peak,
                     "unit": "Tops/s (32-bit int)", "frac": achieved_tops / int_peak,
                     "traffic": (SWEEP_TRAFFIC_BYTES_2P21
                                 if wl["R0"] == 1 << 21 and SWEEP_TRAFFIC_BYTES_2P21 else None),
                     "traffic_note": "ncu dram bytes at 2^20 replicas x 2 (profiles/)",
                     "kernel": "k_sweep_l64 (theta=10 sweeps + measurement)",
                     "ops_per_attempt": OPS_PER_ATTEMPT,
                     "peak_note": "measured in this run: the fastest 32-bit integer op "
                                  "stream of pa_bench_intops (int_peaks.peak_kind; of measured)",
                     "derived_peak": ALU_PEAK_TOPS,
                     "frac_of_derived": achieved_tops / ALU_PEAK_TOPS,
                     "multiply_bound": {
                         "achieved_t_products_per_s": mult_rate,
                         "peak_t_products_per_s": mult_peak, "frac": mult_rate / mult_peak,
                         "note": f"the sweep's Philox multiplies ({MULTIPLIES_PER_ATTEMPT:g} per "
                                 "attempt) against the "
                                 "fastest measured 32x32->64 product rate (mul.wide+xor chains "
                                 "or the generator alone, whichever is higher)"}},
        "int_peaks": ipk,
        "philox_ceiling": rng_ceiling,
        "resample_roofline": {"bound": "hbm", "achieved": res_gbs, "peak": hbm, "unit": "GB/s",
                              "frac": res_gbs / hbm, "traffic": None,
                              "kernel": "k_resample (counts + lookback scan + gather)",
                              "bytes_per_launch": res_bytes,
                              "sources_per_launch": sources, "R_in": R_in, "R_out": R_out,
                              "peak_note": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
        # kernels inside the headline timed region: k_tau, k_resample, the sweep
        # kernel and k_obs per graph-replayed step
        "gpu_launches": 4 * args.steps,
        "clocks": clk.result,
    }
    if e2e:
        line["e2e"] = e2e
    if cpu:
        line["cpu_baseline"] = cpu
    if nxt:
        line["next_items"] = nxt
    if cfg1:
        line["config1"] = cfg1
    if cfg2:
        line["config2"] = cfg2
    if srv:
        line["serving"] = srv
    # last, so that the end of the line (what a log tail keeps) holds the
    # batched-over-plain comparison of config 4 and its parity
    if ens:
        line["batched_ensemble"] = ens
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
