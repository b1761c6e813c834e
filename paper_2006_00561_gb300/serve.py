"""Serving loop: continuous batching of population-annealing runs.

Requests (one PA run each) arrive over time.  A request is admitted when its
workspace fits the HBM budget; its population then stays resident in device
memory until it finishes.  Every iteration advances all resident runs together
with the batched form (one launch per phase for all of them, each run at its
own step of its own schedule), so requests that arrive while others are
running join the device work at the next iteration.  A finished run's final
observables are read back, its workspace is released, and waiting requests
take the freed memory.  Results do not depend on which runs shared a batch:
every run gives the bits it gives when stepped alone.

The loop is host code around the C ABI (pa_init, pa_batch_*, pa_observables);
PyTorch provides the device memory and the stream.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

from . import pa as P


@dataclasses.dataclass
class Request:
    rid: int
    spec: dict                   # make_config keyword arguments (plus 'arrival' seconds)
    arrival: float               # seconds after the server's start
    admitted: float | None = None
    finished: float | None = None
    result: dict | None = None   # final observables
    history: list | None = None  # observables of every step, if kept
    error: str | None = None
    run: object = None
    step: int = 0                # annealing steps done (tracked on the host)
    spins: object = None         # final population (int8), if kept

    @property
    def latency(self):
        return None if self.finished is None else self.finished - self.arrival

    def attempts(self) -> int:
        N = self.spec["L"] ** self.spec["dim"]
        return sum(h["R"] for h in (self.history or [])[1:]) * N * self.spec["theta"]


class Server:
    """Continuous-batching server over one GPU.

    hbm_budget: bytes of device memory the resident runs' workspaces may use.
    quantum: most steps run between two admission / retirement points.
    layout: spin layout of every admitted run.
    """

    def __init__(self, hbm_budget: int, quantum: int = 8, layout: int = P.LAYOUT_PACKED,
                 keep_history: bool = True, keep_spins: bool = False, stream=None):
        if stream is None:
            import torch
            stream = torch.cuda.Stream()
        self.budget = int(hbm_budget)
        self.quantum = int(quantum)
        self.layout = layout
        self.keep_history = keep_history
        self.keep_spins = keep_spins
        self.stream = stream
        self.queue: list[Request] = []
        self.resident: list[Request] = []
        self.done: list[Request] = []
        self.rejected: list[Request] = []
        self.used = 0
        self.max_used = 0
        self.batch = None
        self.batch_members: tuple = ()
        self.iterations = 0
        self.max_resident = 0
        self.t0 = None
        self.phase_s = {"admit": 0.0, "batch": 0.0, "steps": 0.0, "retire": 0.0}

    # -- requests --------------------------------------------------------------
    def _cfg(self, spec: dict) -> P.Config:
        keys = ("dim", "L", "model", "K", "theta", "instance_id", "R0", "beta0", "beta_max",
                "seed", "coupling_seed", "init", "resample")
        return P.make_config(layout=self.layout, **{k: spec[k] for k in keys if k in spec})

    def footprint(self, spec: dict) -> int:
        return P.pa_workspace_size(self._cfg(spec))

    def submit(self, rid: int, spec: dict, arrival: float):
        req = Request(rid, dict(spec), arrival)
        need = self.footprint(spec)
        if need == 0 or need > self.budget:
            req.error = "rejected: footprint above the HBM budget" if need else "invalid config"
            self.rejected.append(req)
        else:
            self.queue.append(req)
        return req

    # -- one iteration ---------------------------------------------------------
    def _now(self) -> float:
        return time.perf_counter() - self.t0

    def _admit(self, now: float) -> bool:
        changed = False
        self.queue.sort(key=lambda r: r.arrival)
        i = 0
        while i < len(self.queue):
            req = self.queue[i]
            if req.arrival > now:
                break
            need = self.footprint(req.spec)
            if self.used + need > self.budget:
                break  # first come, first served: later requests wait too
            req.run = P.Run(self._cfg(req.spec), stream=self.stream)
            req.admitted = now
            self.used += need
            self.max_used = max(self.max_used, self.used)
            self.resident.append(req)
            self.queue.pop(i)
            changed = True
        self.max_resident = max(self.max_resident, len(self.resident))
        return changed

    def _retire(self) -> bool:
        keep, changed = [], False
        for req in self.resident:
            if req.step >= req.spec["K"]:
                if self.keep_spins:
                    req.spins = req.run.spins()
                if self.keep_history:
                    req.history = req.run.history(0, req.spec["K"] + 1)
                req.result = req.run.observables()
                req.finished = self._now()
                self.used -= self.footprint(req.spec)
                req.run.close()
                req.run = None
                self.done.append(req)
                changed = True
            else:
                keep.append(req)
        self.resident = keep
        return changed

    def step(self) -> int:
        """Admit, advance every resident run by up to `quantum` steps, retire.
        Returns the number of steps advanced."""
        if self.t0 is None:
            self.t0 = time.perf_counter()
        t = time.perf_counter()
        now = t - self.t0
        self._admit(now)
        t1 = time.perf_counter()
        self.phase_s["admit"] += t1 - t
        if not self.resident:
            return 0
        members = tuple(id(r) for r in self.resident)
        if self.batch is None or members != self.batch_members:
            if self.batch is not None:
                self.batch.close()
            self.batch = P.Batch([r.run for r in self.resident], stream=self.stream)
            self.batch_members = members
        t2 = time.perf_counter()
        self.phase_s["batch"] += t2 - t1
        left = min(r.spec["K"] - r.step for r in self.resident)
        n = max(1, min(self.quantum, left))
        self.batch.run_steps(n)
        rc = self.batch.sync()
        if rc != 0:
            raise P.PaError(rc, "batched step")
        for r in self.resident:
            r.step += n
        self.iterations += 1
        t3 = time.perf_counter()
        self.phase_s["steps"] += t3 - t2
        if self._retire():
            self.batch.close()
            self.batch = None
            self.batch_members = ()
        self.phase_s["retire"] += time.perf_counter() - t3
        return n

    def idle(self) -> bool:
        return not self.resident and not self.queue

    def run_trace(self, trace: list, time_scale: float = 1.0, max_seconds: float = 1e9) -> dict:
        """Serves a list of request specs with an 'arrival' key (seconds, scaled
        by time_scale) in real time and returns latency / throughput stats."""
        self.t0 = time.perf_counter()
        pending = sorted(enumerate(trace), key=lambda x: x[1]["arrival"])
        k = 0
        while k < len(pending) or not self.idle():
            now = self._now()
            while k < len(pending) and pending[k][1]["arrival"] * time_scale <= now:
                rid, spec = pending[k]
                self.submit(rid, spec, spec["arrival"] * time_scale)
                k += 1
            if self.resident or (self.queue and self.queue[0].arrival <= now):
                self.step()
            elif k < len(pending):
                time.sleep(min(0.001, max(0.0, pending[k][1]["arrival"] * time_scale - now)))
            if now > max_seconds:
                break
        if self.batch is not None:
            self.batch.close()
            self.batch = None
        return self.stats()

    def stats(self) -> dict:
        lat = np.array([r.latency for r in self.done if r.latency is not None])
        wall = self._now() if self.t0 is not None else 0.0
        attempts = sum(r.attempts() for r in self.done) if self.keep_history else None
        out = {"served": len(self.done), "rejected": len(self.rejected),
               "waiting": len(self.queue), "resident": len(self.resident),
               "max_resident": self.max_resident, "iterations": self.iterations,
               "max_hbm_bytes": self.max_used, "hbm_budget": self.budget,
               "host_phase_s": dict(self.phase_s),
               "wall_s": wall}
        if lat.size:
            out.update({"p50_latency_s": float(np.percentile(lat, 50)),
                        "p99_latency_s": float(np.percentile(lat, 99)),
                        "mean_latency_s": float(lat.mean())})
        if attempts is not None and wall > 0:
            out["served_attempts_per_ns"] = attempts / (wall * 1e9)
        if wall > 0 and type(self) is Server:
            # the device works only while the host waits in the steps phase
            out["gpu_idle_fraction_host_estimate"] = max(0.0, 1.0 - self.phase_s["steps"] / wall)
        return out


class Arena:
    """First-fit sub-allocator of one device buffer, in 256-byte aligned blocks.
    The pipelined server takes every workspace from it, so admitting a request
    never calls the CUDA allocator (which may wait for the device) while
    batched steps are in flight."""

    ALIGN = 256

    def __init__(self, nbytes: int, buffer=None):
        self.size = int(nbytes) // self.ALIGN * self.ALIGN
        self.buffer = buffer
        self.free = [(0, self.size)]  # (offset, length), sorted by offset

    def _buf(self):
        if self.buffer is None:
            import torch
            self.buffer = torch.empty(self.size, dtype=torch.uint8, device="cuda")
        return self.buffer

    def alloc(self, nbytes: int):
        """Offset of a free block of nbytes (rounded up), or None."""
        n = -(-int(nbytes) // self.ALIGN) * self.ALIGN
        for i, (off, ln) in enumerate(self.free):
            if ln >= n:
                if ln == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + n, ln - n)
                return off
        return None

    def release(self, off: int, nbytes: int):
        n = -(-int(nbytes) // self.ALIGN) * self.ALIGN
        self.free.append((off, n))
        self.free.sort()
        merged = []
        for o, ln in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o:
                merged[-1] = (merged[-1][0], merged[-1][1] + ln)
            else:
                merged.append((o, ln))
        self.free = merged

    def view(self, off: int, nbytes: int):
        return self._buf()[off:off + int(nbytes)]

    def free_bytes(self) -> int:
        return sum(ln for _, ln in self.free)


@dataclasses.dataclass
class _Quantum:
    batch: object
    members: list
    n: int
    start: object
    end: object


class PipelinedServer(Server):
    """Continuous batching with the device kept busy between quanta.

    Up to `depth` quanta (batched steps of the resident runs, replayed from a
    CUDA graph) are in flight on the compute stream.  While they run, the host
    admits arrived requests (their pa_init on a separate admission stream,
    which the compute stream waits for by event before their first step),
    builds the next quantum's batch without waiting for the device
    (pa_batch_init_async, the remaining steps known on the host), polls the
    oldest quantum's completion event, and retires the runs that quantum
    finished (reading their results, returning their memory).  Workspaces come
    from one preallocated arena of `hbm_budget` bytes.  Results are those of
    the same runs stepped alone.  Statistics add the device-busy time of the
    quanta and the GPU-idle fraction between the first quantum's start and the
    last one's end."""

    BATCH_RESERVE = 8 << 20

    def __init__(self, hbm_budget: int, quantum: int = 8, depth: int = 2,
                 layout: int = P.LAYOUT_PACKED, keep_history: bool = True,
                 keep_spins: bool = False, stream=None, admit_stream=None, arena=None):
        super().__init__(hbm_budget, quantum, layout, keep_history, keep_spins, stream)
        self.depth = int(depth)
        if admit_stream is None:
            import torch
            admit_stream = torch.cuda.Stream()
        self.admit_stream = admit_stream
        # the runs' workspaces (up to the budget) plus room for the batch
        # descriptors of a few quanta
        self.arena = arena if arena is not None else Arena(self.budget + self.BATCH_RESERVE)
        self.inflight: collections.deque = collections.deque()
        self.cur_batch = None
        self.cur_members: tuple = ()
        self.batch_refs: dict = {}
        self.batch_ws: dict = {}
        self.busy_ms = 0.0
        self.first_start = None
        self.last_end = None
        self.quanta = 0

    # -- device hooks (replaced by fakes in the host tests) ------------------
    def _event(self, timing: bool = False):
        import torch
        return torch.cuda.Event(enable_timing=timing)

    @staticmethod
    def _record(ev, stream):
        ev.record(stream)

    @staticmethod
    def _wait(stream, ev):
        stream.wait_event(ev)

    # -- admission -------------------------------------------------------------
    def _admit(self, now: float) -> bool:
        changed = False
        self.queue.sort(key=lambda r: r.arrival)
        while self.queue and self.queue[0].arrival <= now:
            req = self.queue[0]
            need = self.footprint(req.spec)
            if self.used + need > self.budget:
                break  # first come, first served: later requests wait too
            off = self.arena.alloc(need)
            if off is None:
                break  # fragmented: wait for a retirement
            try:
                req.run = P.Run(self._cfg(req.spec), stream=self.admit_stream,
                                workspace=self.arena.view(off, need))
            except Exception:
                self.arena.release(off, need)
                raise
            req.ws = (off, need)
            req.init_event = self._event()
            self._record(req.init_event, self.admit_stream)
            req.admitted = now
            req.enq = 0
            self.used += need
            self.max_used = max(self.max_used, self.used)
            self.resident.append(req)
            self.queue.pop(0)
            changed = True
        self.max_resident = max(self.max_resident, len(self.resident))
        return changed

    # -- quanta ----------------------------------------------------------------
    def _close_batch(self, b):
        b.close()
        off, n = self.batch_ws.pop(id(b))
        self.arena.release(off, n)
        self.batch_refs.pop(id(b), None)

    def _enqueue(self) -> bool:
        active = [r for r in self.resident if r.enq < r.spec["K"]]
        if not active:
            return False
        members = tuple(r.rid for r in active)
        if self.cur_batch is None or members != self.cur_members:
            old = self.cur_batch
            need = int(P.lib().pa_batch_workspace_size(len(active)))
            off = self.arena.alloc(need)
            if off is None:
                return False
            try:
                self.cur_batch = P.Batch([r.run for r in active], stream=self.stream,
                                         steps_left=[r.spec["K"] - r.enq for r in active],
                                         workspace=self.arena.view(off, need))
            except Exception:
                self.arena.release(off, need)
                self.cur_batch = old
                raise
            self.batch_ws[id(self.cur_batch)] = (off, need)
            self.batch_refs[id(self.cur_batch)] = 0
            self.cur_members = members
            if old is not None and self.batch_refs.get(id(old), 0) == 0:
                self._close_batch(old)
        for r in active:
            if getattr(r, "init_event", None) is not None:
                self._wait(self.stream, r.init_event)
                r.init_event = None
        n = max(1, min(self.quantum, min(r.spec["K"] - r.enq for r in active)))
        q = _Quantum(self.cur_batch, active, n, self._event(True), self._event(True))
        self._record(q.start, self.stream)
        self.cur_batch.run_steps(n)
        self._record(q.end, self.stream)
        for r in active:
            r.enq += n
            r.last_q = q
        self.batch_refs[id(q.batch)] += 1
        self.inflight.append(q)
        self.quanta += 1
        if self.first_start is None:
            self.first_start = q.start
        return True

    def _complete(self, block: bool = False) -> bool:
        """Retires the oldest quantum if it is done (waits for it if block)."""
        if not self.inflight:
            return False
        q = self.inflight[0]
        if block:
            q.end.synchronize()
        elif not q.end.query():
            return False
        self.inflight.popleft()
        self.busy_ms += q.start.elapsed_time(q.end)
        self.last_end = q.end
        self.iterations += 1
        for r in q.members:
            r.step += q.n
        self.batch_refs[id(q.batch)] -= 1
        now = self._now()
        keep = []
        for r in self.resident:
            if r.step >= r.spec["K"] and getattr(r, "last_q", None) is q:
                self._retire_one(r, now)
            else:
                keep.append(r)
        self.resident = keep
        if q.batch is not self.cur_batch and self.batch_refs.get(id(q.batch), 1) == 0:
            self._close_batch(q.batch)
        return True

    def _retire_one(self, req, now: float):
        if self.keep_spins:
            req.spins = req.run.spins()
        if self.keep_history:
            req.history = req.run.history(0, req.spec["K"] + 1)
        req.result = req.run.observables()
        req.finished = now
        req.run.close()
        req.run = None
        off, need = req.ws
        self.arena.release(off, need)
        self.used -= need
        self.done.append(req)

    def idle(self) -> bool:
        return not self.resident and not self.queue and not self.inflight

    def run_trace(self, trace: list, time_scale: float = 1.0, max_seconds: float = 1e9) -> dict:
        t = time.perf_counter
        self.t0 = t()
        pending = sorted(enumerate(trace), key=lambda x: x[1]["arrival"])
        k = 0
        while k < len(pending) or not self.idle():
            now = self._now()
            while k < len(pending) and pending[k][1]["arrival"] * time_scale <= now:
                rid, spec = pending[k]
                self.submit(rid, spec, spec["arrival"] * time_scale)
                k += 1
            t1 = t()
            self._admit(now)
            t2 = t()
            self.phase_s["admit"] += t2 - t1
            while len(self.inflight) < self.depth and self._enqueue():
                pass
            t3 = t()
            self.phase_s["batch"] += t3 - t2
            done = self._complete()
            while done and self._complete():
                pass
            self.phase_s["retire"] += t() - t3
            if not done:
                if len(self.inflight) >= self.depth or (self.inflight and k >= len(pending)):
                    t4 = t()
                    self._complete(block=True)
                    self.phase_s["steps"] += t() - t4
                elif not self.inflight and k < len(pending):
                    time.sleep(min(0.001, max(0.0, pending[k][1]["arrival"] * time_scale -
                                               self._now())))
                elif self.inflight:
                    time.sleep(0.0002)
            if now > max_seconds:
                break
        while self.inflight:
            self._complete(block=True)
        if self.cur_batch is not None:
            self._close_batch(self.cur_batch)
            self.cur_batch = None
        return self.stats()

    def stats(self) -> dict:
        out = super().stats()
        out["quanta"] = self.quanta
        out["device_busy_s"] = self.busy_ms / 1e3
        if self.keep_history and self.busy_ms > 0:
            # the batched form's own rate on this mix: attempts over the
            # quanta's device time
            out["device_attempts_per_ns"] = (sum(r.attempts() for r in self.done) /
                                             (self.busy_ms * 1e6))
        if self.first_start is not None and self.last_end is not None:
            span = self.first_start.elapsed_time(self.last_end)
            out["device_span_s"] = span / 1e3
            out["gpu_idle_fraction"] = max(0.0, 1.0 - self.busy_ms / span) if span > 0 else 0.0
        return out


def main(argv=None):
    """python -m paper_2006_00561_gb300.serve --requests 256 --rate 50 [--server sync]
    Serves the seeded request trace in real time (by the pipelined server
    unless --server sync) and prints latency / throughput statistics
    (offered vs served load) as one JSON line."""
    import argparse
    import json

    from . import workloads
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--rate", type=float, default=50.0)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--quantum", type=int, default=8)
    ap.add_argument("--r0-exp", type=int, nargs=2, default=(12, 18))
    ap.add_argument("--k-range", type=int, nargs=2, default=(100, 300))
    ap.add_argument("--server", choices=("pipelined", "sync"), default="pipelined")
    ap.add_argument("--depth", type=int, default=2)
    a = ap.parse_args(argv)
    trace = workloads.serving_trace(a.requests, rate=a.rate, seed=a.seed, R0_exp=tuple(a.r0_exp),
                                    K_range=tuple(a.k_range))
    offered = sum(t["R0"] * t["L"] ** t["dim"] * t["theta"] * t["K"] for t in trace)
    span = trace[-1]["arrival"]
    budget = int(a.budget_gb * (1 << 30))
    if a.server == "sync":
        srv = Server(hbm_budget=budget, quantum=a.quantum)
    else:
        srv = PipelinedServer(hbm_budget=budget, quantum=a.quantum, depth=a.depth)
    st = srv.run_trace(trace)
    st.update({"server": a.server, "requests": a.requests, "rate_per_s": a.rate, "seed": a.seed,
               "offered_attempts": offered, "offered_attempts_per_ns": offered / (span * 1e9),
               "trace_span_s": span, "R0_exp": list(a.r0_exp), "K_range": list(a.k_range)})
    print(json.dumps(st))
    return st


if __name__ == "__main__":
    main()
