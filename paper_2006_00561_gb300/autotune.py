"""Autotuner of the batched sweep launch shape.

For every sweep class of a batch (runs sharing layout, dim, L and model) it
times whole batched steps with each candidate block shape (warps per block =
replicas in flight per CTA) and keeps the fastest.  The launch shape never
changes the results (random numbers are keyed by replica and site, not by
thread), so the timed steps are real steps of the runs.  Choices are cached
per (GPU, class, slot count rounded to a power of two) in a JSON file.
"""
from __future__ import annotations

import json
import os

CANDIDATES = (2, 4, 8)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "pa_gb300", "autotune.json")


def _key(gpu: str, c: dict) -> str:
    slots = 1 << max(0, int(c["slots"]) - 1).bit_length()
    return f"{gpu}|layout{c['layout']}|d{c['dim']}|L{c['L']}|m{c['model']}|slots{slots}"


def tune(batch, steps_left: int, cache_path: str | None = DEFAULT_CACHE, verbose=False) -> dict:
    """Chooses warps per block for every class; returns {class index: warps} and
    the number of batch steps it consumed."""
    import torch
    gpu = torch.cuda.get_device_name()
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
    used = 0
    choice = {}
    for ci, c in enumerate(batch.classes()):
        k = _key(gpu, c)
        if c["warps"] == 16:          # the L = 64 register kernel has one shape
            choice[ci] = 16
            continue
        if k in cache:
            batch.set_warps(ci, int(cache[k]))
            choice[ci] = int(cache[k])
            continue
        best, best_ms = None, None
        for w in CANDIDATES:
            if used >= steps_left:
                break
            try:
                batch.set_warps(ci, w)
            except RuntimeError:       # a shape this class's kernel does not take
                continue
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            batch.sync()
            e0.record(batch.stream)
            batch.step()
            e1.record(batch.stream)
            batch.sync()
            used += 1
            ms = e0.elapsed_time(e1)
            if verbose:
                print(f"autotune class {ci} {k}: warps={w} step {ms:.3f} ms")
            if best_ms is None or ms < best_ms:
                best, best_ms = w, ms
        if best is not None:
            batch.set_warps(ci, best)
            choice[ci] = best
            cache[k] = best
    if cache_path:
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return {"choice": choice, "steps_used": used}
