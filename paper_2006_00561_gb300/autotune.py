"""Autotuner of the batched sweep launch shape.

For every sweep class of a batch (runs sharing layout, dim, L and model) it
times whole batched steps with each candidate shape and keeps the fastest.  A
shape is (warps per block, slots per claim):
  * warps per block: 2, 4 or 8 (replicas in flight per CTA: one per warp for
    the warp-per-replica kernels, 32 per warp for the replica-sliced one); the
    L = 64 register kernel has a single block shape;
  * slots per claim: how many consecutive replicas of one run a warp claims
    at a time from the class's slot space (1 .. 32, or 0 for the engine's
    automatic choice of about four claims per resident warp).  The
    replica-sliced kernel (packed lattices with L <= 32) always claims 32.
The launch shape never changes the results (random numbers are keyed by
replica and site, not by thread), so the timed steps are real steps of the
runs.  Choices are cached per (GPU, class, slot count rounded to a power of
two) in a JSON file.

The resample's copy tile (replicas per tile, loads in flight per thread) sizes
each run's lookback descriptors in its workspace, so it is fixed when the
library is built and tuned offline.
"""
from __future__ import annotations

import json
import os

WARPS = (2, 4, 8)
CHUNKS = (0, 4, 8, 16, 32)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "pa_gb300", "autotune.json")


def _key(gpu: str, c: dict) -> str:
    slots = 1 << max(0, int(c["slots"]) - 1).bit_length()
    return f"{gpu}|layout{c['layout']}|d{c['dim']}|L{c['L']}|m{c['model']}|slots{slots}"


def replica_sliced(c: dict) -> bool:
    """The class runs the replica-sliced kernel (32 replicas per warp, claims
    of 32 slots): packed layout with L <= 32."""
    return c["layout"] == 1 and c["L"] <= 32


def candidates(c: dict) -> list:
    """(warps, chunk) shapes to try for one class."""
    if c["layout"] == 1 and c["dim"] == 2 and c["L"] in (64, 128):
        return [(c["warps"], ch) for ch in CHUNKS]  # register kernels: one block shape
    if replica_sliced(c):
        return [(w, 0) for w in WARPS]
    return [(w, ch) for w in WARPS for ch in CHUNKS]


def tune(batch, steps_left: int, cache_path: str | None = DEFAULT_CACHE, verbose=False) -> dict:
    """Chooses a (warps, chunk) shape for every class; returns {"shapes":
    {class index: (warps, chunk)}, "choice": {class index: warps},
    "steps_used": batch steps consumed}."""
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
    shapes = {}
    for ci, c in enumerate(batch.classes()):
        k = _key(gpu, c)
        cached = cache.get(k)
        if isinstance(cached, list) and len(cached) == 2:
            batch.set_shape(ci, int(cached[0]), int(cached[1]))
            shapes[ci] = (int(cached[0]), int(cached[1]))
            continue
        best, best_ms = None, None
        for w, ch in candidates(c):
            if used >= steps_left:
                break
            try:
                batch.set_shape(ci, w, ch)
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
                print(f"autotune class {ci} {k}: warps={w} chunk={ch} step {ms:.3f} ms")
            if best_ms is None or ms < best_ms:
                best, best_ms = (w, ch), ms
        if best is not None:
            batch.set_shape(ci, best[0], best[1])
            shapes[ci] = best
            cache[k] = list(best)
    if cache_path:
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return {"shapes": shapes, "choice": {ci: s[0] for ci, s in shapes.items()},
            "steps_used": used}
