"""Host logic of the batched-sweep autotuner (paper_2006_00561_gb300/autotune.py)
on the CPU: a fake batch whose step time depends on each class's block shape,
and fake CUDA events on a fake clock.  The tuner must keep the fastest shape
per class, skip shapes a class's kernel refuses, respect its step budget, and
reuse its cache without timing anything.  A shape is (warps per block, slots
per claim); the replica-sliced classes (packed, L <= 32) take warps only and
the L = 64 / 128 register kernels slots per claim only."""
from __future__ import annotations

import json

import pytest

torch = pytest.importorskip("torch")

from paper_2006_00561_gb300 import autotune  # noqa: E402


class Clock:
    t = 0.0


class FakeEvent:
    def __init__(self, enable_timing=False):
        self.t = None

    def record(self, stream=None):
        self.t = Clock.t

    def elapsed_time(self, other):
        return other.t - self.t


class FakeBatch:
    """Classes as pa_batch_class_info reports them; times[(class, warps)] is the
    class's share of a step in ms, a shape missing from it is refused, and
    chunk_ms[(class, chunk)] is added for the slots per claim."""

    def __init__(self, classes, times, chunk_ms=None):
        self._classes = classes
        self.times = times
        self.chunk_ms = chunk_ms or {}
        self.warps = {i: c["warps"] for i, c in enumerate(classes)}
        self.chunk = {i: 0 for i in range(len(classes))}
        self.stream = None
        self.steps = 0

    def classes(self):
        return [dict(c, warps=self.warps[i]) for i, c in enumerate(self._classes)]

    def set_shape(self, ci, w, ch=0):
        w = w or self.warps[ci]
        if (ci, w) not in self.times:
            raise RuntimeError("shape not available for this class")
        self.warps[ci] = w
        self.chunk[ci] = ch

    def sync(self):
        pass

    def step(self):
        self.steps += 1
        Clock.t += sum(self.times[(i, w)] + self.chunk_ms.get((i, self.chunk[i]), 0.0)
                       for i, w in self.warps.items())


def cls(dim, L, slots, warps=4, model=1):
    return {"layout": 1, "dim": dim, "L": L, "model": model, "runs": 3, "warps": warps,
            "slots": slots, "chunk": 32}


@pytest.fixture
def fake_cuda(monkeypatch):
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FakeGPU")
    Clock.t = 0.0


def test_keeps_the_fastest_shape_per_class_and_caches_it(fake_cuda, tmp_path):
    # 3D L = 8 and 10: replica-sliced (warps only); 2D L = 64: the register
    # kernel (one block shape, slots per claim only)
    classes = [cls(3, 8, 3_000_000), cls(3, 10, 1_000_000), cls(2, 64, 500_000, warps=16, model=0)]
    times = {(0, 2): 9.0, (0, 4): 7.0, (0, 8): 8.0,
             (1, 2): 5.0, (1, 4): 6.0, (1, 8): 4.5,
             (2, 16): 3.0}
    chunk_ms = {(2, 0): 0.5, (2, 4): 0.9, (2, 8): 0.3, (2, 16): 0.1, (2, 32): 0.2}
    b = FakeBatch(classes, times, chunk_ms)
    path = tmp_path / "tune.json"
    out = autotune.tune(b, steps_left=100, cache_path=str(path))
    assert out["shapes"] == {0: (4, 0), 1: (8, 0), 2: (16, 16)}
    assert out["choice"] == {0: 4, 1: 8, 2: 16}
    assert out["steps_used"] == 11 and b.steps == 11  # 3 + 3 warps, 5 chunks
    assert b.warps == {0: 4, 1: 8, 2: 16} and b.chunk[2] == 16
    cache = json.loads(path.read_text())
    assert sorted(cache.values()) == [[4, 0], [8, 0], [16, 16]]
    assert all(k.startswith("FakeGPU|") for k in cache)

    # a second batch of the same classes takes the cached shapes without timing
    b2 = FakeBatch(classes, times, chunk_ms)
    out2 = autotune.tune(b2, steps_left=100, cache_path=str(path))
    assert out2["shapes"] == out["shapes"] and out2["steps_used"] == 0 and b2.steps == 0
    assert b2.warps == {0: 4, 1: 8, 2: 16} and b2.chunk[2] == 16


def test_warp_per_replica_classes_search_warps_and_chunks(fake_cuda, tmp_path):
    """An int8 class (layout 0) takes both knobs: 3 warps x 5 chunks."""
    c = dict(cls(2, 16, 100_000), layout=0)
    times = {(0, 2): 2.0, (0, 4): 1.0, (0, 8): 3.0}
    chunk_ms = {(0, 8): -0.5}
    b = FakeBatch([c], times, chunk_ms)
    out = autotune.tune(b, steps_left=100, cache_path=None)
    assert out["shapes"] == {0: (4, 8)} and out["steps_used"] == 15


def test_skips_refused_shapes_and_respects_the_step_budget(fake_cuda, tmp_path):
    classes = [cls(3, 6, 2_000_000), cls(3, 8, 2_000_000)]
    times = {(0, 4): 6.0, (0, 8): 5.0,            # class 0 refuses 2 warps
             (1, 2): 7.0, (1, 4): 3.0, (1, 8): 1.0}
    b = FakeBatch(classes, times)
    out = autotune.tune(b, steps_left=3, cache_path=str(tmp_path / "t.json"))
    # class 0 times 4 and 8 (2 steps); class 1 has one step left: only 2 warps
    assert out["steps_used"] == 3
    assert out["choice"] == {0: 8, 1: 2}


def test_cache_key_rounds_the_slot_count_to_a_power_of_two():
    a = autotune._key("G", cls(3, 8, 3_000_000))
    b = autotune._key("G", cls(3, 8, 4_194_304))
    c = autotune._key("G", cls(3, 8, 4_194_305))
    assert a == b != c
