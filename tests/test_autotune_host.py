"""Host logic of the batched-sweep autotuner (paper_2006_00561_gb300/autotune.py)
on the CPU: a fake batch whose step time depends on each class's block shape,
and fake CUDA events on a fake clock.  The tuner must keep the fastest shape
per class, skip shapes a class's kernel refuses, respect its step budget, and
reuse its cache without timing anything."""
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
    class's share of a step in ms, and a shape missing from it is refused."""

    def __init__(self, classes, times):
        self._classes = classes
        self.times = times
        self.warps = {i: c["warps"] for i, c in enumerate(classes)}
        self.stream = None
        self.steps = 0

    def classes(self):
        return [dict(c, warps=self.warps[i]) for i, c in enumerate(self._classes)]

    def set_warps(self, ci, w):
        if (ci, w) not in self.times:
            raise RuntimeError("shape not available for this class")
        self.warps[ci] = w

    def sync(self):
        pass

    def step(self):
        self.steps += 1
        Clock.t += sum(self.times[(i, w)] for i, w in self.warps.items())


def cls(dim, L, slots, warps=4, model=1):
    return {"layout": 1, "dim": dim, "L": L, "model": model, "runs": 3, "warps": warps,
            "slots": slots, "chunk": 32}


@pytest.fixture
def fake_cuda(monkeypatch):
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda *a: "FakeGPU")
    Clock.t = 0.0


def test_keeps_the_fastest_shape_per_class_and_caches_it(fake_cuda, tmp_path):
    classes = [cls(3, 8, 3_000_000), cls(3, 10, 1_000_000), cls(2, 64, 500_000, warps=16, model=0)]
    times = {(0, 2): 9.0, (0, 4): 7.0, (0, 8): 8.0,
             (1, 2): 5.0, (1, 4): 6.0, (1, 8): 4.5,
             (2, 16): 3.0}
    b = FakeBatch(classes, times)
    path = tmp_path / "tune.json"
    out = autotune.tune(b, steps_left=100, cache_path=str(path))
    assert out["choice"] == {0: 4, 1: 8, 2: 16}
    assert out["steps_used"] == 6 and b.steps == 6  # the L = 64 class has one shape: not timed
    assert b.warps == {0: 4, 1: 8, 2: 16}
    cache = json.loads(path.read_text())
    assert sorted(cache.values()) == [4, 8] and all(k.startswith("FakeGPU|") for k in cache)

    # a second batch of the same classes takes the cached shapes without timing
    b2 = FakeBatch(classes, times)
    out2 = autotune.tune(b2, steps_left=100, cache_path=str(path))
    assert out2 == {"choice": {0: 4, 1: 8, 2: 16}, "steps_used": 0} and b2.steps == 0
    assert b2.warps == {0: 4, 1: 8, 2: 16}


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
