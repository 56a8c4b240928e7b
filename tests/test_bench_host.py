"""Host logic of bench.py, without a GPU: the walk-shape policy and the
roofline traffic lookup."""
import argparse
import os

import bench


class FakeCtx:
    """Walk times per shape, an autotuner that reports the fastest of them
    (with some noise of its own) and the config calls the bench makes."""

    def __init__(self, times, tuner_pick):
        self.times = times
        self.tuner_pick = tuner_pick
        self.shape = bench.DEFAULT_SHAPE
        self.timing = False
        self._last = 0.0

    def autotune(self, theta, eps, reps=3):
        self.shape = self.tuner_pick
        g, t, w = self.tuner_pick
        return {"gmax": g, "tile": t, "warps": w}, self.times[self.tuner_pick] * 0.97

    def set_config(self, gmax, tile, warps):
        self.shape = (gmax, tile, warps)

    def forces(self, theta, eps):
        self._last = self.times[self.shape]

    def sync(self):
        pass

    def set_timing(self, on):
        self.timing = on

    def timings(self):
        return {"walk_ms": self._last}


def _args(shape=None):
    return argparse.Namespace(shape=shape)


def test_tuned_shape_kept_when_clearly_faster():
    ctx = FakeCtx({bench.DEFAULT_SHAPE: 1.0, (32, 256, 2): 0.85}, (32, 256, 2))
    s = bench.walk_shape(ctx, _args(), 0.7)
    assert (s["gmax"], s["tile"], s["warps"]) == (32, 256, 2) and ctx.shape == (32, 256, 2)
    assert s["walk_ms_when_chosen"] == 0.85


def test_default_kept_when_the_tuned_shape_is_within_noise():
    ctx = FakeCtx({bench.DEFAULT_SHAPE: 1.0, (64, 64, 2): 0.99}, (64, 64, 2))
    s = bench.walk_shape(ctx, _args(), 0.5)
    assert (s["gmax"], s["tile"], s["warps"]) == bench.DEFAULT_SHAPE and ctx.shape == bench.DEFAULT_SHAPE
    assert s["walk_ms_when_chosen"] == 1.0


def test_explicit_shape_skips_the_tuner():
    ctx = FakeCtx({(32, 128, 4): 1.0}, None)
    s = bench.walk_shape(ctx, _args("32,128,4"), 0.5)
    assert s["chosen_by"] == "--shape" and ctx.shape == (32, 128, 4)


def test_traffic_needs_the_current_source_and_shape(tmp_path, monkeypatch):
    src = tmp_path / "walk.cuh"
    src.write_text("kernel source")
    import hashlib

    sha = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    prof = tmp_path / "walk.txt"
    prof.write_text(f"walk_source_sha256_16: {sha}\nwalk_shape: 64,128,4\ndram_bytes_per_phase: 1234\n")
    monkeypatch.setattr(bench, "WALK_SRC", str(src))
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(prof))
    assert bench._traffic_from_profile({"gmax": 64, "tile": 128, "warps": 4}) == 1234.0
    assert bench._traffic_from_profile({"gmax": 32, "tile": 256, "warps": 2}) is None
    src.write_text("kernel source, changed")
    assert bench._traffic_from_profile({"gmax": 64, "tile": 128, "warps": 4}) is None
    assert os.path.exists(prof)
