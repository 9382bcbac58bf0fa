"""The launch-shape autotuner's search and cache (CPU only): a fake scene whose per-kernel
timer returns a made-up cost for the shape last applied."""
import json

import pytest
import torch

from paper_2409_16385_gb300 import autotune


@pytest.fixture(autouse=True)
def _no_device(monkeypatch):
    """No GPU here: the device key is fixed and the stream synchronisation is a no-op."""
    monkeypatch.setattr(autotune, "device_key", lambda: "fake|sm_103|152sm")
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)


class FakeScene:
    def __init__(self, cost):
        self.cost = cost                   # (kernel, shape) -> ms
        self.shape = {}
        self.enabled = []
        self.stage_calls = 0

    def set_launch(self, kernel, threads, bps, variant=2):
        self.shape[kernel] = (threads, bps, variant)
        self.last = kernel

    def timing_enable(self, names=None):
        self.enabled = list(names or [])

    def timing_read(self):
        # a timer can bracket several knobs (the evaluation's shape and its queue tile):
        # the cost is that of the knob set last among those the timer covers
        out = {}
        for timer in self.enabled:
            knobs = [k for k, t in autotune.TIMERS.items() if t == timer]
            kernel = self.last if getattr(self, "last", None) in knobs else knobs[0]
            out[timer] = (self.cost(kernel, self.shape.get(kernel)), 1)
        return out


def _cost(kernel, shape):
    if shape is None:
        return 10.0
    threads, bps, variant = shape
    best = {"eval_barrier": (64, 4, 3), "bvh_query": (256, 12, 2), "bvh_refit": (256, 8, 1),
            "eval_tile": (64, 1, 0), "ccd_tile": (128, 1, 0)}[kernel]
    return 1.0 + abs(threads - best[0]) / 64 + abs(bps - best[1]) + abs(variant - best[2])


def test_picks_the_fastest_shape_and_caches_it(tmp_path):
    cache = str(tmp_path / "tune.json")
    cs = FakeScene(_cost)

    def stage():
        cs.stage_calls += 1

    res = autotune.tune(cs, stage, "workload-a", cache_path=cache)
    assert res["eval_barrier"]["shape"] == [64, 4, 3] and not res["eval_barrier"]["cached"]
    assert res["bvh_query"]["shape"] == [256, 12, 2]
    assert res["bvh_refit"]["shape"] == [256, 8, 1]
    assert res["eval_tile"]["shape"] == [64, 1, 0] and res["ccd_tile"]["shape"] == [128, 1, 0]
    assert cs.shape == {"eval_barrier": (64, 4, 3), "bvh_query": (256, 12, 2), "bvh_refit": (256, 8, 1),
                        "eval_tile": (64, 1, 0), "ccd_tile": (128, 1, 0)}
    assert res["eval_barrier"]["ms"] == 1.0
    assert len(res["eval_barrier"]["candidates"]) == len(autotune.EVAL_SPACE)
    table = json.load(open(cache))
    assert "fake|sm_103|152sm|workload-a" in table

    # a second run on the same device and workload reads the cache and times nothing
    cs2 = FakeScene(_cost)
    calls = []
    res2 = autotune.tune(cs2, lambda: calls.append(1), "workload-a", cache_path=cache)
    assert not calls and all(r["cached"] for r in res2.values())
    assert cs2.shape["eval_barrier"] == (64, 4, 3)

    # another workload key, or force, searches again
    calls = []
    autotune.tune(FakeScene(_cost), lambda: calls.append(1), "workload-b", cache_path=cache)
    assert calls
    calls = []
    autotune.tune(FakeScene(_cost), lambda: calls.append(1), "workload-a", cache_path=cache, force=True)
    assert calls


def test_unreadable_cache_is_ignored(tmp_path):
    cache = tmp_path / "tune.json"
    cache.write_text("{ not json")
    cs = FakeScene(_cost)
    res = autotune.tune(cs, lambda: None, "w", kernels=("bvh_refit",), cache_path=str(cache))
    assert res["bvh_refit"]["shape"] == [256, 8, 1]
    assert json.loads(cache.read_text())["fake|sm_103|152sm|w"]["bvh_refit"]["shape"] == [256, 8, 1]
