"""The autotuning cache's host logic with a stand-in context and device (no GPU): a miss tunes
and stores the plan, a hit applies the stored plan without timing anything, `refresh` tunes
again, another size bucket misses, and an unreadable cache file counts as empty."""
import json
import types

import pytest
import torch

from paper_2108_07346_gb300 import autotune


class StandInContext:
    device = "cuda:0"

    def __init__(self):
        self.tuned = 0
        self.applied = None

    def autotune(self, u, v, V, reps=3):
        self.tuned += 1
        return {"M": 4, "fan_in": 4, "block": 512, "warm_edges": 1000 * self.tuned, "warm_block": 256}

    def set_opts(self, **kw):
        self.applied = kw


@pytest.fixture(autouse=True)
def stand_in_device(monkeypatch):
    props = types.SimpleNamespace(multi_processor_count=152, name="stand-in GPU")
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda device: props)


def edges(E):
    return torch.zeros(E, dtype=torch.int32), torch.zeros(E, dtype=torch.int32)


def test_miss_tunes_and_hit_applies(tmp_path):
    path = str(tmp_path / "sub" / "cache.json")
    u, v = edges(5000)
    c = StandInContext()
    plan, hit = autotune.tune(c, u, v, 300, path=path)
    assert not hit and c.tuned == 1 and c.applied is None
    stored = json.load(open(path))
    assert list(stored.values()) == [plan]
    c2 = StandInContext()
    plan2, hit2 = autotune.tune(c2, u, v, 310, path=path)  # same bucket: log2 sizes round alike
    assert hit2 and c2.tuned == 0 and plan2 == plan
    assert c2.applied == {"M": 4, "fan_in": 4, "block": 512, "warm_edges": 1000, "warm_block": 256}


def test_refresh_and_other_buckets(tmp_path):
    path = str(tmp_path / "cache.json")
    c = StandInContext()
    autotune.tune(c, *edges(5000), 300, path=path)
    plan, hit = autotune.tune(c, *edges(5000), 300, path=path, refresh=True)
    assert not hit and c.tuned == 2 and plan["warm_edges"] == 2000
    autotune.tune(c, *edges(5000), 5000, path=path)  # another vertex bucket
    autotune.tune(c, *edges(80000), 300, path=path)  # another edge bucket
    assert c.tuned == 4 and len(json.load(open(path))) == 3


def test_unreadable_cache_counts_as_empty(tmp_path):
    path = tmp_path / "cache.json"
    path.write_text("{ not json")
    c = StandInContext()
    plan, hit = autotune.tune(c, *edges(100), 50, path=str(path))
    assert not hit and c.tuned == 1
    assert list(json.load(open(path)).values()) == [plan]


class StandInBatchContext:
    device = "cuda:0"

    def __init__(self):
        self.tuned = 0
        self.applied = None

    def batch_autotune(self, u, v, edge_off, Vs, reps=3):
        self.tuned += 1
        plan = [{"vmax": b, "group": 1024 if b > 1024 else 512, "split": 1 << 20, "warm_per_v": 2,
                 "warm_add": 1024 * self.tuned} for b in autotune.BATCH_BUCKETS]
        return plan, 1234.0

    def set_batch_plan(self, buckets):
        self.applied = buckets


def test_batched_plan_cached_per_bucket(tmp_path):
    path = str(tmp_path / "cache.json")
    u, v = edges(100)
    ctx = StandInBatchContext()
    plan, hit = autotune.tune_batched(ctx, u, v, [0, 50, 100], [300, 3000], path=path)
    assert not hit and ctx.tuned == 1
    stored = json.load(open(path))
    # only the buckets the batch's graphs fall in (V = 300 -> 512, V = 3000 -> 4096) are stored
    assert sorted(k.split(":")[1] for k in stored) == ["4096", "512"]
    assert all(k.endswith(":152:stand-in GPU") and k.startswith("batch:") for k in stored)
    # a batch within the cached buckets hits and applies the stored entries without tuning
    ctx2 = StandInBatchContext()
    plan2, hit2 = autotune.tune_batched(ctx2, u, v, [0, 100], [500], path=path)
    assert hit2 and ctx2.tuned == 0
    applied = {d["vmax"]: d for d in ctx2.applied}
    assert applied[512]["warm_add"] == 1024 and applied[512]["group"] == 512
    assert applied[256]["group"] == 0  # uncached buckets stay automatic
    # a graph in an uncached bucket (V = 100 -> 256) misses and tunes again
    plan3, hit3 = autotune.tune_batched(ctx2, u, v, [0, 50, 100], [100, 500], path=path)
    assert not hit3 and ctx2.tuned == 1
    # refresh tunes even when everything is cached
    _, hit4 = autotune.tune_batched(ctx2, u, v, [0, 100], [500], path=path, refresh=True)
    assert not hit4 and ctx2.tuned == 2
