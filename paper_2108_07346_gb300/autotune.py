"""Persistent cache of autotuning results keyed by problem size and GPU (a small JSON file).

Single graphs (bridges_autotune): key (round(log2 V), round(log2 E), number of SMs, device
name).  Batches (bridges_batch_autotune): one entry per size bucket of the batched plan, key
("batch", the bucket's vertex bound, number of SMs, device name).  A hit applies the cached plan
to the context without timing anything; a miss tunes on the caller's input and stores the result.
"""
from __future__ import annotations

import json
import math
import os

import torch

DEFAULT_PATH = os.path.join(os.path.expanduser("~"), ".cache", "bridges_autotune.json")


def _key(E: int, V: int, device) -> str:
    p = torch.cuda.get_device_properties(device)
    return f"{round(math.log2(max(V, 1)))}:{round(math.log2(max(E, 1)))}:{p.multi_processor_count}:{p.name}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, cache):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


BATCH_BUCKETS = (256, 512, 1024, 2048, 4096)  # the vertex bounds bridges_batch_autotune tunes


def _batch_key(vmax: int, device) -> str:
    p = torch.cuda.get_device_properties(device)
    return f"batch:{vmax}:{p.multi_processor_count}:{p.name}"


def tune_batched(ctx, u, v, edge_off, Vs, path: str = DEFAULT_PATH, reps: int = 3, refresh: bool = False):
    """Applies the cached batched plan to `ctx` when every size bucket the batch's graphs fall in
    is cached for this GPU; otherwise tunes on the batch (bridges_batch_autotune) and stores each
    bucket.  Returns (per-bucket plan list, hit)."""
    present = sorted({next((b for b in BATCH_BUCKETS if int(x) <= b), None) for x in Vs} - {None})
    cache = _load(path)
    keys = {b: _batch_key(b, ctx.device) for b in BATCH_BUCKETS}
    if not refresh and present and all(keys[b] in cache for b in present):
        plan = [dict(cache[keys[b]], vmax=b) if keys[b] in cache else
                {"vmax": b, "group": 0, "split": 0, "warm_per_v": 0, "warm_add": 0} for b in BATCH_BUCKETS]
        ctx.set_batch_plan(plan)
        return plan, True
    plan, us = ctx.batch_autotune(u, v, edge_off, Vs, reps=reps)
    for d in plan:
        if d["vmax"] in present:
            cache[keys[d["vmax"]]] = {k: d[k] for k in ("group", "split", "warm_per_v", "warm_add")}
    _store(path, cache)
    return plan, False


def tune(ctx, u, v, V: int, path: str = DEFAULT_PATH, reps: int = 3, refresh: bool = False):
    """Applies the cached plan for this size bucket to `ctx`, tuning (and caching) on a miss.
    Returns (plan dict, hit)."""
    key = _key(u.numel(), V, ctx.device)
    cache = _load(path)
    if not refresh and key in cache:
        plan = cache[key]
        ctx.set_opts(M=plan["M"], fan_in=plan["fan_in"], block=plan["block"], warm_edges=plan["warm_edges"],
                     warm_block=plan.get("warm_block", 0))
        return plan, True
    plan = ctx.autotune(u, v, V, reps=reps)
    cache[key] = plan
    _store(path, cache)
    return plan, False
