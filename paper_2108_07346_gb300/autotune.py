"""Persistent cache of autotuning results (bridges_autotune) keyed by problem size and GPU.

Key: (round(log2 V), round(log2 E), number of SMs, device name).  A hit applies the cached plan
to the context without timing anything; a miss runs bridges_autotune on the caller's input and
stores the result.  The cache is a small JSON file.
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
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)
    return plan, False
