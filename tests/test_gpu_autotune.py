"""The autotuner picks a plan by timing; tuned results stay exact; the JSON cache round-trips."""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu


def test_autotune_and_cache(cuda_lib, tmp_path):
    from paper_2108_07346_gb300 import autotune

    g = graphgen.workload("mid")
    u = torch.from_numpy(np.array(g.u)).cuda()
    v = torch.from_numpy(np.array(g.v)).cuda()
    ctx = cuda_lib.Context(device="cuda:0")
    path = str(tmp_path / "tune.json")
    plan, hit = autotune.tune(ctx, u, v, g.V, path=path, reps=2)
    assert not hit and plan["M"] >= 1 and plan["us_per_call"] > 0
    got = ctx.find(u, v, g.V).cpu().numpy()
    assert ctx.last_config()["M"] == plan["M"]
    assert got.tolist() == oracle.bridges(g.u, g.v, g.V, 16).tolist()
    ctx2 = cuda_lib.Context(device="cuda:0")
    plan2, hit2 = autotune.tune(ctx2, u, v, g.V, path=path)
    assert hit2 and plan2 == plan
    assert ctx2.find(u, v, g.V).cpu().numpy().tolist() == got.tolist()
