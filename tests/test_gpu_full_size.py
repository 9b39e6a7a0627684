"""Full-size parity in the benchmark's launch configuration.

* large: the 1.07 G-edge workload, autotuned plan (as bench.py runs it), against the oracle's
  Sec. 3 pipeline on the whole graph (single-threaded C, several seconds) and the planted set.
* batched: all 4,096 graphs of the batched workload in one launch, each against the oracle.
"""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def test_large_workload_full_size(cuda_lib):
    g = graphgen.workload("large")
    du = torch.from_numpy(np.array(g.u)).cuda()
    dv = torch.from_numpy(np.array(g.v)).cuda()
    ctx = cuda_lib.Context(device="cuda:0", profile=True)
    plan = ctx.autotune(du, dv, g.V, reps=1)
    got = ctx.find(du, dv, g.V).cpu().numpy()
    assert ctx.last_config()["M"] == plan["M"]
    ref = oracle.bridges(g.u, g.v, g.V, max(plan["M"], 1))
    assert got.tolist() == ref.tolist()
    assert got.tolist() == g.planted.tolist()
    # the paper-like plan with a real merge tree gives the same exact set
    assert ctx.find(du, dv, g.V, 8).cpu().numpy().tolist() == ref.tolist()


def test_batched_workload_full_size(cuda_lib):
    import bench

    u, v, off, Vs, planted = bench.make_batch(3, 4096)
    ctx = cuda_lib.Context(device="cuda:0")
    out, counts, out_off = ctx.find_batched(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), off, Vs)
    out = out.cpu().numpy()
    counts = counts.cpu().numpy()
    for gi in range(len(Vs)):
        a, b = off[gi], off[gi + 1]
        ref = oracle.dfs_bridges(u[a:b], v[a:b], int(Vs[gi]))
        n = int(counts[gi])
        assert n == len(ref), gi
        assert out[out_off[gi]: out_off[gi] + 2 * n].tolist() == ref.ravel().tolist(), gi


def test_large_workload_articulation_points(cuda_lib):
    """The 1.07 G-edge workload through bridges_articulation_points in the benchmark's launch
    configuration.  By construction its blocks are the dense cluster (with the two-edge vertices)
    and the planted bridges, so the cut vertices are the bridge ends with another edge; a sample
    is also checked against the definition on the whole graph (one vertex deleted at a time)."""
    g = graphgen.workload("large")
    du = torch.from_numpy(np.array(g.u)).cuda()
    dv = torch.from_numpy(np.array(g.v)).cuda()
    ctx = cuda_lib.Context(device="cuda:0", profile=True)
    ctx.autotune(du, dv, g.V, reps=1)
    pts, br = ctx.articulation_points(du, dv, g.V, with_bridges=True)
    pts = pts.cpu().numpy()
    assert br.cpu().numpy().tolist() == g.planted.tolist()
    loop = g.u == g.v
    deg = np.bincount(np.concatenate([g.u[~loop], g.v[~loop]]), minlength=g.V)
    ends = np.unique(g.planted.ravel())
    assert pts.tolist() == ends[deg[ends] >= 2].tolist()
    inside = np.setdiff1d(np.arange(g.V), pts)
    rng = np.random.default_rng(64)
    for x in [int(pts[0]), int(pts[-1]), int(rng.choice(inside))]:
        assert oracle.is_articulation(g.u, g.v, g.V, x) == (x in set(pts.tolist())), x
