"""The one-block final stage (graphs of 2..4,096 vertices, bridges only) against the oracle and
against the grid final stage on the same inputs.

A context whose grid-barrier poll cap is set (a test knob; here far above anything a barrier
needs) keeps the cooperative grid stage, so the two forms of A5-A8 are compared call by call."""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctxs(cuda_lib):
    one = cuda_lib.Context(device="cuda:0")
    grid = cuda_lib.Context(device="cuda:0")
    grid.set_opts(test_barrier_polls=1 << 24)
    return one, grid


def run(ctx, u, v, V, M=1):
    du = torch.from_numpy(np.array(u, dtype=np.int32)).cuda()  # a copy: generator arrays are read-only
    dv = torch.from_numpy(np.array(v, dtype=np.int32)).cuda()
    return ctx.find(du, dv, V, M).cpu().numpy().tolist()


def cases():
    rng = np.random.default_rng(77)
    out = [
        ("one edge", np.array([0], np.int32), np.array([1], np.int32), 2),
        ("parallel pair", np.array([0, 1], np.int32), np.array([1, 0], np.int32), 2),
        ("no edges", np.zeros(0, np.int32), np.zeros(0, np.int32), 50),
        ("self-loops only", np.array([3, 3, 7], np.int32), np.array([3, 3, 7], np.int32), 9),
    ]
    star = np.arange(1, 100, dtype=np.int32)
    out.append(("star", np.zeros(99, np.int32), star, 100))
    for n in (4096, 4097):  # the largest one-block graph, and the first on the grid
        path_u = np.arange(n - 1, dtype=np.int32)
        out.append((f"path {n}", path_u, path_u + 1, n))
        par = (rng.random(n - 1) * np.arange(1, n)).astype(np.int32)
        out.append((f"random tree {n}", par, np.arange(1, n, dtype=np.int32), n))
    for t in range(6):  # multigraphs with many components, isolated vertices and self-loops
        V = int(rng.integers(2, 4097))
        E = int(rng.integers(0, 3 * V))
        u, v = graphgen.random_multigraph(7000 + t, V, E)
        out.append((f"multigraph {V}/{E}", u, v, V))
    g = graphgen.generate(graphgen.Spec(seed=41, n_clusters=3, core_vertices=1200, p=0.3, n_pendant=20,
                                        n_paths=6, path_min=2, path_max=9, n_trees=4, tree_min=3, tree_max=40))
    out.append(("clusters with pendant paths and trees", g.u, g.v, g.V))
    return out


@pytest.mark.parametrize("name,u,v,V", cases(), ids=lambda x: x if isinstance(x, str) else None)
def test_one_block_matches_grid_and_oracle(ctxs, name, u, v, V):
    one, grid = ctxs
    ref = oracle.dfs_bridges(u, v, V).tolist()
    assert run(one, u, v, V) == ref
    assert run(grid, u, v, V) == ref
    assert run(one, u, v, V, M=4) == ref  # several partitions merged before the stage


def test_one_block_enqueue_only_and_errors(ctxs):
    """The count lands on the device in the enqueue-only form; an id outside [0, V) reports
    ERANGE through the same count, and the next call on the context is exact again."""
    one, _ = ctxs
    u, v = graphgen.random_multigraph(123, 3000, 9000)
    ref = oracle.dfs_bridges(u, v, 3000).tolist()
    du = torch.from_numpy(np.array(u)).cuda()
    dv = torch.from_numpy(np.array(v)).cuda()
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    out = one.find(du, dv, 3000, 1, count_device=cnt)
    torch.cuda.synchronize()
    n = int(cnt.item())
    assert out[: 2 * n].view(n, 2).cpu().numpy().tolist() == ref
    bad_v = dv.clone()
    bad_v[17] = 3000
    one.find(du, bad_v, 3000, 1, count_device=cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == -2
    assert run(one, u, v, 3000) == ref
