"""2-edge-connected components and incremental edge additions against the oracle."""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.array(a, dtype=np.int32)).cuda()


def test_two_edge_components(cuda_lib):
    ctx = cuda_lib.Context(device="cuda:0")
    cases = [graphgen.random_multigraph(70000 + t, 40 + 30 * t, (40 + 30 * t) * (1 + t % 3)) + (40 + 30 * t,)
             for t in range(20)]
    for name in ("small", "mid"):
        g = graphgen.workload(name)
        cases.append((np.array(g.u), np.array(g.v), g.V))
    for u, v, V in cases:
        n, lab = ctx.two_edge_components(dev(u), dev(v), V, 3)
        rn, rlab = oracle.two_edge_components(u, v, V)
        assert n == rn and lab.cpu().numpy().tolist() == rlab.tolist()


def test_incremental_matches_oracle_on_the_union(cuda_lib):
    rng = np.random.default_rng(9)
    inc = cuda_lib.Incremental(device="cuda:0")
    g = graphgen.workload("small")
    u, v = np.array(g.u), np.array(g.v)
    V = g.V
    got = inc.reset(dev(u), dev(v), V, 4).cpu().numpy()
    assert got.tolist() == g.planted.tolist()
    allu, allv = u, v
    for step in range(8):
        k = int(rng.integers(1, 30))
        yu = rng.integers(0, V, k).astype(np.int32)
        yv = rng.integers(0, V, k).astype(np.int32)
        if step == 3:  # parallel copies of current bridges: they stop being bridges
            b = oracle.dfs_bridges(allu, allv, V)[:5]
            yu, yv = b[:, 0].copy(), b[:, 1].copy()
        if step == 5:  # pendant vertices become leaves of new paths: nothing changes for others
            yu, yv = np.array([0, 0], np.int32), np.array([0, 0], np.int32)  # self-loops
        allu = np.concatenate([allu, yu])
        allv = np.concatenate([allv, yv])
        got = inc.add(dev(yu), dev(yv)).cpu().numpy()
        assert got.tolist() == oracle.dfs_bridges(allu, allv, V).tolist(), step
        assert inc.certificate_size() <= 2 * (V - 1)
        n, lab = inc.two_edge_components()
        rn, rlab = oracle.two_edge_components(allu, allv, V)
        assert n == rn and lab.cpu().numpy().tolist() == rlab.tolist()


def test_incremental_bad_ids_leave_state_unchanged(cuda_lib):
    inc = cuda_lib.Incremental(device="cuda:0")
    n = 50
    a = np.arange(n - 1, dtype=np.int32)
    assert len(inc.reset(dev(a), dev(a + 1), n)) == n - 1
    with pytest.raises(cuda_lib.BridgesError) as ei:
        inc.add(dev([0, 3]), dev([49, 99]))  # 99 is out of range: the whole batch is rejected
    assert ei.value.code == -2
    assert len(inc.add(dev([0]), dev([49]))) == 0  # closing the cycle removes every bridge
