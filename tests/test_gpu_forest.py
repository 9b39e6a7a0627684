"""Parity of the final stage's rooted forest (bridges_rooted_forest, through the C ABI) with the
CPU oracle's depth-first numbering (oracle.rooted_forest).

For each tree rooted at its minimum vertex, the parents and the subtree sizes are unique and
must match bit for bit.  The preorder is unique once the order of siblings is fixed; the GPU's
order follows its adjacency lists, which are built with atomics, so the oracle replays the DFS
with the siblings in the GPU's order and must reproduce every number exactly.  Either way, the
trees must take consecutive ranges in increasing order of their roots.
"""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.array(a, dtype=np.int32)).to("cuda:0")


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    return cuda_lib.Context(device="cuda:0")


def check(ctx, tu, tv, V):
    parent, pre, size = (t.cpu().numpy() for t in ctx.rooted_forest(dev(tu), dev(tv), V))
    ref_parent, ref_pre, ref_size = oracle.rooted_forest(tu, tv, V, child_key=pre)
    assert parent.tolist() == ref_parent.tolist()
    assert size.tolist() == ref_size.tolist()
    assert pre.tolist() == ref_pre.tolist()
    return parent, pre, size


def random_forest(rng, V, p_edge):
    """A random recursive forest on V vertices (each vertex joins an earlier one with
    probability p_edge), vertex ids relabelled, edges shuffled and randomly oriented."""
    relabel = rng.permutation(V)
    edges = [(int(relabel[x]), int(relabel[rng.integers(0, x)])) for x in range(1, V) if rng.random() < p_edge]
    rng.shuffle(edges)
    e = np.array(edges, np.int32).reshape(-1, 2)
    flip = rng.random(len(e)) < 0.5
    return np.where(flip, e[:, 1], e[:, 0]), np.where(flip, e[:, 0], e[:, 1])


def test_random_forests(ctx):
    rng = np.random.default_rng(91)
    for t in range(24):
        V = int(rng.integers(1, 3000)) if t < 16 else int(rng.integers(3000, 60000))
        tu, tv = random_forest(rng, V, float(rng.choice([1.0, 0.97, 0.6, 0.1])))
        check(ctx, tu, tv, V)


def test_shapes(ctx):
    n = 100_000
    a = np.arange(n - 1, dtype=np.int32)
    perm = np.random.default_rng(92).permutation(n - 1)
    parent, pre, size = check(ctx, a[perm] + 1, a[perm], n)  # a path: one deep tree
    assert pre.tolist() == list(range(n))
    parent, pre, size = check(ctx, np.full(n - 1, 5, np.int32), np.delete(np.arange(n, dtype=np.int32), 5), n)
    assert parent[5] == 0 and size[0] == n  # a star rooted at its leaf 0
    k = 30_000  # a caterpillar: a spine with one leaf on every spine vertex
    spine = np.arange(k - 1, dtype=np.int32)
    check(ctx, np.concatenate([spine, np.arange(k, dtype=np.int32)]),
          np.concatenate([spine + 1, np.arange(k, 2 * k, dtype=np.int32)]), 2 * k)


@pytest.mark.parametrize("name", ["small", "mid"])
def test_certificate_forests(ctx, name):
    """The spanning forest F of a real certificate (bridges_certificate), as the bridge path
    roots it."""
    g = graphgen.workload(name)
    cu, cv, tree = ctx.certificate(dev(g.u), dev(g.v), g.V, 4)
    tree = tree.cpu().numpy().astype(bool)
    check(ctx, cu.cpu().numpy()[tree], cv.cpu().numpy()[tree], g.V)


def test_edge_cases(ctx, cuda_lib):
    e = np.zeros(0, np.int32)
    assert all(len(t) == 0 for t in ctx.rooted_forest(dev(e), dev(e), 0))
    parent, pre, size = check(ctx, e, e, 1)
    assert parent.tolist() == [-1] and pre.tolist() == [0] and size.tolist() == [1]
    parent, pre, size = check(ctx, e, e, 7)  # no edges: seven one-vertex trees in id order
    assert pre.tolist() == list(range(7))
    check(ctx, np.array([3], np.int32), np.array([1], np.int32), 4)
    with pytest.raises(cuda_lib.BridgesError) as ei:  # an id outside [0, V)
        ctx.rooted_forest(dev([0, 1]), dev([1, 9]), 5)
    assert ei.value.code == -2
    with pytest.raises(cuda_lib.BridgesError) as ei:  # more edges than a forest on V vertices has
        ctx.rooted_forest(dev([0, 1, 2]), dev([1, 2, 0]), 3)
    assert ei.value.code == -1
