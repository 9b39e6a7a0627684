"""The oracle against a third-party library it shares nothing with (networkx, pure Python, CPU).

The paper's bridge test (Alg. 1), the Sec. 3 pipeline, the cut-vertex test and the
2-edge-connected components are compared with networkx's own routines on seeded random simple
graphs: sparse ones with many bridges and cut vertices, dense ones with few, and disconnected ones
with isolated vertices.  networkx's bridge finder is a chain decomposition and its cut-vertex
finder a separate DFS, written and tested independently of this project, so a dropped term, a
wrong comparison or a lost edge in the oracle would show up here.  networkx handles simple graphs
only; parallel edges and self-loops are pinned elsewhere (fixtures, closed forms, brute force).
Of the twelve planted mistakes of test_oracle_mutants, these three tests alone reject eleven; the
twelfth (the DFS skipping its parent by vertex instead of by edge) differs only on parallel edges.
Skipped where networkx is not installed.
"""
import numpy as np
import pytest

import oracle

nx = pytest.importorskip("networkx")


def _simple_graph(rng, V, p):
    """A seeded G(V, p) as a shuffled (u, v) list with random end order, plus the networkx graph."""
    a, b = np.triu_indices(V, 1)
    keep = rng.random(a.shape[0]) < p
    a, b = a[keep], b[keep]
    flip = rng.random(a.shape[0]) < 0.5
    u = np.where(flip, b, a).astype(np.int32)
    v = np.where(flip, a, b).astype(np.int32)
    order = rng.permutation(u.shape[0])
    u, v = u[order], v[order]
    G = nx.Graph()
    G.add_nodes_from(range(V))
    G.add_edges_from(zip(u.tolist(), v.tolist()))
    return u, v, G


def _cases():
    rng = np.random.default_rng(2108)
    for k in range(240):
        V = int(rng.integers(2, 160))
        # around the connectivity threshold (many bridges), sparse forests, and dense graphs
        p = [1.2 / V, 2.5 / V, np.log(V) / V, 0.3][k % 4]
        yield k, V, min(p, 1.0), rng


def _nx_bridges(G):
    return sorted((min(a, b), max(a, b)) for a, b in nx.bridges(G))


def test_bridges_match_networkx():
    n_bridges = 0
    for k, V, p, rng in _cases():
        u, v, G = _simple_graph(rng, V, p)
        ref = _nx_bridges(G)
        n_bridges += len(ref)
        assert [tuple(x) for x in oracle.dfs_bridges(u, v, V).tolist()] == ref, (k, V, p)
        assert [tuple(x) for x in oracle.chain_bridges(u, v, V).tolist()] == ref, (k, V, p)
        M = int(rng.integers(1, 9))
        assert [tuple(x) for x in oracle.bridges(u, v, V, M).tolist()] == ref, (k, V, p, M)
    assert n_bridges > 1000  # the cases do exercise the test, not only bridge-free graphs


def test_articulation_points_match_networkx():
    n_cut = 0
    for k, V, p, rng in _cases():
        u, v, G = _simple_graph(rng, V, p)
        ref = sorted(nx.articulation_points(G))
        n_cut += len(ref)
        assert oracle.articulation_points(u, v, V).tolist() == ref, (k, V, p)
    assert n_cut > 1000


def test_components_and_two_edge_components_match_networkx():
    for k, V, p, rng in _cases():
        u, v, G = _simple_graph(rng, V, p)
        c, lab = oracle.components(u, v, V)
        ref = list(nx.connected_components(G))
        assert c == len(ref), (k, V, p)
        for comp in ref:
            assert set(lab[list(comp)].tolist()) == {min(comp)}
        # 2-edge-connected components: the components left after deleting every bridge
        H = G.copy()
        H.remove_edges_from(nx.bridges(G))
        ref2 = list(nx.connected_components(H))
        c2, lab2 = oracle.two_edge_components(u, v, V)
        assert c2 == len(ref2), (k, V, p)
        for comp in ref2:
            assert set(lab2[list(comp)].tolist()) == {min(comp)}


def test_rooted_forest_matches_networkx_dfs():
    """oracle.rooted_forest (Alg. 1's numbering of a spanning forest: trees rooted at their minimum
    vertex and searched in root order, siblings by increasing id, one global counter) equals
    networkx's depth-first preorder, predecessors and subtree sizes, with each vertex's neighbours
    inserted in increasing order."""
    rng = np.random.default_rng(7346)
    for k in range(60):
        V = int(rng.integers(1, 400))
        # a random forest: vertex x > 0 hangs under a random earlier vertex unless it starts a tree
        perm = rng.permutation(V)
        edges = [(int(perm[x]), int(perm[rng.integers(0, x)])) for x in range(1, V) if rng.random() < 0.9]
        tu = np.array([a for a, _ in edges], np.int32)
        tv = np.array([b for _, b in edges], np.int32)
        parent, pre, size = oracle.rooted_forest(tu, tv, V)
        G = nx.Graph()
        G.add_nodes_from(range(V))
        G.add_edges_from(sorted((min(a, b), max(a, b)) for a, b in edges))  # neighbours in id order
        order, ref_parent, ref_size = [], np.full(V, -1), np.zeros(V, int)
        for r in sorted(min(c) for c in nx.connected_components(G)):
            order += list(nx.dfs_preorder_nodes(G, r))
            for y, x in nx.dfs_predecessors(G, r).items():
                ref_parent[y] = x
            T = nx.dfs_tree(G, r)
            for x in T:
                ref_size[x] = len(nx.descendants(T, x)) + 1
        ref_pre = np.empty(V, int)
        ref_pre[np.array(order, int)] = np.arange(V)
        assert pre.tolist() == ref_pre.tolist(), k
        assert parent.tolist() == ref_parent.tolist(), k
        assert size.tolist() == ref_size.tolist(), k


def _nx_of(g):
    G = nx.Graph()
    G.add_nodes_from(range(g.V))
    G.add_edges_from(zip(np.asarray(g.u).tolist(), np.asarray(g.v).tolist()))
    assert G.number_of_edges() == g.E  # no parallel edges or loops: networkx sees the same graph
    return G


def test_generated_workloads_match_networkx():
    """The seeded workloads: networkx's bridges equal the oracle's (Sec. 3 pipeline) and contain
    every planted bridge; on the small workload they are exactly the planted set."""
    import graphgen

    g = graphgen.workload("small")
    ref = _nx_bridges(_nx_of(g))
    assert ref == [tuple(x) for x in g.planted.tolist()]
    assert [tuple(x) for x in oracle.bridges(g.u, g.v, g.V, 16).tolist()] == ref
    specs = [graphgen.workload_spec("batched", 3, i) for i in range(24)] + \
        [graphgen.workload_spec("served", 4, i) for i in range(3)]
    checked = 0
    for spec in specs:
        g = graphgen.generate(spec)
        if g.E > 400_000:
            continue
        ref = _nx_bridges(_nx_of(g))
        assert [tuple(x) for x in oracle.bridges(g.u, g.v, g.V, 4).tolist()] == ref
        assert set(map(tuple, g.planted.tolist())) <= set(ref)
        checked += 1
    assert checked >= 20
