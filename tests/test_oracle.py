"""Pins the CPU oracle to facts that do not come from the oracle itself.

* hand-derived fixtures (tests/golden, Sec. 1 definition);
* closed forms: trees, paths, cycles, complete graphs, doubled edges;
* agreement of three independent methods (Alg. 1 DFS, Schmidt chains, the definition by
  brute force) and of the Sec. 3 pipeline for many M on random multigraphs with V <= 64;
* the generators' planted bridges (known by construction);
* certificate invariants from Sec. 3 and Lemma 1.

A plausible mistake in the oracle fails at least one of these: a dropped F' (Alg. 2) changes
bridges on any cycle; a vertex-based parent skip (Alg. 1) makes a doubled edge a bridge; a
">=" for ">" in the low/disc test makes cycle edges bridges; a lost merge partner (Sec. 3)
changes components; a wrong partition bound loses edges.  test_oracle_mutants builds these
mistakes and others into the oracle's C source and checks that a pin here rejects each one.
"""
import itertools

import numpy as np
import pytest

import graphgen
import oracle
from conftest import golden_names, load_golden, load_golden_cuts

ALL_METHODS = {
    "dfs": lambda u, v, V: oracle.dfs_bridges(u, v, V),
    "chain": lambda u, v, V: oracle.chain_bridges(u, v, V),
    "brute": lambda u, v, V: oracle.brute_bridges(u, v, V),
    "pipe1": lambda u, v, V: oracle.bridges(u, v, V, 1),
    "pipe2": lambda u, v, V: oracle.bridges(u, v, V, 2),
    "pipe3": lambda u, v, V: oracle.bridges(u, v, V, 3),
    "pipe5": lambda u, v, V: oracle.bridges(u, v, V, 5),
    "pipe16": lambda u, v, V: oracle.bridges(u, v, V, 16),
    "pipe64": lambda u, v, V: oracle.bridges(u, v, V, 64),
}


def as_set(b):
    return {tuple(x) for x in np.asarray(b).reshape(-1, 2).tolist()}


@pytest.mark.parametrize("name", golden_names())
@pytest.mark.parametrize("method", sorted(ALL_METHODS))
def test_golden(name, method):
    u, v, V, exp = load_golden(name)
    got = ALL_METHODS[method](u, v, V)
    assert got.tolist() == exp.tolist()


@pytest.mark.parametrize("name", golden_names())
def test_golden_cut_vertices(name):
    """The fixtures' hand-derived cut vertices: Tarjan's low/disc test, the definition (brute
    force) and the block-certificate restatement all give exactly them."""
    u, v, V, _ = load_golden(name)
    exp = load_golden_cuts(name)
    assert exp is not None, "every fixture carries its cut vertices"
    assert oracle.articulation_points(u, v, V).tolist() == exp.tolist()
    assert oracle.brute_articulation(u, v, V).tolist() == exp.tolist()
    assert sorted(oracle.block_certificate(u, v, V)[2].tolist()) == exp.tolist()


def _random_tree(rng, n):
    par = [int(rng.integers(0, i)) for i in range(1, n)]
    return np.array(par, np.int32), np.arange(1, n, dtype=np.int32)


@pytest.mark.parametrize("method", sorted(ALL_METHODS))
def test_closed_forms(method):
    f = ALL_METHODS[method]
    rng = np.random.default_rng(11)
    for n in [1, 2, 3, 7, 33, 64]:
        # random recursive tree: every edge is a bridge
        u, v = _random_tree(rng, n)
        assert len(f(u, v, n)) == n - 1
        # path of n-1 edges: n-1 bridges
        u = np.arange(0, n - 1, dtype=np.int32)
        v = u + 1
        got = f(u, v, n)
        assert got.tolist() == np.stack([u, v], 1).tolist()
        # the same path with every edge doubled: no bridges
        assert len(f(np.concatenate([u, v]), np.concatenate([v, u]), n)) == 0
        if n >= 3:
            # cycle: no bridges
            u = np.arange(n, dtype=np.int32)
            v = (u + 1) % n
            assert len(f(u, v, n)) == 0
            # complete graph: no bridges
            pairs = np.array(list(itertools.combinations(range(n), 2)), np.int32)
            assert len(f(pairs[:, 0], pairs[:, 1], n)) == 0
            # star: every edge is a bridge
            u = np.zeros(n - 1, np.int32)
            v = np.arange(1, n, dtype=np.int32)
            assert len(f(u, v, n)) == n - 1
    # no edges / no vertices
    e = np.zeros(0, np.int32)
    assert len(f(e, e, 0)) == 0
    assert len(f(e, e, 5)) == 0
    # one self-loop
    assert len(f(np.array([0], np.int32), np.array([0], np.int32), 1)) == 0


def test_random_multigraphs_agree():
    """Thousands of random multigraphs (self-loops and duplicates included), V <= 64."""
    rng = np.random.default_rng(5)
    for t in range(1500):
        V = int(rng.integers(1, 65))
        E = int(rng.integers(0, 3 * V + 2))
        u, v = graphgen.random_multigraph(1000 + t, V, E)
        ref = oracle.brute_bridges(u, v, V)
        for name, f in ALL_METHODS.items():
            if name == "brute":
                continue
            got = f(u, v, V)
            assert got.tolist() == ref.tolist(), (t, name, V, E)


def test_sparse_random_trees_plus_edges():
    """Near-tree graphs, where most edges are bridges and the low/disc test decides each one."""
    rng = np.random.default_rng(6)
    for t in range(300):
        n = int(rng.integers(2, 65))
        u, v = _random_tree(rng, n)
        k = int(rng.integers(0, 4))
        xu = rng.integers(0, n, k).astype(np.int32)
        xv = rng.integers(0, n, k).astype(np.int32)
        u = np.concatenate([u, xu])
        v = np.concatenate([v, xv])
        perm = rng.permutation(len(u))
        u, v = u[perm], v[perm]
        ref = oracle.brute_bridges(u, v, n)
        for M in (1, 2, 7):
            assert oracle.bridges(u, v, n, M).tolist() == ref.tolist()
        assert oracle.chain_bridges(u, v, n).tolist() == ref.tolist()


@pytest.mark.parametrize("name", ["small", "mid"])
def test_planted_bridges(name):
    """The generators plant bridges whose status is known by construction."""
    g = graphgen.workload(name)
    got = oracle.bridges(g.u, g.v, g.V, 16)
    # planted subset of found always; equal here because the ER clusters are 2-edge-connected
    assert as_set(g.planted) <= as_set(got)
    assert got.tolist() == g.planted.tolist()
    assert oracle.chain_bridges(g.u, g.v, g.V).tolist() == got.tolist()


def test_planted_counts_small():
    """The small workload: 40 pendant vertices are bridges, and of the 7 cluster-tree edges only
    those no inter-cluster pair covers (here exactly one, computed on the cluster tree)."""
    g = graphgen.workload("small")
    assert g.V == 2048 + 40
    assert len(g.planted) == 41


def _cert_invariants(u, v, V, ids, f1, M):
    ids = np.asarray(ids)
    # subset of the input, each input edge at most once (ids distinct)
    assert len(np.unique(ids)) == len(ids)
    assert ids.min(initial=0) >= 0 and ids.max(initial=-1) < len(u)
    cu, cv = u[ids], v[ids]
    c, lab = oracle.components(u, v, V)
    c2, lab2 = oracle.components(cu, cv, V)
    # same connected components
    assert c == c2 and np.array_equal(lab, lab2)
    # Lemma 1 (per component form): |S| <= 2(V - c)
    assert len(ids) <= 2 * (V - c)
    # F is a spanning forest: V - c edges, and acyclic (components of F equal those of S)
    assert int(f1.sum()) == V - c
    cf, labf = oracle.components(cu[f1], cv[f1], V)
    assert cf == c and np.array_equal(labf, lab)
    # same bridges (Sec. 3 "G(V, E u Y) = G(V, S u Y)" with Y empty)
    assert oracle.dfs_bridges(cu, cv, V).tolist() == oracle.dfs_bridges(u, v, V).tolist()


def test_certificate_invariants_random():
    rng = np.random.default_rng(7)
    for t in range(300):
        V = int(rng.integers(1, 80))
        E = int(rng.integers(0, 8 * V))
        u, v = graphgen.random_multigraph(5000 + t, V, E)
        ids, f1 = oracle.certificate(u, v, V)
        _cert_invariants(u, v, V, ids, f1, 1)
        for M in (2, 3, 8):
            ids, f1, pm = oracle.pipeline_certificate(u, v, V, M)
            _cert_invariants(u, v, V, ids, f1, M)
            # Q = 1 + ceil(log2 M) phases, every intermediate |X_i| <= 2(V - 1)
            assert len(pm) == 1 + int(np.ceil(np.log2(M)))
            assert (pm <= 2 * max(V - 1, 0)).all()


@pytest.mark.parametrize("M", [1, 4, 16, 33])
def test_certificate_invariants_small_workload(M):
    g = graphgen.workload("small")
    ids, f1, pm = oracle.pipeline_certificate(g.u, g.v, g.V, M)
    _cert_invariants(g.u, g.v, g.V, ids, f1, M)


def test_certificate_cut_property():
    """For every vertex set X, |delta_S(X)| >= min(|delta_E(X)|, 2) (the reading of the Sec. 3
    certificate definition used throughout); checked exhaustively over all cuts of small graphs."""
    rng = np.random.default_rng(8)
    for t in range(60):
        V = int(rng.integers(2, 11))
        E = int(rng.integers(0, 4 * V))
        u, v = graphgen.random_multigraph(9000 + t, V, E)
        ids, _ = oracle.certificate(u, v, V)
        cu, cv = u[ids], v[ids]
        for mask in range(1, 1 << (V - 1)):
            side = np.array([(mask >> i) & 1 for i in range(V)], bool)
            de = int(np.sum(side[u] != side[v]))
            ds = int(np.sum(side[cu] != side[cv]))
            assert ds >= min(de, 2)


def test_dropping_second_forest_is_caught():
    """Planted mistake (in the oracle's inputs, on the CPU): keeping only F of Alg. 2 turns every
    cycle edge into a 'bridge', which the invariant 'bridges(S) == bridges(E)' rejects."""
    n = 6
    u = np.arange(n, dtype=np.int32)
    v = (u + 1) % n
    ids, f1 = oracle.certificate(u, v, n)
    only_f = ids[f1]
    assert len(oracle.dfs_bridges(u[only_f], v[only_f], n)) == n - 1
    assert len(oracle.dfs_bridges(u[ids], v[ids], n)) == 0


def test_invalid_ids_rejected():
    with pytest.raises(ValueError):
        oracle.bridges(np.array([0], np.int32), np.array([5], np.int32), 3)
    with pytest.raises(ValueError):
        oracle.dfs_bridges(np.array([-1], np.int32), np.array([0], np.int32), 3)


def _brute_2ecc(u, v, V):
    """Definition: x and y are 2-edge-connected iff they stay connected after deleting any one
    edge (Menger: two edge-disjoint paths).  Labels = min vertex of each class."""
    E = len(u)

    def comp(skip):
        par = list(range(V))

        def f(x):
            while par[x] != x:
                par[x] = par[par[x]]
                x = par[x]
            return x

        for e in range(E):
            if e != skip:
                a, b = f(int(u[e])), f(int(v[e]))
                if a != b:
                    par[max(a, b)] = min(a, b)
        return [f(x) for x in range(V)]

    base = comp(-1)
    cut = [comp(e) for e in range(E)]
    lab = []
    for x in range(V):
        cls = [y for y in range(V) if base[y] == base[x] and all(c[x] == c[y] for c in cut)]
        lab.append(min(cls))
    return lab


def test_two_edge_components_brute():
    for t in range(200):
        rng = np.random.default_rng(600 + t)
        V = int(rng.integers(1, 11))
        E = int(rng.integers(0, 2 * V + 3))
        u, v = graphgen.random_multigraph(8800 + t, V, E)
        c, lab = oracle.two_edge_components(u, v, V)
        assert lab.tolist() == _brute_2ecc(u, v, V), (t, V, E)
        assert c == len(set(lab.tolist()))


def test_two_edge_components_closed_forms():
    u, v, V, _ = load_golden("barbell.txt")
    c, lab = oracle.two_edge_components(u, v, V)
    assert lab.tolist() == [0, 0, 0, 0, 4, 4, 4, 4, 8] and c == 3
    n = 9
    a = np.arange(n - 1, dtype=np.int32)
    c, lab = oracle.two_edge_components(a, a + 1, n)  # a path: every vertex alone
    assert c == n and lab.tolist() == list(range(n))


def test_articulation_points_brute_and_closed_forms():
    rng = np.random.default_rng(41)
    for t in range(1000):
        V = int(rng.integers(1, 40))
        E = int(rng.integers(0, 3 * V + 2))
        u, v = graphgen.random_multigraph(12000 + t, V, E)
        ref = oracle.brute_articulation(u, v, V).tolist()
        assert oracle.articulation_points(u, v, V).tolist() == ref, t
        if t % 10 == 0:
            assert [x for x in range(V) if oracle.is_articulation(u, v, V, x)] == ref, t
    n = 12
    a = np.arange(n - 1, dtype=np.int32)
    assert oracle.articulation_points(a, a + 1, n).tolist() == list(range(1, n - 1))  # path
    assert oracle.articulation_points(np.zeros(n - 1, np.int32), a + 1, n).tolist() == [0]  # star
    c = np.arange(n, dtype=np.int32)
    assert len(oracle.articulation_points(c, (c + 1) % n, n)) == 0  # cycle
    # two triangles sharing vertex 2 (bow tie): 2 is the only cut vertex
    u = np.array([0, 1, 2, 2, 3, 4], np.int32)
    v = np.array([1, 2, 0, 3, 4, 2], np.int32)
    assert oracle.articulation_points(u, v, 5).tolist() == [2]
    # a random tree: exactly the vertices of degree >= 2
    rng = np.random.default_rng(43)
    for n in (2, 3, 50, 3000):
        par = (rng.random(n - 1) * np.arange(1, n)).astype(np.int32)
        ch = np.arange(1, n, dtype=np.int32)
        deg = np.bincount(np.concatenate([par, ch]), minlength=n)
        assert oracle.articulation_points(par, ch, n).tolist() == np.flatnonzero(deg >= 2).tolist()
        assert oracle.block_certificate(par, ch, n)[2].tolist() == np.flatnonzero(deg >= 2).tolist()
    # complete graph K_6 with every edge doubled and self-loops: none
    a, b = np.triu_indices(6, 1)
    u = np.concatenate([a, b, np.arange(6)]).astype(np.int32)
    v = np.concatenate([b, a, np.arange(6)]).astype(np.int32)
    assert len(oracle.articulation_points(u, v, 6)) == 0 and len(oracle.block_certificate(u, v, 6)[2]) == 0
    # barbell fixture: the path 3-8-4 makes 3, 8 and 4 cut vertices
    bu, bv, bV, _ = load_golden("barbell.txt")
    assert oracle.articulation_points(bu, bv, bV).tolist() == [3, 4, 8]


def test_block_certificate_articulation_points():
    """The fundamental-cycle classes over a spanning forest give the cut vertices of the
    definition; T plus the kept edges keeps them, with at most V - 1 kept non-tree edges."""
    rng = np.random.default_rng(42)
    for t in range(1500):
        V = int(rng.integers(1, 40))
        E = int(rng.integers(0, 6 * V + 2))
        u, v = graphgen.random_multigraph(13000 + t, V, E)
        ids, tr, pts = oracle.block_certificate(u, v, V)
        brute = oracle.brute_articulation(u, v, V).tolist()
        assert pts.tolist() == brute, t
        c, _ = oracle.components(u, v, V)
        assert int(tr.sum()) == V - c and int((~tr).sum()) <= max(V - 1, 0)
        assert oracle.brute_articulation(u[ids], v[ids], V).tolist() == brute, t
        assert len(np.unique(ids)) == len(ids)


def test_arbitrary_forests_do_not_keep_articulation_points():
    """Why a separate certificate: the union-find forests of Alg. 2 keep bridges but not cut
    vertices.  A 4-cycle 0-1-2-3 with chord 1-3 and a pendant path through 0: an Alg. 2
    certificate may drop edges so that a non-cut vertex becomes one."""
    found = False
    for t in range(300):
        rng = np.random.default_rng(t)
        V = 7
        u, v = graphgen.random_multigraph(14000 + t, V, 14)
        ids, f1 = oracle.certificate(u, v, V)
        if oracle.articulation_points(u[ids], v[ids], V).tolist() != oracle.articulation_points(u, v, V).tolist():
            found = True
            break
    assert found


def test_streaming_certificate_equals_two_pass():
    """Alg. 2 taken as one streaming pass (each edge to F, else to F') -- the GPU's form -- gives
    the same certificate as the two passes (F over the list, then F' over what F rejected)."""
    for t in range(300):
        rng = np.random.default_rng(15000 + t)
        V = int(rng.integers(1, 50))
        E = int(rng.integers(0, 8 * V))
        u, v = graphgen.random_multigraph(15000 + t, V, E)
        ids2, f2 = oracle.certificate(u, v, V)
        ids1, f1 = oracle.certificate_stream(u, v, V)
        assert sorted(zip(ids1.tolist(), f1.tolist())) == sorted(zip(ids2.tolist(), f2.tolist())), t


def _check_rooted_forest(tu, tv, V, parent, pre, size, key):
    """The rooted forest by its definitions, not by a second search: the parent edges are the
    input edges, every root is its component's minimum vertex, sizes count the vertices whose
    root path passes through each vertex, and the numbering is the preorder for the sibling
    order `key` (a vertex, then its children's subtrees in key order, the trees consecutive in
    increasing order of their roots)."""
    tu, tv = np.asarray(tu), np.asarray(tv)
    got = {(min(x, int(p)), max(x, int(p))) for x, p in enumerate(parent) if p >= 0}
    assert got == {(min(a, b), max(a, b)) for a, b in zip(tu.tolist(), tv.tolist())}
    _, comp = oracle.components(tu, tv, V)
    roots = [x for x in range(V) if parent[x] < 0]
    assert roots == sorted(set(comp.tolist()))  # one root per component, its minimum vertex
    count = np.zeros(V, np.int64)
    for y in range(V):  # brute force: y counts for every vertex on its root path
        x, steps = y, 0
        while x >= 0:
            count[x] += 1
            x = parent[x]
            steps += 1
            assert steps <= V
    assert count.tolist() == np.asarray(size).tolist()
    kids = [[] for _ in range(V)]
    for x in range(V):
        if parent[x] >= 0:
            kids[parent[x]].append(x)
    at = 0
    for r in roots:
        assert pre[r] == at
        at += size[r]
    for p in range(V):
        nxt = pre[p] + 1
        for c in sorted(kids[p], key=lambda c: key[c]):
            assert pre[c] == nxt
            nxt += size[c]
        assert nxt == pre[p] + size[p]
    assert sorted(np.asarray(pre).tolist()) == list(range(V))


def test_rooted_forest_closed_forms():
    rng = np.random.default_rng(81)
    n = 50
    a = np.arange(n - 1)
    perm = rng.permutation(n - 1)
    flip = rng.random(n - 1) < 0.5
    pu, pv = np.where(flip, a + 1, a)[perm], np.where(flip, a, a + 1)[perm]
    parent, pre, size = oracle.rooted_forest(pu, pv, n)  # path in shuffled order and direction
    assert parent.tolist() == [-1] + list(range(n - 1))
    assert pre.tolist() == list(range(n)) and size.tolist() == list(range(n, 0, -1))
    c = 7  # star around vertex 7: the root is leaf 0, then the centre, then the other leaves
    leaves = np.array([x for x in range(n) if x != c])
    parent, pre, size = oracle.rooted_forest(np.full(n - 1, c), leaves, n)
    assert parent[0] == -1 and parent[c] == 0 and all(parent[x] == c for x in leaves[1:])
    assert size[0] == n and size[c] == n - 1 and pre[c] == 1
    assert [pre[x] for x in leaves[1:]] == list(range(2, n))
    parent, pre, size = oracle.rooted_forest([], [], 5)  # no edges: five one-vertex trees
    assert parent.tolist() == [-1] * 5 and pre.tolist() == list(range(5)) and size.tolist() == [1] * 5
    for bad in (([0, 1, 2], [1, 2, 0], 3), ([0, 0], [1, 1], 2), ([0], [3], 3)):
        with pytest.raises(ValueError):
            oracle.rooted_forest(*bad)


def test_rooted_forest_against_definitions():
    rng = np.random.default_rng(82)
    for t in range(60):
        V = int(rng.integers(1, 120))
        par = [int(rng.integers(0, x)) if (x and rng.random() < 0.8) else -1 for x in range(V)]
        relabel = rng.permutation(V)
        edges = [(int(relabel[x]), int(relabel[p])) for x, p in enumerate(par) if p >= 0]
        rng.shuffle(edges)
        tu = np.array([e[0] for e in edges], np.int32)
        tv = np.array([e[1] for e in edges], np.int32)
        key = rng.permutation(V) if t % 2 else None
        parent, pre, size = oracle.rooted_forest(tu, tv, V, key)
        _check_rooted_forest(tu, tv, V, parent, pre, size, np.arange(V) if key is None else key)
