"""Input generators: determinism, normalisation and the sizes of the named workloads."""
import numpy as np

import graphgen


def test_deterministic_and_normalised():
    a = graphgen.workload("small")
    b = graphgen.workload("small")
    assert np.array_equal(a.u, b.u) and np.array_equal(a.v, b.v)
    assert (a.u < a.v).all() and a.u.min() >= 0 and a.v.max() < a.V
    # shuffled: edge order is not sorted by (u, v)
    k = a.u.astype(np.int64) * a.V + a.v
    assert not (np.diff(k) >= 0).all()
    c = graphgen.workload("small", seed=1)
    assert not np.array_equal(a.u, c.u)


def test_sizes():
    s = graphgen.workload("small")
    # 8 clusters of 256 with p = 0.5: 8 * C(256, 2) / 2 = 130,560 expected ER edges
    assert abs(s.n_er - 130560) < 5 * np.sqrt(8 * 32640 * 0.25)
    assert s.E == s.n_er + 7 + 40 + 40
    m = graphgen.workload("mid")
    assert abs(m.n_er - 64 * 130816 * 0.3) < 5 * np.sqrt(64 * 130816 * 0.21)
    assert m.V > 32768 + 1000


def test_unshuffled_identity_labels():
    g = graphgen.generate(graphgen.Spec(seed=3, n_clusters=1, core_vertices=10, p=1.0, shuffle=0, relabel=0))
    assert g.E == 45
    assert g.u.tolist() == [a for a in range(10) for b in range(a + 1, 10)]


def test_workload_specs_in_range():
    for i in range(200):
        s = graphgen.workload_spec("batched", 3, i)
        V = s.core_vertices + s.n_pendant
        assert 64 <= V <= 4096 and 0.1 <= s.p <= 0.9
        assert 2 <= s.n_clusters <= 8 and 1 <= s.n_clusters - 1 + s.n_pendant <= 32
        t = graphgen.workload_spec("served", 4, i)
        assert 256 <= t.core_vertices <= 65536 and 0.05 <= t.p <= 0.6


def test_batched_planted_subset():
    import oracle
    for i in range(20):
        g = graphgen.generate(graphgen.workload_spec("batched", 3, i))
        found = {tuple(x) for x in oracle.bridges(g.u, g.v, g.V, 4).tolist()}
        assert {tuple(x) for x in g.planted.tolist()} <= found


def test_rmat_is_seeded_skewed_and_in_range():
    u, v = graphgen.rmat(5, 12, 60000)
    u2, v2 = graphgen.rmat(5, 12, 60000)
    assert np.array_equal(u, u2) and np.array_equal(v, v2)
    assert u.min() >= 0 and v.min() >= 0 and u.max() < 4096 and v.max() < 4096
    deg = np.bincount(np.concatenate([u, v]), minlength=4096)
    assert deg.max() > 50 * np.median(deg[deg > 0])  # hubs
    assert not np.array_equal(graphgen.rmat(6, 12, 60000)[0], u)
    # the uniform quadrant mix is a uniform random multigraph: no hubs
    uu, vv = graphgen.rmat(5, 12, 60000, 0.25, 0.25, 0.25)
    d2 = np.bincount(np.concatenate([uu, vv]), minlength=4096)
    assert d2.max() < 3 * d2.mean()


def test_layout_matches_generated_graph():
    """The host layout (sizes, structural edges, planted bridges) that the device form of the
    generator starts from is the generated graph's."""
    import ctypes

    lib = graphgen._load()
    lib.gg_layout_make.restype = ctypes.POINTER(graphgen._Layout)
    lib.gg_layout_make.argtypes = [ctypes.POINTER(graphgen._Spec)]
    lib.gg_layout_free.argtypes = [ctypes.POINTER(graphgen._Layout)]
    for spec in [graphgen.WORKLOADS["small"], graphgen.workload_spec("served", 4, 2),
                 graphgen.workload_spec("batched", 3, 5)]:
        g = graphgen.generate(spec)
        h = lib.gg_layout_make(ctypes.byref(spec._c()))
        L = h.contents
        assert L.V == g.V and L.n_struct == g.E - g.n_er
        pl = np.ctypeslib.as_array(L.planted, shape=(2 * L.n_planted,)).reshape(-1, 2)
        assert np.array_equal(pl, g.planted)
        lib.gg_layout_free(h)
