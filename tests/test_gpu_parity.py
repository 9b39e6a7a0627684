"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bridge sets are unique, so the sorted (a<b) list must match the oracle bit for bit.  Forests
are not unique (concurrent union-find), so certificates are checked by their invariants:
|S| <= 2(V - c), S a sub-multiset of the input, same components, same bridges.
"""
import numpy as np
import pytest
import torch

import graphgen
import oracle
from conftest import golden_names, load_golden

pytestmark = pytest.mark.gpu


def dev_edges(u, v):
    d = torch.device("cuda", 0)
    return (torch.from_numpy(np.array(u, dtype=np.int32)).to(d),
            torch.from_numpy(np.array(v, dtype=np.int32)).to(d))


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    return cuda_lib.Context(device="cuda:0")


def gpu_bridges(ctx, u, v, V, M=0):
    du, dv = dev_edges(u, v)
    return ctx.find(du, dv, V, M).cpu().numpy()


@pytest.mark.parametrize("name", golden_names())
@pytest.mark.parametrize("M", [1, 2, 5])
def test_golden(ctx, name, M):
    u, v, V, exp = load_golden(name)
    assert gpu_bridges(ctx, u, v, V, M).tolist() == exp.tolist()


def test_random_multigraphs(ctx):
    rng = np.random.default_rng(21)
    for t in range(400):
        V = int(rng.integers(1, 65))
        E = int(rng.integers(0, 4 * V + 2))
        u, v = graphgen.random_multigraph(20000 + t, V, E)
        ref = oracle.brute_bridges(u, v, V)
        M = int(rng.choice([1, 2, 3, 7, 16, 200]))
        got = gpu_bridges(ctx, u, v, V, M)
        assert got.tolist() == ref.tolist(), (t, V, E, M)


def test_random_sparse_mid(ctx):
    """Sparse random graphs (many bridges, many components) spanning several tiles."""
    rng = np.random.default_rng(22)
    for t in range(30):
        V = int(rng.integers(100, 5000))
        E = int(rng.integers(V // 2, 2 * V))
        u, v = graphgen.random_multigraph(30000 + t, V, E)
        ref = oracle.dfs_bridges(u, v, V)
        for M in (1, 4, 33):
            assert gpu_bridges(ctx, u, v, V, M).tolist() == ref.tolist(), (t, V, E, M)


@pytest.mark.parametrize("M", [1, 2, 16, 64, 1000])
def test_small_workload(ctx, M):
    g = graphgen.workload("small")
    got = gpu_bridges(ctx, g.u, g.v, g.V, M)
    assert got.tolist() == oracle.bridges(g.u, g.v, g.V, 16).tolist()
    assert got.tolist() == g.planted.tolist()


@pytest.mark.parametrize("M", [16, 64, 256, 1024])
def test_mid_workload_M_sweep(ctx, M):
    g = graphgen.workload("mid")
    got = gpu_bridges(ctx, g.u, g.v, g.V, M)
    ref = oracle.bridges(g.u, g.v, g.V, 16)
    assert got.tolist() == ref.tolist()
    assert got.tolist() == g.planted.tolist()


def test_trees_paths_stars(ctx):
    """Closed forms at sizes that exercise the radix-sort path (more than 16k bridges)."""
    rng = np.random.default_rng(23)
    for n in (2, 1000, 20000, 70000):
        par = (rng.random(n - 1) * np.arange(1, n)).astype(np.int32)
        ch = np.arange(1, n, dtype=np.int32)
        perm = rng.permutation(n - 1)
        got = gpu_bridges(ctx, par[perm], ch[perm], n, 1)
        exp = np.sort(np.stack([np.minimum(par, ch), np.maximum(par, ch)], 1).view(np.int64).ravel())
        assert len(got) == n - 1
        assert got.tolist() == oracle.dfs_bridges(par, ch, n).tolist()
    n = 50000
    u = np.arange(n - 1, dtype=np.int32)
    assert len(gpu_bridges(ctx, u, u + 1, n, 3)) == n - 1  # path
    assert len(gpu_bridges(ctx, np.concatenate([u, u + 1]), np.concatenate([u + 1, u]), n, 3)) == 0  # doubled
    w = (u + 1) % (n - 1)
    assert len(gpu_bridges(ctx, u, w, n, 2)) == 0  # cycle on n-1 vertices, vertex n-1 isolated
    star = np.zeros(n - 1, np.int32)
    assert len(gpu_bridges(ctx, star, u + 1, n, 4)) == n - 1


def test_edge_cases(ctx, cuda_lib):
    e = np.zeros(0, np.int32)
    assert len(gpu_bridges(ctx, e, e, 0)) == 0
    assert len(gpu_bridges(ctx, e, e, 10)) == 0
    assert len(gpu_bridges(ctx, np.zeros(5, np.int32), np.zeros(5, np.int32), 1)) == 0  # self-loops
    assert gpu_bridges(ctx, np.array([3], np.int32), np.array([1], np.int32), 4).tolist() == [[1, 3]]
    # out-of-range ids -> ERANGE, and the context stays usable
    with pytest.raises(cuda_lib.BridgesError) as ei:
        gpu_bridges(ctx, np.array([0, 1], np.int32), np.array([1, 9], np.int32), 5)
    assert ei.value.code == -2
    with pytest.raises(cuda_lib.BridgesError):
        gpu_bridges(ctx, np.array([-1], np.int32), np.array([1], np.int32), 5)
    with pytest.raises(cuda_lib.BridgesError) as ei:
        du, dv = dev_edges(np.array([0], np.int32), np.array([1], np.int32))
        ctx.find(du, dv, -3)
    assert ei.value.code == -1
    assert gpu_bridges(ctx, np.array([0], np.int32), np.array([1], np.int32), 2).tolist() == [[0, 1]]


def test_misaligned_and_offset_inputs(ctx):
    """Pointers that are not 16-byte aligned (and misaligned relative to each other) take the
    scalar load path; results are unchanged."""
    g = graphgen.workload("small")
    ref = oracle.bridges(g.u, g.v, g.V, 16)
    du, dv = dev_edges(np.concatenate([[0], g.u]), np.concatenate([[0, 0, 0], g.v]))
    u1, v1 = du[1:], dv[3:]
    assert u1.data_ptr() % 16 != 0
    assert ctx.find(u1, v1, g.V, 4).cpu().numpy().tolist() == ref.tolist()


def test_repeatable(ctx):
    g = graphgen.workload("mid")
    du, dv = dev_edges(g.u, g.v)
    first = ctx.find(du, dv, g.V, 32).cpu().numpy()
    for _ in range(3):
        assert np.array_equal(ctx.find(du, dv, g.V, 32).cpu().numpy(), first)


def _cert_check(u, v, V, cu, cv, ct):
    c, lab = oracle.components(u, v, V)
    assert len(cu) <= 2 * (V - c)
    # sub-multiset of the input (edges as unordered pairs)
    key = lambda a, b: np.minimum(a, b).astype(np.int64) * V + np.maximum(a, b)
    ku, kc = np.unique(key(u, v), return_counts=True)
    cku, ckc = np.unique(key(cu, cv), return_counts=True)
    pos = np.searchsorted(ku, cku)
    assert (pos < len(ku)).all() and (ku[np.minimum(pos, len(ku) - 1)] == cku).all()
    assert (ckc <= kc[pos]).all()
    c2, lab2 = oracle.components(cu, cv, V)
    assert c2 == c and np.array_equal(lab, lab2)
    # the tree part is a spanning forest: V - c edges with the same components
    assert int(ct.sum()) == V - c
    c3, lab3 = oracle.components(cu[ct], cv[ct], V)
    assert c3 == c and np.array_equal(lab3, lab)
    assert oracle.dfs_bridges(cu, cv, V).tolist() == oracle.dfs_bridges(u, v, V).tolist()


@pytest.mark.parametrize("name,M", [("small", 1), ("small", 16), ("mid", 8), ("mid", 300)])
def test_certificate_invariants(ctx, name, M):
    g = graphgen.workload(name)
    du, dv = dev_edges(g.u, g.v)
    cu, cv, ct = ctx.certificate(du, dv, g.V, M)
    _cert_check(g.u, g.v, g.V, cu.cpu().numpy(), cv.cpu().numpy(), ct.cpu().numpy())


def test_certificate_invariants_random(ctx):
    for t in range(60):
        V = 10 + 7 * t
        u, v = graphgen.random_multigraph(40000 + t, V, 6 * V)
        du, dv = dev_edges(u, v)
        cu, cv, ct = ctx.certificate(du, dv, V, 1 + t % 9)
        _cert_check(u, v, V, cu.cpu().numpy(), cv.cpu().numpy(), ct.cpu().numpy())


def test_from_forest_matches_oracle(ctx):
    """The final stage alone, fed the oracle's own certificate (Alg. 2 forests)."""
    for name in ("small", "mid"):
        g = graphgen.workload(name)
        ids, f1 = oracle.certificate(g.u, g.v, g.V)
        tu, tv = dev_edges(g.u[ids[f1]], g.v[ids[f1]])
        xu, xv = dev_edges(g.u[ids[~f1]], g.v[ids[~f1]])
        got = ctx.from_forest(tu, tv, xu, xv, g.V).cpu().numpy()
        assert got.tolist() == oracle.dfs_bridges(g.u, g.v, g.V).tolist()


@pytest.mark.parametrize("V", [2060, 3090, 33_812, 70_000, 1_230_860])
def test_from_forest_path_ranges(ctx, V):
    """The final stage on the path 0-1-...-(V-1) given as the forest: its preorder is the vertex
    order whatever order the arcs come in, so vertex y's subtree is the range [y, V) and every
    start of a range ending at V is queried.  V is chosen one chunk past a superchunk (32 chunks
    of 32 preorder numbers; 64 chunks above about a million vertices), so for y in the chunk
    before that superchunk the range's whole chunks fill it exactly.  Random extra edges close
    cycles over the path; the bridges are the path edges no cycle covers."""
    rng = np.random.default_rng(V)
    tu = np.arange(V - 1, dtype=np.int32)
    tv = tu + 1
    a, b = rng.integers(0, V, 40), rng.integers(0, V, 40)
    xu, xv = a[a != b].astype(np.int32), b[a != b].astype(np.int32)
    got = ctx.from_forest(*dev_edges(tu, tv), *dev_edges(xu, xv), V).cpu().numpy()
    assert got.tolist() == oracle.dfs_bridges(np.concatenate([tu, xu]), np.concatenate([tv, xv]), V).tolist()


def test_find_host_and_async(ctx, cuda_lib):
    g = graphgen.workload("small")
    ref = oracle.bridges(g.u, g.v, g.V, 16)
    hu = torch.from_numpy(np.array(g.u)).pin_memory()
    hv = torch.from_numpy(np.array(g.v)).pin_memory()
    assert ctx.find_host(hu, hv, g.V, 8).numpy().tolist() == ref.tolist()
    du, dv = dev_edges(g.u, g.v)
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    out = ctx.find(du, dv, g.V, 8, count_device=cnt)
    torch.cuda.synchronize()
    n = int(cnt.item())
    assert out[: 2 * n].view(n, 2).cpu().numpy().tolist() == ref.tolist()


def test_user_workspace_and_plain_call(cuda_lib):
    g = graphgen.workload("small")
    ref = oracle.bridges(g.u, g.v, g.V, 16)
    probe = cuda_lib.Context(device="cuda:0")
    need = probe.workspace_bytes(g.E, g.V, 4)
    c2 = cuda_lib.Context(device="cuda:0", workspace_bytes=need)
    du, dv = dev_edges(g.u, g.v)
    assert c2.find(du, dv, g.V, 4).cpu().numpy().tolist() == ref.tolist()
    with pytest.raises(cuda_lib.BridgesError) as ei:
        c2.find(du, dv, g.V, 64)  # needs a bigger workspace than was given
    assert ei.value.code == -3
    assert cuda_lib.bridges_find(du, dv, g.V, 16).cpu().numpy().tolist() == ref.tolist()


def test_stage_timings_and_launch_count(cuda_lib):
    g = graphgen.workload("mid")
    c = cuda_lib.Context(device="cuda:0", profile=True)
    du, dv = dev_edges(g.u, g.v)
    before = c.launches()
    c.find(du, dv, g.V, 4)
    ms = c.stage_ms()
    assert set(ms) == {"warmup", "snapshot", "forest", "merge", "final", "total"}
    assert ms["total"] > 0 and c.launches() > before
    cfg = c.last_config()
    assert cfg["M"] == 4


def test_host_read_in_place(cuda_lib):
    """opts.host_read: kernels stream pinned host memory directly (no device copy of the edges),
    the out-of-core form; results unchanged."""
    g = graphgen.workload("mid")
    ref = oracle.bridges(g.u, g.v, g.V, 16)
    hu = torch.from_numpy(np.array(g.u)).pin_memory()
    hv = torch.from_numpy(np.array(g.v)).pin_memory()
    c = cuda_lib.Context(device="cuda:0", host_read=True)
    assert c.find_host(hu, hv, g.V, 4).numpy().tolist() == ref.tolist()
    # pageable host memory falls back to copying
    assert c.find_host(torch.from_numpy(np.array(g.u)), torch.from_numpy(np.array(g.v)), g.V, 4).numpy().tolist() \
        == ref.tolist()


@pytest.mark.parametrize("warm_block", [32, 64, 256, 1024])
@pytest.mark.parametrize("warm_edges", [0, 1000, 200000])
def test_plan_options(cuda_lib, warm_block, warm_edges):
    """Every plan the options can select gives the same exact set: warm-up launch block sizes,
    no snapshot at all (0), a short warm-up (many misses take the union-find path) and a long one."""
    g = graphgen.workload("mid")
    ref = oracle.bridges(g.u, g.v, g.V, 16)
    c = cuda_lib.Context(device="cuda:0", warm_edges=warm_edges, warm_block=warm_block)
    du, dv = dev_edges(g.u, g.v)
    for M in (1, 6):
        assert c.find(du, dv, g.V, M).cpu().numpy().tolist() == ref.tolist(), (warm_block, warm_edges, M)
    assert c.get_opts()["warm_block"] == warm_block


@pytest.mark.parametrize("scale,factor", [(10, 4), (12, 16), (14, 8), (16, 16), (17, 4), (19, 16), (20, 8),
                                          (21, 4)])
def test_rmat_skewed_degrees(ctx, scale, factor):
    """Power-law (R-MAT) graphs: hubs with thousands of edges, many leaves and isolated vertices,
    self-loops and repeats -- a contention pattern the uniform workloads do not have.  From 2^17
    vertices on, 16-bit labels no longer fit in shared memory and the forest pass takes the
    bitmap snapshot of the largest F' component; 2^21 vertices exceed the bitmap's reach (the
    vertices past it always take the union-find path)."""
    V = 1 << scale
    u, v = graphgen.rmat(100 + scale, scale, factor * V)
    ref = oracle.dfs_bridges(u, v, V)
    for M in (1, 5):
        assert gpu_bridges(ctx, u, v, V, M).tolist() == ref.tolist(), M
    if scale >= 17:  # the bitmap path, with and without a warm-up long enough to take it
        for warm in (4096, 1 << 20, 0):
            c = cuda_lib_ctx(warm_edges=warm)
            assert gpu_bridges(c, u, v, V, 1).tolist() == ref.tolist(), warm


def cuda_lib_ctx(**kw):
    import paper_2108_07346_gb300 as pb

    return pb.Context(device="cuda:0", **kw)


def test_find_host_pipelined_chunks(cuda_lib):
    """bridges_find_host on a list long enough to be copied in chunks overlapped with the forest
    pass (the large workload's vertex set at density 0.04: about 86 M edges, 6 chunks): the same
    exact set as the device path and the planted bridges, pinned and pageable input alike."""
    g = graphgen.workload("large", p=0.04)
    assert g.E > 64 << 20
    c = cuda_lib.Context(device="cuda:0", profile=True)
    hu = torch.from_numpy(np.array(g.u)).pin_memory()
    hv = torch.from_numpy(np.array(g.v)).pin_memory()
    got = c.find_host(hu, hv, g.V, 1).numpy()
    assert got.tolist() == g.planted.tolist()
    du, dv = dev_edges(g.u, g.v)
    assert c.find(du, dv, g.V, 1).cpu().numpy().tolist() == got.tolist()
    assert c.find_host(hu, hv, g.V, 1).numpy().tolist() == got.tolist()  # reuses the chunk events
    assert c.find_host(torch.from_numpy(np.array(g.u)), torch.from_numpy(np.array(g.v)), g.V, 1).numpy().tolist() \
        == got.tolist()


def test_large_v_closed_forms(ctx):
    """Closed forms beyond the 16-bit label capacity (the bitmap snapshot): a star and a path of
    300,000 vertices (every edge a bridge), a perfect matching (largest F' component of two
    vertices), the same matching with every edge doubled (no bridges), and no edges at all."""
    n = 300_000
    a = np.arange(n - 1, dtype=np.int32)
    perm = np.random.default_rng(71).permutation(n - 1)
    star = gpu_bridges(ctx, np.zeros(n - 1, np.int32)[perm], (a + 1)[perm], n, 1)
    assert len(star) == n - 1 and star[:, 0].max() == 0
    assert len(gpu_bridges(ctx, a[perm], (a + 1)[perm], n, 1)) == n - 1
    m = np.arange(0, n, 2, dtype=np.int32)
    assert gpu_bridges(ctx, m, m + 1, n, 1).tolist() == np.stack([m, m + 1], 1).tolist()
    assert len(gpu_bridges(ctx, np.concatenate([m, m + 1]), np.concatenate([m + 1, m]), n, 1)) == 0
    e = np.zeros(0, np.int32)
    assert len(gpu_bridges(ctx, e, e, n, 1)) == 0


def test_seeded_fuzz_against_oracle(cuda_lib):
    """A seeded mix of graph families and plans: uniform multigraphs, R-MAT, trees with a few
    cycles, duplicated lists, planted clusters; M, warm-up length and warm-up block size drawn at
    random.  Bridges and cut vertices against the oracle every time."""
    rng = np.random.default_rng(77)
    for t in range(120):
        fam = t % 5
        if fam == 0:
            V = int(rng.integers(2, 3000))
            u, v = graphgen.random_multigraph(60000 + t, V, int(rng.integers(V // 2, 8 * V)))
        elif fam == 1:
            scale = int(rng.integers(6, 15))
            V = 1 << scale
            u, v = graphgen.rmat(61000 + t, scale, int(rng.integers(2, 24)) << scale)
        elif fam == 2:
            V = int(rng.integers(2, 20000))
            par = (rng.random(V - 1) * np.arange(1, V)).astype(np.int32)
            ch = np.arange(1, V, dtype=np.int32)
            k = int(rng.integers(0, 20))
            u = np.concatenate([par, rng.integers(0, V, k).astype(np.int32)])
            v = np.concatenate([ch, rng.integers(0, V, k).astype(np.int32)])
        elif fam == 3:
            V = int(rng.integers(2, 2000))
            u0, v0 = graphgen.random_multigraph(62000 + t, V, int(rng.integers(0, 3 * V)))
            u, v = np.concatenate([u0, v0, u0]), np.concatenate([v0, u0, v0])
        else:
            g = graphgen.generate(graphgen.workload_spec("batched", 9, t))
            u, v, V = g.u, g.v, g.V
        perm = rng.permutation(len(u))
        u, v = np.ascontiguousarray(u[perm]), np.ascontiguousarray(v[perm])
        M = int(rng.choice([1, 1, 2, 3, 8]))
        c = cuda_lib.Context(device="cuda:0", warm_edges=int(rng.choice([-1, 0, 500, 20000])),
                             warm_block=int(rng.choice([0, 64, 256, 1024])))
        du, dv = dev_edges(u, v)
        assert c.find(du, dv, V, M).cpu().numpy().tolist() == oracle.dfs_bridges(u, v, V).tolist(), (t, fam, V, M)
        if t % 3 == 0:
            assert c.articulation_points(du, dv, V, M).cpu().numpy().tolist() == \
                oracle.articulation_points(u, v, V).tolist(), (t, fam, V, M)
