"""Parity of the articulation-point path (through the C ABI) with the CPU oracle.

The set of cut vertices is unique, so the sorted list must match the oracle's bit for bit:
Tarjan's low/disc test (oracle.articulation_points) and, on small graphs, the definition itself
(oracle.brute_articulation).  Sizes span several 4,096-edge tiles with ragged tails, and M
varies the bridge path's partitioning underneath.
"""
import numpy as np
import pytest
import torch

import graphgen
import oracle
from conftest import golden_names, load_golden, load_golden_cuts

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.array(a, dtype=np.int32)).to("cuda:0")


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    return cuda_lib.Context(device="cuda:0")


def gpu_points(ctx, u, v, V, M=0):
    return ctx.articulation_points(dev(u), dev(v), V, M).cpu().numpy()


@pytest.mark.parametrize("name", golden_names())
@pytest.mark.parametrize("M", [1, 3])
def test_golden(ctx, name, M):
    u, v, V, _ = load_golden(name)
    got = gpu_points(ctx, u, v, V, M).tolist()
    assert got == oracle.brute_articulation(u, v, V).tolist()
    assert got == load_golden_cuts(name).tolist()  # the fixture's hand-derived cut vertices


def test_random_multigraphs_against_definition(ctx):
    rng = np.random.default_rng(61)
    for t in range(400):
        V = int(rng.integers(1, 65))
        E = int(rng.integers(0, 4 * V + 2))
        u, v = graphgen.random_multigraph(50000 + t, V, E)
        M = int(rng.choice([1, 2, 5, 64]))
        assert gpu_points(ctx, u, v, V, M).tolist() == oracle.brute_articulation(u, v, V).tolist(), (t, V, E, M)


def test_random_sparse_mid(ctx):
    """Sparse graphs: many small blocks, long tree paths, many components."""
    rng = np.random.default_rng(62)
    for t in range(30):
        V = int(rng.integers(100, 20000))
        E = int(rng.integers(V // 2, 3 * V))
        u, v = graphgen.random_multigraph(51000 + t, V, E)
        ref = oracle.articulation_points(u, v, V)
        for M in (1, 7):
            assert gpu_points(ctx, u, v, V, M).tolist() == ref.tolist(), (t, V, E, M)


def test_dense_with_snapshot(ctx):
    """Dense enough that the block pass takes its label snapshot (E > warm-up)."""
    for t, (V, E) in enumerate([(300, 200000), (2000, 600000), (5000, 3000001)]):
        u, v = graphgen.random_multigraph(52000 + t, V, E)
        ref = oracle.articulation_points(u, v, V)
        for M in (1, 4):
            assert gpu_points(ctx, u, v, V, M).tolist() == ref.tolist(), (t, M)


@pytest.mark.parametrize("name,Ms", [("small", (1, 16)), ("mid", (1, 8, 64))])
def test_workloads(ctx, name, Ms):
    g = graphgen.workload(name)
    ref = oracle.articulation_points(g.u, g.v, g.V)
    assert len(ref) > 0
    for M in Ms:
        assert gpu_points(ctx, g.u, g.v, g.V, M).tolist() == ref.tolist(), M


def test_closed_forms(ctx):
    rng = np.random.default_rng(63)
    for n in (2, 3, 1000, 70000):  # random trees: the vertices of degree >= 2
        par = (rng.random(n - 1) * np.arange(1, n)).astype(np.int32)
        ch = np.arange(1, n, dtype=np.int32)
        perm = rng.permutation(n - 1)
        deg = np.bincount(np.concatenate([par, ch]), minlength=n)
        assert gpu_points(ctx, par[perm], ch[perm], n, 1).tolist() == np.flatnonzero(deg >= 2).tolist()
    n = 50000
    a = np.arange(n - 1, dtype=np.int32)
    assert gpu_points(ctx, a, a + 1, n, 3).tolist() == list(range(1, n - 1))  # path
    c = np.arange(n, dtype=np.int32)
    assert len(gpu_points(ctx, c, (c + 1) % n, n, 2)) == 0  # cycle
    assert gpu_points(ctx, np.zeros(n - 1, np.int32), a + 1, n, 4).tolist() == [0]  # star
    # a chain of 1,000 triangles sharing one vertex each: the 999 shared vertices
    k = 1000
    base = 2 * np.arange(k, dtype=np.int32)
    u = np.concatenate([base, base + 1, base + 2])
    v = np.concatenate([base + 1, base + 2, base])
    assert gpu_points(ctx, u, v, 2 * k + 1, 2).tolist() == (2 * np.arange(1, k)).tolist()


def test_edge_cases(ctx, cuda_lib):
    e = np.zeros(0, np.int32)
    assert len(gpu_points(ctx, e, e, 0)) == 0
    assert len(gpu_points(ctx, e, e, 1)) == 0
    assert len(gpu_points(ctx, e, e, 10)) == 0
    assert len(gpu_points(ctx, np.zeros(5, np.int32), np.zeros(5, np.int32), 1)) == 0  # self-loops
    assert len(gpu_points(ctx, np.array([3], np.int32), np.array([1], np.int32), 4)) == 0  # one edge
    # doubled path: every edge has a parallel copy, yet the inner vertices still cut
    a = np.arange(9, dtype=np.int32)
    assert gpu_points(ctx, np.concatenate([a, a]), np.concatenate([a + 1, a + 1]), 10).tolist() == list(range(1, 9))
    with pytest.raises(cuda_lib.BridgesError) as ei:
        gpu_points(ctx, np.array([0, 1], np.int32), np.array([1, 9], np.int32), 5)
    assert ei.value.code == -2
    assert gpu_points(ctx, np.array([0, 1], np.int32), np.array([1, 2], np.int32), 3).tolist() == [1]


def test_misaligned_input(ctx):
    g = graphgen.workload("small")
    ref = oracle.articulation_points(g.u, g.v, g.V)
    du, dv = dev(np.concatenate([[0], g.u])), dev(np.concatenate([[0, 0, 0], g.v]))
    assert ctx.articulation_points(du[1:], dv[3:], g.V, 2).cpu().numpy().tolist() == ref.tolist()


def test_with_bridges_async_and_profile(cuda_lib):
    g = graphgen.workload("mid")
    ref_ap = oracle.articulation_points(g.u, g.v, g.V)
    ref_br = oracle.dfs_bridges(g.u, g.v, g.V)
    c = cuda_lib.Context(device="cuda:0", profile=True)
    du, dv = dev(g.u), dev(g.v)
    pts, br = c.articulation_points(du, dv, g.V, 4, with_bridges=True)
    assert pts.cpu().numpy().tolist() == ref_ap.tolist()
    assert br.cpu().numpy().tolist() == ref_br.tolist()
    ms = c.ap_stage_ms()
    assert set(ms) == {"warmup", "snapshot", "stream", "mark", "total"} and ms["total"] > 0
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda:0")
    out = c.articulation_points(du, dv, g.V, 4, counts_device=cnt)
    torch.cuda.synchronize()
    na, nb = (int(x) for x in cnt.cpu())
    assert na == len(ref_ap) and nb == len(ref_br)
    assert out[:na].cpu().numpy().tolist() == ref_ap.tolist()


@pytest.mark.parametrize("M,fused", [(2, 0), (1, 1)])
def test_user_workspace(cuda_lib, M, fused):
    """A caller's workspace of exactly bridges_articulation_workspace_bytes suffices for the form
    the call takes (the fused one for a single partition).  With less, a single-partition call
    falls back to the two-pass form while that fits; below the two-pass need it is ENOMEM."""
    g = graphgen.workload("small")
    ref = oracle.articulation_points(g.u, g.v, g.V).tolist()
    need = cuda_lib.Context(device="cuda:0").articulation_workspace_bytes(g.E, g.V, M)
    c = cuda_lib.Context(device="cuda:0", workspace_bytes=need)
    assert c.articulation_points(dev(g.u), dev(g.v), g.V, M).cpu().numpy().tolist() == ref
    assert c.last_config()["ap_fused"] == fused
    two_pass = cuda_lib.Context(device="cuda:0", ap_fused=-1).articulation_workspace_bytes(g.E, g.V, M)
    if fused:
        assert two_pass < need
        c = cuda_lib.Context(device="cuda:0", workspace_bytes=need - 1)
        assert c.articulation_points(dev(g.u), dev(g.v), g.V, M).cpu().numpy().tolist() == ref
        assert c.last_config()["ap_fused"] == 0
    small = cuda_lib.Context(device="cuda:0", workspace_bytes=two_pass - 1)
    with pytest.raises(cuda_lib.BridgesError) as ei:
        small.articulation_points(dev(g.u), dev(g.v), g.V, M)
    assert ei.value.code == -3


def test_budget_falls_back_to_two_passes(cuda_lib):
    """A memory budget that holds the two-pass workspace but not the fused one: the call runs
    two passes (same result) instead of failing."""
    g = graphgen.workload("small")
    ref = oracle.articulation_points(g.u, g.v, g.V).tolist()
    two_pass = cuda_lib.Context(device="cuda:0", ap_fused=-1).articulation_workspace_bytes(g.E, g.V, 1)
    fused = cuda_lib.Context(device="cuda:0").articulation_workspace_bytes(g.E, g.V, 1)
    assert two_pass < fused
    c = cuda_lib.Context(device="cuda:0", mem_budget=(two_pass + fused) // 2)
    assert c.articulation_points(dev(g.u), dev(g.v), g.V, 1).cpu().numpy().tolist() == ref
    assert c.last_config()["ap_fused"] == 0


def test_host_entry(cuda_lib):
    """bridges_articulation_points_host: pinned and pageable host input, copied or read in place."""
    g = graphgen.workload("mid")
    ref = oracle.articulation_points(g.u, g.v, g.V).tolist()
    hu = torch.from_numpy(np.array(g.u)).pin_memory()
    hv = torch.from_numpy(np.array(g.v)).pin_memory()
    for host_read in (False, True):
        c = cuda_lib.Context(device="cuda:0", host_read=host_read)
        assert c.articulation_points_host(hu, hv, g.V, 4).numpy().tolist() == ref
        assert c.articulation_points_host(torch.from_numpy(np.array(g.u)), torch.from_numpy(np.array(g.v)), g.V,
                                          2).numpy().tolist() == ref


@pytest.mark.parametrize("ap_warm_edges", [-1, 0, 5000, 10_000_000])
def test_block_pass_prefix_options(cuda_lib, ap_warm_edges):
    """The block pass's prefix before its snapshot: none (-1), automatic, short, and longer than
    the list (no snapshot): the cut vertices do not change."""
    g = graphgen.workload("mid")
    ref = oracle.articulation_points(g.u, g.v, g.V).tolist()
    c = cuda_lib.Context(device="cuda:0", ap_warm_edges=ap_warm_edges, ap_fused=-1)
    assert c.articulation_points(dev(g.u), dev(g.v), g.V, 3).cpu().numpy().tolist() == ref
    cfg = c.last_config()
    assert cfg["ap_warm_edges"] == (-1 if ap_warm_edges >= g.E else (0 if ap_warm_edges < 0 else cfg["ap_warm_edges"]))


@pytest.mark.parametrize("scale,factor", [(10, 4), (13, 16), (16, 8), (18, 8)])
def test_rmat_skewed_degrees(ctx, scale, factor):
    V = 1 << scale
    u, v = graphgen.rmat(200 + scale, scale, factor * V)
    assert gpu_points(ctx, u, v, V, 2).tolist() == oracle.articulation_points(u, v, V).tolist()


def test_host_entry_pipelined(cuda_lib):
    """bridges_articulation_points_host on a list long enough for the chunked copy overlapped with
    the forest pass (the large workload's vertex set at density 0.04, about 86 M edges): the
    cut vertices are the construction's, as on the device path."""
    import bench

    g = graphgen.workload("large", p=0.04)
    expect = bench.planted_cut_vertices(g).tolist()
    hu = torch.from_numpy(np.array(g.u)).pin_memory()
    hv = torch.from_numpy(np.array(g.v)).pin_memory()
    c = cuda_lib.Context(device="cuda:0")
    assert c.articulation_points_host(hu, hv, g.V).numpy().tolist() == expect
    assert c.articulation_points_host(hu, hv, g.V).numpy().tolist() == expect
    assert c.articulation_points(dev(g.u), dev(g.v), g.V).cpu().numpy().tolist() == expect


def chain_of_blocks(seed, k, size, deg):
    """k random blocks of `size` vertices and about deg * size edges each, block i sharing its
    last vertex with block i + 1 (a chain through k - 1 shared vertices), ids shuffled."""
    rng = np.random.default_rng(seed)
    us, vs = [], []
    for i in range(k):
        lo = i * (size - 1)
        m = deg * size
        us.append(lo + rng.integers(0, size, m))
        vs.append(lo + rng.integers(0, size, m))
    V = k * (size - 1) + 1
    perm = rng.permutation(V).astype(np.int32)
    u, v = perm[np.concatenate(us)], perm[np.concatenate(vs)]
    order = rng.permutation(len(u))
    return u[order].astype(np.int32), v[order].astype(np.int32), V


@pytest.mark.parametrize("ap_warm_edges", [-1, 0, 5000])
def test_large_v_bitmap_snapshot(cuda_lib, ap_warm_edges):
    """More vertices than 16-bit labels fit in shared memory: the block pass snapshots the
    largest class as a bitmap (vertices past its reach always walk).  R-MAT graphs (one large
    block and a periphery), a chain of dense blocks, and a graph beyond the bitmap's reach."""
    c = cuda_lib.Context(device="cuda:0", ap_warm_edges=ap_warm_edges)
    cases = [graphgen.rmat(317, 17, 8 << 17) + (1 << 17,), graphgen.rmat(319, 19, 4 << 19) + (1 << 19,),
             chain_of_blocks(321, 150, 1000, 12)]
    for u, v, V in cases:
        ref = oracle.articulation_points(u, v, V).tolist()
        assert c.articulation_points(dev(u), dev(v), V, 1).cpu().numpy().tolist() == ref, V
        cfg = c.last_config()
        assert cfg["ap_warm_edges"] == (0 if ap_warm_edges < 0 else cfg["ap_warm_edges"]) and cfg["ap_warm_edges"] >= 0


@pytest.mark.slow
def test_beyond_bitmap_reach(ctx):
    """2^21 vertices: ids past the bitmap's reach (about 1.85 M) take the cycle walk."""
    u, v = graphgen.rmat(323, 21, 4 << 21)
    V = 1 << 21
    assert gpu_points(ctx, u, v, V, 1).tolist() == oracle.articulation_points(u, v, V).tolist()


def two_clusters(seed, n, m, cross, tail=True, pendants=0):
    """Two dense random clusters of n vertices (m edges each) joined by `cross` disjoint edges,
    listed after every cluster edge when `tail` (so they arrive after the forest pass's warm-up,
    between two trees of its forest), plus `pendants` vertices hung on the first cluster."""
    rng = np.random.default_rng(seed)
    a = rng.integers(0, n, (2, m))
    b = rng.integers(n, 2 * n, (2, m))
    body_u, body_v = np.concatenate([a[0], b[0]]), np.concatenate([a[1], b[1]])
    cu, cv = rng.permutation(n)[:cross], n + rng.permutation(n)[:cross]
    pu = 2 * n + np.arange(pendants)
    pv = rng.integers(0, n, pendants)
    if tail:  # body shuffled, then the pendants, then the cross edges
        order = rng.permutation(len(body_u))
        u, v = np.concatenate([body_u[order], pu, cu]), np.concatenate([body_v[order], pv, cv])
    else:  # everything shuffled together
        u, v = np.concatenate([body_u, pu, cu]), np.concatenate([body_v, pv, cv])
        order = rng.permutation(len(u))
        u, v = u[order], v[order]
    return u.astype(np.int32), v.astype(np.int32), 2 * n + pendants


def test_fused_against_two_pass(cuda_lib):
    """One read of the list (the default for one partition with labels) and the two-pass form
    agree with the oracle on dense graphs, on graphs whose late edges join two trees of the
    warm-up's forest (walked once the final tree is known), and with the bridges alongside."""
    fused = cuda_lib.Context(device="cuda:0")
    two = cuda_lib.Context(device="cuda:0", ap_fused=-1)
    cases = [graphgen.random_multigraph(53000 + t, V, E) + (V,) for t, (V, E) in
             enumerate([(300, 200000), (2000, 600000), (5000, 3000001)])]
    cases += [two_clusters(54000, 1500, 400000, 3, pendants=5), two_clusters(54001, 800, 200000, 400),
              two_clusters(54002, 1200, 300000, 1, pendants=3), two_clusters(54003, 1000, 250000, 50, tail=False)]
    g = graphgen.workload("mid")
    cases.append((g.u, g.v, g.V))
    for u, v, V in cases:
        ref = oracle.articulation_points(u, v, V).tolist()
        refb = oracle.bridges(u, v, V).tolist()
        pts, br = fused.articulation_points(dev(u), dev(v), V, 0, with_bridges=True)
        assert fused.last_config()["ap_fused"] == 1, V
        assert pts.cpu().numpy().tolist() == ref and br.cpu().numpy().tolist() == refb, V
        assert two.articulation_points(dev(u), dev(v), V, 0).cpu().numpy().tolist() == ref, V
        assert two.last_config()["ap_fused"] == 0


def test_fused_enqueue_only(cuda_lib):
    """The fused form enqueued with device counts: points and bridges as from the synchronous
    call, on a graph with edges marked for the final tree."""
    c = cuda_lib.Context(device="cuda:0")
    u, v, V = two_clusters(55000, 1500, 400000, 200, pendants=7)
    ref, refb = oracle.articulation_points(u, v, V).tolist(), oracle.bridges(u, v, V).tolist()
    cnt = torch.zeros(2, dtype=torch.int64, device="cuda:0")
    out = torch.full((V,), -7, dtype=torch.int32, device="cuda:0")
    for _ in range(3):  # the marks of one call must not leak into the next
        pts, br = c.articulation_points(dev(u), dev(v), V, 0, with_bridges=True, counts_device=cnt, out=out)
        torch.cuda.synchronize()
        n, nb = (int(x) for x in cnt.cpu())
        assert c.last_config()["ap_fused"] == 1
        assert out[:n].cpu().numpy().tolist() == ref
        assert br[: 2 * nb].view(nb, 2).cpu().numpy().tolist() == refb


def blocks_tree(rng, nblocks, size, deg):
    """Random blocks (dense random graphs of `size` vertices and deg * size edges) hung on a random
    tree of cut vertices: block k shares one vertex with an earlier block; plus pendant paths."""
    us, vs = [], []
    base = [0]
    for k in range(nblocks):
        lo = base[-1]
        verts = np.arange(lo, lo + size)
        if k:  # share one vertex with a random earlier block
            j = int(rng.integers(0, k))
            verts[0] = int(rng.integers(base[j], base[j] + size))
        m = deg * size
        us.append(verts[rng.integers(0, size, m)])
        vs.append(verts[rng.integers(0, size, m)])
        base.append(lo + size)
    V = base[-1]
    npend = int(rng.integers(0, 50))
    for p in range(npend):  # a pendant path of 1-5 edges
        L = int(rng.integers(1, 6))
        path = np.concatenate([[int(rng.integers(0, V))], np.arange(V, V + L)])
        us.append(path[:-1])
        vs.append(path[1:])
        V += L
    u, v = np.concatenate(us), np.concatenate(vs)
    perm = rng.permutation(V)
    order = rng.permutation(len(u))
    return perm[u][order].astype(np.int32), perm[v][order].astype(np.int32), V


def test_fused_fuzz(cuda_lib):
    """Seeded fuzz of the fused form on graph families dense enough to take it: trees of dense
    blocks with pendant paths, and two clusters whose joining edges come late in the list."""
    c = cuda_lib.Context(device="cuda:0")
    rng = np.random.default_rng(56)
    for t in range(24):
        if t % 3 == 2:
            n = int(rng.integers(300, 1500))
            u, v, V = two_clusters(56000 + t, n, int(rng.integers(60, 200)) * n, int(rng.integers(1, 60)),
                                   tail=bool(rng.integers(0, 2)), pendants=int(rng.integers(0, 20)))
        else:
            u, v, V = blocks_tree(rng, int(rng.integers(2, 40)), int(rng.integers(20, 400)), int(rng.integers(30, 120)))
        ref = oracle.articulation_points(u, v, V).tolist()
        refb = oracle.bridges(u, v, V).tolist()
        pts, br = c.articulation_points(dev(u), dev(v), V, 0, with_bridges=True)
        assert c.last_config()["ap_fused"] == 1, (t, V, len(u))
        assert pts.cpu().numpy().tolist() == ref, (t, V, len(u))
        assert br.cpu().numpy().tolist() == refb, (t, V, len(u))


@pytest.mark.parametrize("where", ["prefix", "stream"])
def test_fused_range_error(cuda_lib, where):
    """An id outside [0, V) in the warm-up prefix or later in the list: ERANGE from the fused
    form, and the context still answers the next call."""
    c = cuda_lib.Context(device="cuda:0")
    u, v, V = two_clusters(57000, 1000, 250000, 20, pendants=4)
    bad = v.copy()
    bad[100 if where == "prefix" else len(bad) - 10] = V + 5
    with pytest.raises(cuda_lib.BridgesError) as ei:
        c.articulation_points(dev(u), dev(bad), V, 0)
    assert ei.value.code == -2
    assert c.articulation_points(dev(u), dev(v), V, 0).cpu().numpy().tolist() == \
        oracle.articulation_points(u, v, V).tolist()
    assert c.last_config()["ap_fused"] == 1


def test_fused_self_loops_only(cuda_lib):
    """A list long enough for the fused form that holds only self-loops: no cut vertices."""
    c = cuda_lib.Context(device="cuda:0")
    V = 3000
    a = np.random.default_rng(58).integers(0, V, 200000).astype(np.int32)
    assert len(c.articulation_points(dev(a), dev(a), V, 0)) == 0
    assert c.last_config()["ap_fused"] == 1
