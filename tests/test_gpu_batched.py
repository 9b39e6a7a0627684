"""Batched path (bridges_find_batched) against the oracle, graph by graph."""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu


def concat(graphs):
    u = np.concatenate([g[0] for g in graphs]).astype(np.int32) if graphs else np.zeros(0, np.int32)
    v = np.concatenate([g[1] for g in graphs]).astype(np.int32) if graphs else np.zeros(0, np.int32)
    off = np.concatenate([[0], np.cumsum([len(g[0]) for g in graphs])]).astype(np.int64)
    Vs = np.array([g[2] for g in graphs], np.int32)
    return u, v, off, Vs


def run_batch(ctx, graphs):
    u, v, off, Vs = concat(graphs)
    du = torch.from_numpy(u).cuda()
    dv = torch.from_numpy(v).cuda()
    out, counts, out_off = ctx.find_batched(du, dv, off, Vs)
    out = out.cpu().numpy()
    counts = counts.cpu().numpy()
    res = []
    for g in range(len(graphs)):
        n = int(counts[g])
        res.append(n if n < 0 else out[out_off[g]: out_off[g] + 2 * n].reshape(n, 2))
    return res


@pytest.fixture(scope="module")
def ctx(cuda_lib):
    return cuda_lib.Context(device="cuda:0")


def test_random_small_graphs(ctx):
    rng = np.random.default_rng(31)
    graphs = []
    for t in range(300):
        V = int(rng.integers(1, 200))
        E = int(rng.integers(0, 4 * V + 1))
        u, v = graphgen.random_multigraph(50000 + t, V, E)
        graphs.append((u, v, V))
    res = run_batch(ctx, graphs)
    for (u, v, V), got in zip(graphs, res):
        assert got.tolist() == oracle.dfs_bridges(u, v, V).tolist()


def test_batched_workload_specs(ctx):
    graphs = []
    for i in range(48):
        g = graphgen.generate(graphgen.workload_spec("batched", 3, i))
        graphs.append((g.u, g.v, g.V, g.planted))
    res = run_batch(ctx, [(a, b, c) for a, b, c, _ in graphs])
    for (u, v, V, planted), got in zip(graphs, res):
        ref = oracle.bridges(u, v, V, 4)
        assert got.tolist() == ref.tolist()
        assert {tuple(x) for x in planted.tolist()} <= {tuple(x) for x in got.tolist()}


def test_split_partitions_and_large_graphs(ctx, cuda_lib):
    """Force partitioning (certificates merged by the last block) and include graphs above the
    shared-memory size (single-graph path)."""
    graphs = []
    for i in range(6):
        g = graphgen.generate(graphgen.workload_spec("batched", 3, 100 + i))
        graphs.append((g.u, g.v, g.V))
    big = graphgen.workload("small")  # V = 2088: still shared memory, many edges
    graphs.append((big.u, big.v, big.V))
    n = 9000  # above 4096 vertices: a tree plus a few cycles
    rng = np.random.default_rng(4)
    par = (rng.random(n - 1) * np.arange(1, n)).astype(np.int32)
    ch = np.arange(1, n, dtype=np.int32)
    graphs.append((np.concatenate([par, [5, 77]]).astype(np.int32), np.concatenate([ch, [8000, 3]]).astype(np.int32), n))
    ctx2 = cuda_lib.Context(device="cuda:0")
    ctx2.set_batch_split(1000)
    for c in (ctx, ctx2):
        res = run_batch(c, graphs)
        for (u, v, V), got in zip(graphs, res):
            assert got.tolist() == oracle.dfs_bridges(u, v, V).tolist()


def test_small_batch_automatic_split(cuda_lib):
    """A small batch of large dense graphs: the automatic split (the batch's edges over three
    certification groups per SM, at least 2^17 edges) cuts each graph into many partitions whose
    certificates the bridge stage merges; every graph equals the oracle.  The same graphs with the
    split left at 2^20 (set explicitly) take fewer partitions and must give the same lists."""
    graphs = []
    for i, (V, p) in enumerate([(4000, 0.45), (3500, 0.6), (3900, 0.3), (2600, 0.8)]):
        g = graphgen.generate(graphgen.Spec(seed=900 + i, n_clusters=1, core_vertices=V - 40, p=p,
                                            n_pendant=6, n_paths=3, path_min=2, path_max=6))
        assert len(g.u) > 4 * (1 << 17)  # several partitions each at the automatic split
        graphs.append((g.u, g.v, g.V, g.planted))
    auto = cuda_lib.Context(device="cuda:0")
    fixed = cuda_lib.Context(device="cuda:0")
    fixed.set_batch_split(1 << 20)
    ref = [oracle.dfs_bridges(u, v, V).tolist() for u, v, V, _ in graphs]
    for c in (auto, fixed):
        res = run_batch(c, [(u, v, V) for u, v, V, _ in graphs])
        for (u, v, V, planted), got, r in zip(graphs, res, ref):
            assert got.tolist() == r
            assert {tuple(x) for x in planted.tolist()} <= {tuple(x) for x in got.tolist()}


def test_many_bridges_at_the_class_limits(ctx):
    """Trees and paths (every edge a bridge) at the group-size limits: 2,000 vertices (a half
    block, bitonic sort), 2,900 and 3,008 (a half block, more keys than its threads and a power of
    two above its key array: the several-keys-per-thread rank sort), 3,009 (a whole block), and a
    sparse multigraph of 2,950 vertices with many components."""
    rng = np.random.default_rng(5)
    graphs = []
    for n in (2000, 2900, 3008, 3009):
        par = (rng.random(n - 1) * np.arange(1, n)).astype(np.int32)
        graphs.append((par, np.arange(1, n, dtype=np.int32), n))
        pu = np.arange(n - 1, dtype=np.int32)
        graphs.append((pu, pu + 1, n))
    u, v = graphgen.random_multigraph(4242, 2950, 2600)
    graphs.append((u, v, 2950))
    res = run_batch(ctx, graphs)
    for (u, v, V), got in zip(graphs, res):
        assert got.tolist() == oracle.dfs_bridges(u, v, V).tolist()


def test_errors_are_per_graph(ctx):
    good = graphgen.random_multigraph(7, 20, 30)
    bad = (np.array([0, 1], np.int32), np.array([1, 50], np.int32), 10)
    res = run_batch(ctx, [(good[0], good[1], 20), bad, (good[0], good[1], 20)])
    assert res[1] == -2
    ref = oracle.dfs_bridges(good[0], good[1], 20).tolist()
    assert res[0].tolist() == ref and res[2].tolist() == ref


def test_replay_with_new_inputs(ctx):
    """The cached CUDA graph is replayed with different graphs and pointers."""
    for seed in range(3):
        graphs = []
        for t in range(20):
            V = 30 + 10 * t
            u, v = graphgen.random_multigraph(seed * 1000 + t, V, 3 * V)
            graphs.append((u, v, V))
        res = run_batch(ctx, graphs)
        for (u, v, V), got in zip(graphs, res):
            assert got.tolist() == oracle.dfs_bridges(u, v, V).tolist()


def test_empty_and_degenerate(ctx):
    e = np.zeros(0, np.int32)
    res = run_batch(ctx, [(e, e, 0), (e, e, 1), (np.array([0], np.int32), np.array([0], np.int32), 1),
                          (np.array([0], np.int32), np.array([1], np.int32), 2)])
    assert [r.tolist() for r in res] == [[], [], [], [[0, 1]]]


def test_rmat_graphs_all_group_sizes(ctx):
    """Skewed-degree graphs of every group size: whole-block (V > 2048), half-block (1025-2048)
    and quarter-block (<= 1024) tasks in one launch, each against the oracle."""
    graphs = []
    for t, scale in enumerate([6, 8, 10, 10, 11, 11, 12, 12] * 6):
        V = 1 << scale
        if t % 3 == 0:
            V -= t  # ragged sizes: not every graph a power of two
        u, v = graphgen.rmat(300 + t, scale, 8 << scale)
        keep = (u < V) & (v < V)
        graphs.append((u[keep], v[keep], V))
    assert any(V > 2048 for _, _, V in graphs) and any(1024 < V <= 2048 for _, _, V in graphs)
    res = run_batch(ctx, graphs)
    for (u, v, V), got in zip(graphs, res):
        assert got.tolist() == oracle.dfs_bridges(u, v, V).tolist()


def test_back_to_back_batches_on_two_streams(ctx):
    """Batches enqueued without a host wait, on one stream and alternating between two: each
    batch's descriptors are uploaded while the one before may still run (two staging copies in
    turn, the shared device area ordered by an event), and every graph of every batch must still
    come out right."""
    rng = np.random.default_rng(44)
    batches = []
    for b in range(6):
        graphs = []
        for t in range(24):
            V = int(rng.choice([int(rng.integers(2, 300)), int(rng.integers(1100, 2048)), int(rng.integers(2100, 4096))]))
            u, v = graphgen.random_multigraph(7000 + 100 * b + t, V, int(rng.integers(V, 6 * V)))
            graphs.append((u, v, V))
        u, v, off, Vs = concat(graphs)
        batches.append((graphs, torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), off, Vs))
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    results = []
    for b, (graphs, du, dv, off, Vs) in enumerate(batches):
        s = streams[[0, 1, 0, 0, 1, 1][b]]
        results.append(ctx.find_batched(du, dv, off, Vs, stream=s, sync=False))
    torch.cuda.synchronize()
    for (graphs, *_), (out, counts, out_off) in zip(batches, results):
        out = out.cpu().numpy()
        counts = counts.cpu().numpy()
        for g, (u, v, V) in enumerate(graphs):
            n = int(counts[g])
            assert out[out_off[g]: out_off[g] + 2 * n].reshape(n, 2).tolist() == oracle.dfs_bridges(u, v, V).tolist()


def _tuning_batch():
    """Graphs of every size bucket: the batched workload's specs, a few dense graphs large
    enough to be split into partitions under small split values, and sparse multigraphs."""
    graphs = []
    for i in range(160):
        g = graphgen.generate(graphgen.workload_spec("batched", 13, i))
        graphs.append((np.array(g.u), np.array(g.v), g.V))
    for i, V in enumerate((3000, 4096)):
        g = graphgen.generate(graphgen.Spec(seed=70 + i, n_clusters=2, core_vertices=V - 4, p=0.6, n_pendant=4))
        graphs.append((np.array(g.u), np.array(g.v), g.V))
    for t in range(20):
        V = 40 + 97 * t
        u, v = graphgen.random_multigraph(880 + t, V, 3 * V)
        graphs.append((u, v, V))
    return graphs


def test_tuned_plan_gives_the_oracle_graph_by_graph(cuda_lib):
    """bridges_batch_autotune changes scheduling only: under the tuned plan, and under a hand-set
    plan that forces every choice away from the automatic one (whole blocks for small graphs,
    partitions of 2^12 edges, the shortest warm-up), every graph's bridges equal the oracle's."""
    graphs = _tuning_batch()
    refs = [oracle.dfs_bridges(u, v, V).tolist() for u, v, V in graphs]
    ctx = cuda_lib.Context(device="cuda:0")
    u, v, off, Vs = concat(graphs)
    plan, us = ctx.batch_autotune(torch.from_numpy(u).cuda(), torch.from_numpy(v).cuda(), off, Vs, reps=2)
    assert us > 0 and [d["vmax"] for d in plan] == [256, 512, 1024, 2048, 4096]
    assert ctx.get_batch_plan() == plan
    for got, ref in zip(run_batch(ctx, graphs), refs):
        assert got.tolist() == ref
    forced = [{"vmax": b, "group": 1024, "split": 1 << 12, "warm_per_v": 1, "warm_add": 1}
              for b in (256, 512, 1024, 2048, 4096)]
    ctx.set_batch_plan(forced)
    for got, ref in zip(run_batch(ctx, graphs), refs):
        assert got.tolist() == ref
    quarter = [{"vmax": 4096, "group": 256, "split": 0, "warm_per_v": 8, "warm_add": 2048}]  # raised where needed
    ctx.set_batch_plan(quarter)
    for got, ref in zip(run_batch(ctx, graphs), refs):
        assert got.tolist() == ref
    with pytest.raises(cuda_lib.BridgesError):
        ctx.set_batch_plan([{"vmax": 4096, "group": 300, "split": 0, "warm_per_v": 0, "warm_add": 0}])
