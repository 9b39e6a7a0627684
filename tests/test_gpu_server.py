"""Serving (continuous batching): every result equals the same graph computed alone."""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.int32)).cuda()


def mixed_graphs():
    gs = []
    for i in range(24):  # small dense graphs (batched launches)
        g = graphgen.generate(graphgen.workload_spec("batched", 5, i))
        gs.append((g.u.copy(), g.v.copy(), g.V))
    for i in range(40):  # served specs; some have V > 4096 (single-graph path)
        s = graphgen.workload_spec("served", 4, i)
        if s.core_vertices > 20000:
            continue
        g = graphgen.generate(s)
        gs.append((g.u.copy(), g.v.copy(), g.V))
        if len(gs) >= 34:
            break
    for t in range(10):  # sparse random multigraphs
        V = 50 + 37 * t
        u, v = graphgen.random_multigraph(777 + t, V, 2 * V)
        gs.append((u, v, V))
    return gs


def test_mix_equals_alone(cuda_lib):
    graphs = mixed_graphs()
    assert any(V > 4096 for _, _, V in graphs) and any(V <= 4096 for _, _, V in graphs)
    ctx = cuda_lib.Context(device="cuda:0")
    dgraphs = [(dev(u), dev(v), V) for u, v, V in graphs]
    alone = [ctx.find(u, v, V).cpu().numpy() for u, v, V in dgraphs]
    srv = cuda_lib.Server(device="cuda:0", max_slots=4)
    for rep in range(2):
        tickets = [srv.submit(u, v, V) for u, v, V in dgraphs]
        for (u, v, V), t, ref, g in zip(dgraphs, tickets, alone, graphs):
            got, lat = srv.wait(t)
            assert got.cpu().numpy().tolist() == ref.tolist()
            assert lat >= 0
    st = srv.stats()
    assert st["completed"] == 2 * len(graphs) and st["batches"] >= 1 and st["singles"] >= 1
    assert st["max_in_flight"] >= 2
    # the results are also the oracle's
    for (u, v, V), ref in list(zip(graphs, alone))[::5]:
        assert ref.tolist() == oracle.dfs_bridges(u, v, V).tolist()
    srv.close()


def test_arrivals_while_running(cuda_lib):
    """Requests submitted while a large one runs are admitted alongside it."""
    big = graphgen.workload("mid")
    small = [graphgen.generate(graphgen.workload_spec("batched", 6, i)) for i in range(16)]
    srv = cuda_lib.Server(device="cuda:0", max_slots=3)
    tb = srv.submit(dev(big.u), dev(big.v), big.V)
    ts = [srv.submit(dev(g.u), dev(g.v), g.V) for g in small]
    for g, t in zip(small, ts):
        got, _ = srv.wait(t)
        assert {tuple(x) for x in g.planted.tolist()} <= {tuple(x) for x in got.cpu().numpy().tolist()}
    got, _ = srv.wait(tb)
    assert got.cpu().numpy().tolist() == big.planted.tolist()
    srv.close()


def test_budget_and_errors(cuda_lib):
    srv = cuda_lib.Server(device="cuda:0", mem_budget=1 << 20, max_slots=2)
    n = 300000
    u = dev(np.arange(n - 1))
    v = dev(np.arange(1, n))
    with pytest.raises(cuda_lib.BridgesError) as ei:
        srv.submit(u, v, n)
    assert ei.value.code == -6  # EAGAIN: can never fit the budget
    t = srv.submit(dev([0, 1]), dev([1, 9]), 5)  # id out of range: that request fails alone
    with pytest.raises(cuda_lib.BridgesError) as ei:
        srv.wait(t)
    assert ei.value.code == -2
    t = srv.submit(dev([0, 1]), dev([1, 2]), 3)
    got, _ = srv.wait(t)
    assert got.cpu().numpy().tolist() == [[0, 1], [1, 2]]
    srv.close()
