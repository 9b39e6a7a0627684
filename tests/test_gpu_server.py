"""Serving (continuous batching): every result equals the same graph computed alone."""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.array(a, dtype=np.int32)).cuda()


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
    # every result is also the oracle's
    for (u, v, V), ref in zip(graphs, alone):
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
        assert got.cpu().numpy().tolist() == oracle.dfs_bridges(g.u, g.v, g.V).tolist()
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


def test_client_threads_and_an_abandoned_ticket(cuda_lib):
    """Several client threads submit and wait concurrently; one thread dies right after
    submitting (its ticket is never waited on).  The others get their exact results, the server
    still completes the abandoned request, and closing it does not hang."""
    import threading

    graphs = [graphgen.generate(graphgen.workload_spec("batched", 8, i)) for i in range(24)]
    refs = [oracle.dfs_bridges(g.u, g.v, g.V).tolist() for g in graphs]
    dgraphs = [(dev(g.u), dev(g.v), g.V) for g in graphs]
    srv = cuda_lib.Server(device="cuda:0", max_slots=3)
    errors = []

    def client(k):
        try:
            for i in range(k, len(dgraphs), 4):
                u, v, V = dgraphs[i]
                got, _ = srv.wait(srv.submit(u, v, V))
                if got.cpu().numpy().tolist() != refs[i]:
                    errors.append(i)
        except Exception as e:  # surfaced below
            errors.append(repr(e))

    def dying_client():
        u, v, V = dgraphs[0]
        srv.submit(u, v, V)  # the thread ends without waiting for its ticket

    threads = [threading.Thread(target=client, args=(k,)) for k in range(4)] + [threading.Thread(target=dying_client)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=120)
        assert not t.is_alive()
    assert errors == []
    import time

    for _ in range(1000):  # the abandoned request completes on its own
        if srv.stats()["completed"] >= len(dgraphs) + 1:
            break
        time.sleep(0.01)
    assert srv.stats()["completed"] == len(dgraphs) + 1 and srv.stats()["failures"] == 0
    srv.close()


def test_cancel_withdraws_queued_requests(cuda_lib):
    """With one slot busy on a large graph, requests queued behind it can be withdrawn: their wait
    raises BRIDGES_ECANCELED, the others complete with the oracle's bridges, and a request that
    already runs cannot be withdrawn.  The slot stays busy for a known time: the test knob that
    holds one block of the final stage back (a bounded sleep of about 30 ms per large request)
    keeps the queue from draining before the cancels, however fast the GPU runs the graph."""
    big = graphgen.workload("mid")
    small = [graphgen.generate(graphgen.workload_spec("batched", 9, i)) for i in range(12)]
    srv = cuda_lib.Server(device="cuda:0", max_slots=1, test_hold_polls=300_000)
    bu, bv = dev(big.u), dev(big.v)
    su = [(dev(g.u), dev(g.v)) for g in small]
    tb = srv.submit(bu, bv, big.V)
    ts = [srv.submit(u, v, g.V) for (u, v), g in zip(su, small)]
    cancelled = [srv.cancel(t) for t in ts[::2]]
    assert any(cancelled)
    for k, (g, t) in enumerate(zip(small, ts)):
        if k % 2 == 0 and cancelled[k // 2]:
            with pytest.raises(cuda_lib.BridgesError) as ei:
                srv.wait(t)
            assert ei.value.code == -9
        else:
            got, _ = srv.wait(t)
            assert got.cpu().numpy().tolist() == oracle.dfs_bridges(g.u, g.v, g.V).tolist()
    got, _ = srv.wait(tb)
    assert got.cpu().numpy().tolist() == big.planted.tolist()
    t = srv.submit(dev(big.u), dev(big.v), big.V)
    import time

    time.sleep(0.05)  # long enough for an idle scheduler to launch it
    assert srv.cancel(t) is False
    assert srv.wait(t)[0].cpu().numpy().tolist() == big.planted.tolist()
    with pytest.raises(cuda_lib.BridgesError):
        srv.cancel(t)  # released
    srv.close()
