"""The sharded form (the paper's M machines as ranks, Sec. 3 phases) on CPU gloo ranks.

Each rank certifies its contiguous shard, the ranks exchange certificates on the paper's
merge schedule, and rank 0 finds the bridges of X_0.  Here the certificate and the final step
are the oracle's (Alg. 2 in list order, Alg. 1), so the distributed X_0 must be exactly the one
the oracle's own Sec. 3 pipeline computes with M = world partitions -- edge for edge, in order --
which checks the schedule and the merge order; the bridges must be those of the whole list."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_merge_schedule_is_the_papers_phases():
    from paper_2108_07346_gb300.sharded import merge_schedule

    assert merge_schedule(1) == []
    assert merge_schedule(2) == [[(0, 1)]]
    assert merge_schedule(3) == [[(0, 1)], [(0, 2)]]
    assert merge_schedule(5) == [[(0, 1), (2, 3)], [(0, 2)], [(0, 4)]]
    assert merge_schedule(8) == [[(0, 1), (2, 3), (4, 5), (6, 7)], [(0, 2), (4, 6)], [(0, 4)]]
    for n in range(1, 40):
        rounds = merge_schedule(n)
        assert len(rounds) == (n - 1).bit_length()  # ceil(log2 n) merge phases
        sent, received = {}, {}
        for q, rnd in enumerate(rounds):
            for recv, send in rnd:
                assert recv % (2 ** (q + 1)) == 0 and send == recv + 2 ** q
                assert send not in sent and recv not in sent  # a rank that sent is done
                sent[send] = q
                received.setdefault(recv, []).append(q)
        assert sorted(sent) == list(range(1, n))  # every rank but 0 sends exactly once
        for send, q in sent.items():  # ... after everything addressed to it has arrived
            assert all(q2 < q for q2 in received.get(send, []))


class OracleCertifier:
    """Alg. 2 and Alg. 1 from the CPU oracle, on CPU tensors."""

    device = torch.device("cpu")

    def certify(self, u, v, V):
        import oracle

        un, vn = u.numpy(), v.numpy()
        ids, f1 = oracle.certificate(un, vn, V)
        return (torch.from_numpy(un[ids].copy()), torch.from_numpy(vn[ids].copy()), torch.from_numpy(f1.copy()))

    def final(self, cu, cv, ct, V):
        import oracle

        return torch.from_numpy(oracle.dfs_bridges(cu.numpy(), cv.numpy(), V))


def _graph(kind):
    import graphgen

    if kind == "multigraph":
        u, v = graphgen.random_multigraph(91, 300, 1500)
        return u, v, 300
    g = graphgen.workload("small")
    return np.array(g.u), np.array(g.v), g.V


def _worker(rank, world, port, kind, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    from paper_2108_07346_gb300.sharded import shard_range, sharded_bridges, sharded_certificate

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        u, v, V = _graph(kind)
        lo, hi = shard_range(len(u), rank, world)
        su, sv = torch.from_numpy(u[lo:hi].copy()), torch.from_numpy(v[lo:hi].copy())
        cert = sharded_certificate(su, sv, V, OracleCertifier())
        br = sharded_bridges(su, sv, V, OracleCertifier())
        q.put((rank, None if cert is None else [c.numpy().tolist() for c in cert], br.numpy().tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,kind", [(2, "small"), (3, "small"), (3, "multigraph"), (4, "multigraph"), (5, "small")])
def test_gloo_ranks_reach_the_oracle_pipeline(world, kind):
    import oracle

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, kind, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    u, v, V = _graph(kind)
    ids, f1, _ = oracle.pipeline_certificate(u, v, V, world)
    cu, cv, ct = res[0][1]
    assert cu == u[ids].tolist() and cv == v[ids].tolist() and ct == f1.tolist()
    assert all(r[1] is None for r in res[1:])  # only rank 0 keeps a certificate
    ref = oracle.dfs_bridges(u, v, V).tolist()
    assert all(r[2] == ref for r in res)  # every rank gets the bridges of the whole list



def _worker_lost_peer(rank, world, port, mode, q):
    """Rank 1 joins the group and then never sends: it dies ("dead": the machine is gone) or hangs
    ("silent").  Rank 0, waiting for rank 1's certificate, must get an error from the exchange --
    at once for a closed connection, else after the group's timeout -- instead of waiting forever."""
    import datetime
    import time

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    from paper_2108_07346_gb300.sharded import shard_range, sharded_bridges

    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        if mode == "silent":
            time.sleep(12)  # past rank 0's 5 s wait
        os._exit(3)  # no clean-up, no message
    u, v, V = _graph("small")
    lo, hi = shard_range(len(u), rank, world)
    t0 = time.monotonic()
    try:
        sharded_bridges(torch.from_numpy(u[lo:hi].copy()), torch.from_numpy(v[lo:hi].copy()), V, OracleCertifier())
        q.put((rank, "no error", time.monotonic() - t0))
    except Exception as e:  # the exchange reports the lost peer
        q.put((rank, type(e).__name__, time.monotonic() - t0))
    q.close()
    q.join_thread()  # flush the result before leaving without tearing the group down
    os._exit(0)


@pytest.mark.parametrize("mode", ["dead", "silent"])
def test_a_lost_rank_surfaces_as_an_error_not_a_hang(mode):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_lost_peer, args=(r, 2, port, mode, q)) for r in range(2)]
    for p in procs:
        p.start()
    rank, what, waited = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
    assert rank == 0 and what == "RuntimeError", what
    assert waited < (2 if mode == "dead" else 11)  # the group's timeout is 5 s
    assert procs[0].exitcode == 0 and procs[1].exitcode == 3
