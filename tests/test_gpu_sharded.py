"""The sharded form on the GPU: ranks (processes, all on cuda:0) certify their shards of the
list with the library's kernels, exchange certificates over a host-staged gloo channel on the
paper's merge schedule (Sec. 3 phases), and rank 0 finds the bridges of X_0.  No kernel of one
process waits for the other: every exchange is a host-side send and receive between launches.
The bridges must equal the oracle's on the whole list, bit for bit."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# about 300 M edges at the large workload's density: ER(34,640, 0.5) plus planted trees
DENSE_300M = dict(seed=5, n_clusters=1, core_vertices=34_640, p=0.5, n_trees=64, tree_min=1, tree_max=64,
                  n_two_edge=32)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _spec(kind):
    import graphgen

    return graphgen.WORKLOADS["mid"] if kind == "mid" else graphgen.Spec(**DENSE_300M)


def _worker(rank, world, port, kind, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import graphgen
    import paper_2108_07346_gb300 as pb
    from paper_2108_07346_gb300.sharded import Certifier, shard_range, sharded_bridges

    try:
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        dist.init_process_group("gloo", rank=rank, world_size=world)
        g = graphgen.generate_device(_spec(kind), dev)
        lo, hi = shard_range(g.E, rank, world)
        u, v, V = g.u[lo:hi].contiguous(), g.v[lo:hi].contiguous(), g.V
        del g
        br = sharded_bridges(u, v, V, Certifier(pb.Context(device=dev)))
        q.put((rank, br.cpu().numpy().tobytes(), int(br.shape[0])))
        dist.destroy_process_group()
    except Exception as e:  # reported to the parent
        q.put((rank, repr(e), -1))


@pytest.mark.parametrize("kind,world", [("mid", 2), ("mid", 3), pytest.param("dense300m", 2, marks=pytest.mark.slow)])
def test_ranks_on_one_gpu_match_the_oracle(kind, world):
    """Two ranks (one merge phase) and three (two phases, the second with an odd rank out)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import graphgen
    import oracle

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, kind, q)) for r in range(world)]
    for p in procs:
        p.start()
    g = graphgen.generate(_spec(kind))
    ref = oracle.dfs_bridges(g.u, g.v, g.V)
    res = sorted((q.get(timeout=600) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
    for rank, payload, n in res:
        assert n >= 0, f"rank {rank}: {payload}"
        got = np.frombuffer(payload, dtype=np.int32).reshape(n, 2)
        assert np.array_equal(got, ref)
    assert np.array_equal(ref, g.planted)  # the planted bridges are all of them here
    assert all(p.exitcode == 0 for p in procs)
