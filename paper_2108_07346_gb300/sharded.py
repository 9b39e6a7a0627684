"""The sharded form: the paper's M machines as ranks, one shard of the edge list each (Sec. 3).

Rank r of N holds the contiguous shard [E r / N, E (r+1) / N) of the list.  Phase 0: every
rank computes the certificate X_r of its shard (Alg. 2; on a GPU, ``bridges_certificate``).
Merge phases q = 1 .. ceil(log2 N): rank r with r = 0 mod 2^q receives X_{r + 2^(q-1)} (when
that rank exists) and replaces X_r by the certificate of X_r followed by the received edges;
the sender is done.  After the last phase rank 0 holds X_0, a certificate of the whole list
(|X_0| <= 2(V-1), Lemma 1), and computes its bridges (the stand-in for Alg. 1 on X_0,
``bridges_from_forest`` on its forest F and the remaining edges F'); the sorted list is then
broadcast to every rank.

Only certificates travel: at most 2(V-1) edges, three int32 words each (ends and the F flag),
sent through ``torch.distributed`` point to point (device buffers with NCCL, host buffers with
gloo).  No kernel reads another rank's memory.  Each step of the computation runs in the
library's kernels through the ``Certifier`` it is given; this module only schedules them and moves
the certificates.

A rank that dies or stops sending surfaces on the rank waiting for it as an exception from the
exchange, never as an endless wait: with gloo at once when the connection closes, else once the
process group's timeout (the ``timeout`` of ``init_process_group``) expires; the caller decides
whether to rerun the call on the surviving ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def merge_schedule(n: int):
    """The merge phases for n ranks: a list of rounds, each a list of (receiver, sender) pairs;
    round q (from 1) pairs every receiver r = 0 mod 2^q with sender r + 2^(q-1) < n."""
    if n < 1:
        raise ValueError("need at least one rank")
    rounds = []
    step = 1
    while step < n:
        rounds.append([(r, r + step) for r in range(0, n, 2 * step) if r + step < n])
        step *= 2
    return rounds


def shard_range(E: int, rank: int, world: int):
    """The contiguous shard [lo, hi) of an E-edge list held by `rank` of `world` (Sec. 3 sets U_i;
    empty past the end when world > E)."""
    return E * rank // world, E * (rank + 1) // world


class Certifier:
    """The library's kernels on one device: a certificate of an edge list and the bridges of a
    final certificate.  Tensors are int32 (and bool for the F flags) on ``ctx.device``."""

    def __init__(self, ctx):
        self.ctx = ctx
        self.device = ctx.device

    def certify(self, u, v, V: int):
        """Alg. 2 on (u, v) as one partition: (cert_u, cert_v, F flags)."""
        return self.ctx.certificate(u, v, V, 1)

    def final(self, cu, cv, ct, V: int):
        """The sorted (n, 2) bridges of the certificate (cu, cv) whose F edges are flagged in ct."""
        return self.ctx.from_forest(cu[ct].contiguous(), cv[ct].contiguous(), cu[~ct].contiguous(),
                                    cv[~ct].contiguous(), V)


def _comm_device(certifier_device, group):
    backend = dist.get_backend(group)
    return torch.device(certifier_device) if backend == "nccl" else torch.device("cpu")


def _send_cert(cu, cv, ct, dst, cdev, group):
    n = int(cu.shape[0])
    dist.send(torch.tensor([n], dtype=torch.int64, device=cdev), dst, group=group)
    if n:
        msg = torch.stack([cu.to(torch.int32), cv.to(torch.int32), ct.to(torch.int32)]).to(cdev)
        dist.send(msg.contiguous(), dst, group=group)


def _recv_cert(src, cdev, group):
    n_t = torch.zeros(1, dtype=torch.int64, device=cdev)
    dist.recv(n_t, src, group=group)
    n = int(n_t.item())
    msg = torch.empty((3, n), dtype=torch.int32, device=cdev)
    if n:
        dist.recv(msg, src, group=group)
    return msg


def sharded_certificate(u, v, V: int, certifier, group=None):
    """Phase 0 and the merge phases.  (u, v): this rank's shard on the certifier's device.
    Returns (cert_u, cert_v, F flags) of X_0 on rank 0, None on the other ranks."""
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    cdev = _comm_device(certifier.device, group)
    cu, cv, ct = certifier.certify(u, v, V)
    for rnd in merge_schedule(world):
        for recv, send in rnd:
            if rank == send:
                _send_cert(cu, cv, ct, _global(recv, group), cdev, group)
                return None
            if rank == recv:
                msg = _recv_cert(_global(send, group), cdev, group).to(certifier.device)
                mu = torch.cat([cu.to(torch.int32), msg[0]])
                mv = torch.cat([cv.to(torch.int32), msg[1]])
                cu, cv, ct = certifier.certify(mu.contiguous(), mv.contiguous(), V)
    return cu, cv, ct  # only rank 0 is never a sender


def _global(rank_in_group, group):
    return rank_in_group if group is None else dist.get_global_rank(group, rank_in_group)


def sharded_bridges(u, v, V: int, certifier, group=None):
    """The bridges of the whole list, given this rank's shard: the sorted (n, 2) int32 pairs on
    the certifier's device, on every rank."""
    rank = dist.get_rank(group)
    cdev = _comm_device(certifier.device, group)
    res = sharded_certificate(u, v, V, certifier, group)
    if rank == 0:
        cu, cv, ct = res
        br = certifier.final(cu, cv, ct, V).to(torch.int32)
        n_t = torch.tensor([br.shape[0]], dtype=torch.int64, device=cdev)
    else:
        n_t = torch.zeros(1, dtype=torch.int64, device=cdev)
    dist.broadcast(n_t, _global(0, group), group=group)
    n = int(n_t.item())
    buf = br.to(cdev).contiguous() if rank == 0 else torch.empty((n, 2), dtype=torch.int32, device=cdev)
    if n:
        dist.broadcast(buf, _global(0, group), group=group)
    return buf.to(certifier.device)
