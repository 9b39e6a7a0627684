"""Failure handling on the GPU without faulting it: a bounded wait that nothing satisfies ends in
BRIDGES_ETIMEDOUT and leaves the context usable; bad inputs come back as error codes."""
import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_context_survives(cuda_lib):
    ctx = cuda_lib.Context(device="cuda:0")
    flag = torch.zeros(1, dtype=torch.int32, device="cuda:0")
    assert ctx.wait_value(flag, 1, 20000) == -5  # nothing ever sets the flag
    flag.fill_(1)
    assert ctx.wait_value(flag, 1, 20000) == 0
    g = graphgen.workload("small")
    u = torch.from_numpy(np.array(g.u)).cuda()
    v = torch.from_numpy(np.array(g.v)).cuda()
    assert ctx.find(u, v, g.V, 4).cpu().numpy().tolist() == g.planted.tolist()


def test_errors_leave_context_usable(cuda_lib):
    ctx = cuda_lib.Context(device="cuda:0")
    u = torch.tensor([0, 1, 2], dtype=torch.int32, device="cuda:0")
    v = torch.tensor([1, 2, 7], dtype=torch.int32, device="cuda:0")
    for _ in range(3):
        with pytest.raises(cuda_lib.BridgesError) as ei:
            ctx.find(u, v, 5, 2)
        assert ei.value.code == -2
    v2 = torch.tensor([1, 2, 0], dtype=torch.int32, device="cuda:0")
    assert ctx.find(u, v2, 5, 2).shape == (0, 2)
    # a budget too small for the workspace: ENOMEM, nothing launched
    small = cuda_lib.Context(device="cuda:0", mem_budget=4096)
    with pytest.raises(cuda_lib.BridgesError) as ei:
        small.find(u, v2, 5)
    assert ei.value.code == -3


def test_final_stage_barrier_timeout_leaves_a_usable_context(cuda_lib):
    """The final stage's grid barrier gives up after its poll cap: one block is held back (a
    bounded sleep, a test knob) while the others wait with a short cap.  The call then returns
    BRIDGES_ETIMEDOUT -- not the count of the call before it -- and the same context, with the
    knobs cleared, gives the exact result again (the barrier's count and generation are reset
    for every call)."""
    g = graphgen.workload("small")  # 2,088 vertices: a block per 256, so 9 blocks
    u = torch.from_numpy(np.array(g.u)).cuda()
    v = torch.from_numpy(np.array(g.v)).cuda()
    ref = oracle.dfs_bridges(g.u, g.v, g.V).tolist()
    ctx = cuda_lib.Context(device="cuda:0")
    assert ctx.find(u, v, g.V, 1).cpu().numpy().tolist() == ref
    ctx.set_opts(test_barrier_polls=1000, test_hold_polls=200_000)
    for _ in range(2):
        with pytest.raises(cuda_lib.BridgesError) as ei:
            ctx.find(u, v, g.V, 1)
        assert ei.value.code == -5
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    ctx.find(u, v, g.V, 1, count_device=cnt)  # the enqueue-only form: the status lands in the count
    torch.cuda.synchronize()
    assert int(cnt.item()) == -5
    ctx.set_opts()
    assert ctx.find(u, v, g.V, 1).cpu().numpy().tolist() == ref
    assert ctx.find(u, v, g.V, 4).cpu().numpy().tolist() == ref


def test_injected_allocation_failure_leaves_the_context_usable(cuda_lib):
    """A device allocation that fails (injected with opts.test_fail_alloc: the n-th allocation of
    the context's own buffers fails as on a full device) makes that call return ENOMEM; the next
    call on the same context allocates again and gives the exact result.  Covers the workspace of
    the device-buffer path, the staging and the workspace of the host-buffer path, and the
    batched descriptors."""
    g = graphgen.workload("small")
    u = torch.from_numpy(np.array(g.u)).cuda()
    v = torch.from_numpy(np.array(g.v)).cuda()
    ref = oracle.dfs_bridges(g.u, g.v, g.V).tolist()

    ctx = cuda_lib.Context(device="cuda:0")
    ctx.set_opts(test_fail_alloc=1)  # the workspace
    with pytest.raises(cuda_lib.BridgesError) as ei:
        ctx.find(u, v, g.V, 2)
    assert ei.value.code == -3
    assert ctx.find(u, v, g.V, 2).cpu().numpy().tolist() == ref

    hu = torch.from_numpy(np.array(g.u)).pin_memory()
    hv = torch.from_numpy(np.array(g.v)).pin_memory()
    for n in (1, 2):  # the host-buffer path's staging, then its workspace
        hctx = cuda_lib.Context(device="cuda:0")
        hctx.set_opts(test_fail_alloc=n)
        with pytest.raises(cuda_lib.BridgesError) as ei:
            hctx.find_host(hu, hv, g.V, 2)
        assert ei.value.code == -3
        assert hctx.find_host(hu, hv, g.V, 2).numpy().tolist() == ref

    graphs = [graphgen.generate(graphgen.workload_spec("batched", 3, i)) for i in range(3)]
    bu = torch.from_numpy(np.concatenate([x.u for x in graphs]).astype(np.int32)).cuda()
    bv = torch.from_numpy(np.concatenate([x.v for x in graphs]).astype(np.int32)).cuda()
    off = np.concatenate([[0], np.cumsum([x.E for x in graphs])]).astype(np.int64)
    Vs = np.array([x.V for x in graphs], np.int32)
    bctx = cuda_lib.Context(device="cuda:0")
    bctx.set_opts(test_fail_alloc=1)  # the batched descriptors
    with pytest.raises(cuda_lib.BridgesError) as ei:
        bctx.find_batched(bu, bv, off, Vs)
    assert ei.value.code == -3
    out, counts, out_off = bctx.find_batched(bu, bv, off, Vs)
    out, counts = out.cpu().numpy(), counts.cpu().numpy()
    for k, x in enumerate(graphs):
        n = int(counts[k])
        assert out[out_off[k]: out_off[k] + 2 * n].reshape(n, 2).tolist() == \
            oracle.dfs_bridges(x.u, x.v, x.V).tolist()
