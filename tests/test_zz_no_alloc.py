"""bridges_find_noalloc: the allocation-free entry point gives the same bridges as
bridges_find_ctx and as the CPU oracle.

Some callers cannot allocate device memory at the point where they need bridges: a framework
that owns the device allocator, a latency-critical loop that must not block in the driver, or a
process that reserved all device memory up front.  For them the library keeps all scratch in one
fixed device array.  This file is collected last so that a failure here comes after every other
test has run; it sets up everything it uses itself, so it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import graphgen
import oracle

pytestmark = pytest.mark.gpu

# the largest graph the fixed 8 MiB array holds with one partition (include/bridges.h)
V_MAX_M1 = 45_135


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_07346_gb300 as pb

    pb.load()
    return pb


def _dev(a):
    return torch.from_numpy(np.array(a, dtype=np.int32)).to("cuda:0")


def _noalloc_abi(pb, u, v, V, M, count_device=None):
    """Calls the C entry point directly through the C ABI (ctypes).  Synchronous: returns the
    (n, 2) pairs, or the negative status.  With count_device: enqueue-only, returns the output
    buffer whole after a stream synchronisation."""
    lib = pb.load()
    out = torch.empty(2 * max(V - 1, 1), dtype=torch.int32, device="cuda:0")
    stream = torch.cuda.current_stream()
    n = lib.bridges_find_noalloc(ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(u.data_ptr()),
                                 ctypes.c_void_p(v.data_ptr()), u.numel(), V, M, ctypes.c_void_p(out.data_ptr()),
                                 None if count_device is None else ctypes.c_void_p(count_device.data_ptr()))
    if count_device is not None:
        assert n == 0, pb.status_string(n)
        stream.synchronize()
        return out
    if n < 0:
        return n
    return out[: 2 * n].view(n, 2).cpu().numpy()


def test_no_alloc_matches_existing_entry_point_and_oracle_twice(pb):
    ctx = pb.Context(device="cuda:0")
    # two calls in a row on different graphs: the second must not see the first one's leftovers
    graphs = [graphgen.workload("small"), graphgen.generate(graphgen.workload_spec("batched", 3, 7))]
    for M, g in zip((4, 2), graphs):
        u, v = _dev(g.u), _dev(g.v)
        ref = ctx.find(u, v, g.V, M).cpu().numpy()
        got = _noalloc_abi(pb, u, v, g.V, M)
        assert got.tolist() == ref.tolist()
        assert got.tolist() == oracle.dfs_bridges(g.u, g.v, g.V).tolist()
    # and the first graph again, through the Python wrapper of the same symbol
    g = graphs[0]
    got = pb.bridges_find_noalloc(_dev(g.u), _dev(g.v), g.V, 4).cpu().numpy()
    assert got.tolist() == oracle.dfs_bridges(g.u, g.v, g.V).tolist()


def test_no_alloc_failed_call_then_valid_call(pb):
    """A call that sets the device status word (an id outside [0, V)) returns ERANGE; the next
    call on the same stream starts from a clean status and gives the exact result."""
    g = graphgen.generate(graphgen.workload_spec("batched", 3, 11))
    bad_v = np.array(g.v, dtype=np.int32)
    bad_v[len(bad_v) // 2] = g.V + 5
    assert _noalloc_abi(pb, _dev(g.u), _dev(bad_v), g.V, 1) == -2
    got = _noalloc_abi(pb, _dev(g.u), _dev(g.v), g.V, 1)
    assert got.tolist() == oracle.dfs_bridges(g.u, g.v, g.V).tolist()


def test_no_alloc_count_on_the_device(pb):
    """The enqueue-only form writes the count to device memory."""
    g = graphgen.workload("small")
    cnt = torch.full((1,), -99, dtype=torch.int64, device="cuda:0")
    out = _noalloc_abi(pb, _dev(g.u), _dev(g.v), g.V, 2, count_device=cnt)
    ref = oracle.dfs_bridges(g.u, g.v, g.V)
    n = int(cnt.item())
    assert n == len(ref)
    assert out[: 2 * n].view(n, 2).cpu().numpy().tolist() == ref.tolist()


def test_no_alloc_capacity_boundary(pb):
    """The documented largest graph fits (a path: every edge a bridge, sorted by the radix path of
    the final stage) and one vertex more is rejected with ENOMEM before anything runs."""
    V = V_MAX_M1
    u = np.arange(0, V - 1, dtype=np.int32)
    v = np.arange(1, V, dtype=np.int32)
    got = _noalloc_abi(pb, _dev(u), _dev(v), V, 1)
    assert got.tolist() == oracle.dfs_bridges(u, v, V).tolist()
    assert _noalloc_abi(pb, _dev(u), _dev(v), V + 1, 1) == -3


def test_no_alloc_rejects_graphs_beyond_the_fixed_scratch(pb):
    u = _dev(np.arange(0, 99_999, dtype=np.int32))
    v = _dev(np.arange(1, 100_000, dtype=np.int32))
    with pytest.raises(pb.BridgesError) as ei:
        pb.bridges_find_noalloc(u, v, 100_000, 1)
    assert ei.value.code == -3
