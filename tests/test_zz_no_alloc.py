"""bridges_find_noalloc: the allocation-free entry point gives the same bridges as bridges_find_ctx.

For callers that cannot allocate device memory, the library keeps all scratch in one fixed
device array.  This file is collected last so that a failure here comes after every other test
has run; it sets up everything it uses itself, so it also passes alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

import graphgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2108_07346_gb300 as pb

    pb.load()
    return pb


def _dev(a):
    return torch.from_numpy(np.array(a, dtype=np.int32)).to("cuda:0")


def _noalloc_abi(pb, u, v, V, M):
    """Calls the C entry point directly through the C ABI (ctypes), synchronously."""
    lib = pb.load()
    out = torch.empty(2 * max(V - 1, 1), dtype=torch.int32, device="cuda:0")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = lib.bridges_find_noalloc(stream, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()), u.numel(),
                                 V, M, ctypes.c_void_p(out.data_ptr()), None)
    assert n >= 0, pb.status_string(n)
    return out[: 2 * n].view(n, 2).cpu().numpy()


def test_noalloc_matches_existing_entry_point_twice(pb):
    ctx = pb.Context(device="cuda:0")
    # two calls in a row on different graphs: the second must not see the first one's leftovers
    graphs = [graphgen.workload("small"), graphgen.generate(graphgen.workload_spec("batched", 3, 7))]
    for M, g in zip((4, 2), graphs):
        u, v = _dev(g.u), _dev(g.v)
        ref = ctx.find(u, v, g.V, M).cpu().numpy()
        got = _noalloc_abi(pb, u, v, g.V, M)
        assert got.tolist() == ref.tolist()
        assert got.tolist() == g.planted.tolist() or set(map(tuple, g.planted.tolist())) <= set(map(tuple, got.tolist()))
    # and the same graph again, through the Python wrapper of the same symbol
    g = graphs[0]
    assert pb.bridges_find_noalloc(_dev(g.u), _dev(g.v), g.V, 4).cpu().numpy().tolist() == g.planted.tolist()


def test_noalloc_rejects_graphs_beyond_the_fixed_scratch(pb):
    u = _dev(np.arange(0, 99_999, dtype=np.int32))
    v = _dev(np.arange(1, 100_000, dtype=np.int32))
    with pytest.raises(pb.BridgesError) as ei:
        pb.bridges_find_noalloc(u, v, 100_000, 1)
    assert ei.value.code == -3
