"""The device form of the input generator gives the host generator's graphs bit for bit.

Inputs only: the served benchmark draws one fresh graph per request on the GPU, so its graphs
must be exactly the ones the oracle regenerates on the host for its sampled checks."""
import dataclasses

import numpy as np
import pytest
import torch

import graphgen

pytestmark = pytest.mark.gpu


def specs():
    out = [("small", graphgen.WORKLOADS["small"]), ("mid", graphgen.WORKLOADS["mid"]),
           ("large p=0.01", dataclasses.replace(graphgen.WORKLOADS["large"], p=0.01)),
           ("unshuffled", graphgen.Spec(seed=3, n_clusters=3, core_vertices=100, p=0.7, n_pendant=5, shuffle=0,
                                        relabel=0))]
    out += [(f"served {i}", graphgen.workload_spec("served", 4, i)) for i in range(8)]
    out += [(f"batched {i}", graphgen.workload_spec("batched", 3, i)) for i in range(8)]
    return out


@pytest.mark.parametrize("name,spec", specs(), ids=[n for n, _ in specs()])
def test_device_graph_equals_host_graph(name, spec):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = graphgen.generate(spec)
    d = graphgen.generate_device(spec, "cuda:0")
    assert d.V == h.V and d.E == h.E and d.n_er == h.n_er
    assert np.array_equal(d.u.cpu().numpy(), h.u) and np.array_equal(d.v.cpu().numpy(), h.v)
    assert np.array_equal(d.planted, h.planted)


def test_many_at_once_equal_host_graphs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    specs_ = [s for _, s in specs()][3:]
    many = graphgen.generate_device_many(specs_, "cuda:0")
    for spec, d in zip(specs_, many):
        h = graphgen.generate(spec)
        assert d.V == h.V and d.E == h.E
        assert np.array_equal(d.u.cpu().numpy(), h.u) and np.array_equal(d.v.cpu().numpy(), h.v)
        assert np.array_equal(d.planted, h.planted)
