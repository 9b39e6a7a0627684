"""Seeded synthetic graph generators (inputs only).

Both the CPU oracle and the CUDA path consume these graphs; this package holds none of the
bridge method's arithmetic.  Graphs are undirected int32 COO edge lists in structure-of-arrays
form (``u``, ``v``), normalised so that ``u < v`` except for self-loops in the test multigraphs.

Named workloads (the sizes of the paper's dense-graph regime, Sec. 3 and Figs. 2-4):

* ``small``: 8 Erdos-Renyi clusters of 256 vertices (p=0.5), a random inter-cluster tree of
  7 edges, 40 pendant vertices and 20 inter-cluster edge pairs; seed 0.
* ``mid``: 64 clusters of 512 vertices (p=0.3), a 63-edge cluster tree, 1,000 pendant paths of
  length 1-8 and 500 extra inter-cluster edges; seed 1.
* ``large``: one ER(65,536, 0.5) core with 256 pendant random recursive trees of 1-64
  vertices and 128 two-edge vertices; seed 2 (about 1.07 G edges, 8.6 GB).
* ``batched``/``served``: per-graph parameters from :func:`workload_spec`.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, asdict

import numpy as np

from . import build as _build

_lib = None


class _Spec(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("n_clusters", ctypes.c_int32),
        ("core_vertices", ctypes.c_int32),
        ("p", ctypes.c_double),
        ("n_pendant", ctypes.c_int32),
        ("n_paths", ctypes.c_int32),
        ("path_min", ctypes.c_int32),
        ("path_max", ctypes.c_int32),
        ("n_extra_pairs", ctypes.c_int32),
        ("n_extra", ctypes.c_int32),
        ("n_trees", ctypes.c_int32),
        ("tree_min", ctypes.c_int32),
        ("tree_max", ctypes.c_int32),
        ("n_two_edge", ctypes.c_int32),
        ("shuffle", ctypes.c_int32),
        ("relabel", ctypes.c_int32),
    ]


class _Graph(ctypes.Structure):
    _fields_ = [
        ("E", ctypes.c_int64),
        ("V", ctypes.c_int32),
        ("n_planted", ctypes.c_int64),
        ("u", ctypes.POINTER(ctypes.c_int32)),
        ("v", ctypes.POINTER(ctypes.c_int32)),
        ("planted", ctypes.POINTER(ctypes.c_int32)),
        ("n_er", ctypes.c_int64),
    ]


class _Perm(ctypes.Structure):
    _fields_ = [("add", ctypes.c_uint64 * 3), ("mul", ctypes.c_uint64 * 3), ("shift", ctypes.c_int),
                ("mask", ctypes.c_uint64), ("n", ctypes.c_uint64)]


class _Layout(ctypes.Structure):
    _fields_ = [
        ("s", _Spec),
        ("Vc", ctypes.c_int64),
        ("nc", ctypes.c_int64),
        ("V", ctypes.c_int64),
        ("n_struct", ctypes.c_int64),
        ("thr", ctypes.c_uint64),
        ("kER", ctypes.c_uint64),
        ("su", ctypes.POINTER(ctypes.c_int32)),
        ("sv", ctypes.POINTER(ctypes.c_int32)),
        ("n_planted", ctypes.c_int64),
        ("planted", ctypes.POINTER(ctypes.c_int32)),
        ("rowcl", ctypes.POINTER(ctypes.c_int32)),
        ("PV", _Perm),
    ]


_dev_lib = None


def _load_dev():
    global _dev_lib
    if _dev_lib is None:
        lib = _load()
        lib.gg_layout_make.restype = ctypes.POINTER(_Layout)
        lib.gg_layout_make.argtypes = [ctypes.POINTER(_Spec)]
        lib.gg_layout_free.argtypes = [ctypes.POINTER(_Layout)]
        dev = ctypes.CDLL(_build.build_dev())
        dev.ggd_count.restype = ctypes.c_int
        dev.ggd_count.argtypes = [ctypes.POINTER(_Layout), ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.POINTER(ctypes.c_int64)]
        dev.ggd_write.restype = ctypes.c_int
        dev.ggd_write.argtypes = [ctypes.POINTER(_Layout), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        LP = ctypes.POINTER(ctypes.POINTER(_Layout))
        dev.ggd_count_many.restype = ctypes.c_int
        dev.ggd_count_many.argtypes = [LP, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_int64)]
        dev.ggd_write_many.restype = ctypes.c_int
        dev.ggd_write_many.argtypes = [LP, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.POINTER(ctypes.c_int64), ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p]
        _dev_lib = dev
    return _dev_lib


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        lib.gg_generate.restype = ctypes.POINTER(_Graph)
        lib.gg_generate.argtypes = [ctypes.POINTER(_Spec)]
        lib.gg_free.argtypes = [ctypes.POINTER(_Graph)]
        lib.gg_workload_spec.restype = ctypes.c_int
        lib.gg_workload_spec.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32,
                                         ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                         ctypes.POINTER(_Spec)]
        lib.gg_rmat.restype = None
        lib.gg_rmat.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
        lib.gg_random_multigraph.argtypes = [ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64,
                                             ctypes.c_void_p, ctypes.c_void_p]
        lib.gg_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


@dataclass
class Spec:
    seed: int = 0
    n_clusters: int = 1
    core_vertices: int = 64
    p: float = 0.5
    n_pendant: int = 0
    n_paths: int = 0
    path_min: int = 1
    path_max: int = 1
    n_extra_pairs: int = 0
    n_extra: int = 0
    n_trees: int = 0
    tree_min: int = 1
    tree_max: int = 1
    n_two_edge: int = 0
    shuffle: int = 1
    relabel: int = 1

    def _c(self) -> _Spec:
        return _Spec(**asdict(self))


class _Owned:
    """Exposes C-owned memory to numpy while holding the C handle: every array made from it keeps
    the generator's allocation alive (numpy stores this object as the array's base)."""

    def __init__(self, handle, ptr, n):
        self._handle = handle
        self.__array_interface__ = {"shape": (n,), "typestr": "<i4", "data": (ptr, True), "version": 3}

    def __del__(self):
        h = getattr(self, "_handle", None)
        if h is not None and h.refs is not None:
            h.refs -= 1
            if h.refs == 0 and _lib is not None:
                _lib.gg_free(h.ptr)
                h.refs = None


class _Handle:
    def __init__(self, ptr):
        self.ptr = ptr
        self.refs = 0


@dataclass
class Graph:
    """An undirected edge list plus the bridges planted by construction.

    ``planted`` holds the bridges the construction guarantees (pendant vertices, pendant paths
    and trees, uncovered cluster-tree edges) as sorted (a<b) pairs, shape (n, 2).  Every planted
    edge is a bridge of the graph; the converse holds when every cluster is 2-edge-connected.
    """

    u: np.ndarray
    v: np.ndarray
    V: int
    planted: np.ndarray
    spec: Spec | None = None
    n_er: int = 0

    @property
    def E(self) -> int:
        return int(self.u.shape[0])


def generate(spec: Spec) -> Graph:
    """Generates the graph of ``spec``.  The edge arrays alias C-owned memory (no copy)."""
    lib = _load()
    cs = spec._c()
    h = lib.gg_generate(ctypes.byref(cs))
    if not h:
        raise ValueError(f"invalid generator spec or out of memory: {spec}")
    g = h.contents
    E, V, npl = int(g.E), int(g.V), int(g.n_planted)
    planted = np.ctypeslib.as_array(g.planted, shape=(max(npl, 1) * 2,))[: 2 * npl].reshape(npl, 2).copy()
    handle = _Handle(h)
    if E > 0:
        handle.refs = 2
        u = np.asarray(_Owned(handle, ctypes.cast(g.u, ctypes.c_void_p).value, E))
        v = np.asarray(_Owned(handle, ctypes.cast(g.v, ctypes.c_void_p).value, E))
    else:
        lib.gg_free(h)
        u = np.zeros(0, np.int32)
        v = np.zeros(0, np.int32)
    return Graph(u=u, v=v, V=V, planted=planted, spec=spec, n_er=int(g.n_er))


@dataclass
class DeviceGraph:
    """A generated graph whose edge arrays are torch int32 tensors on a CUDA device."""

    u: object
    v: object
    V: int
    planted: np.ndarray
    n_er: int = 0

    @property
    def E(self) -> int:
        return int(self.u.shape[0])


def generate_device(spec: Spec, device="cuda", stream=None) -> DeviceGraph:
    """The graph of ``spec`` generated on a GPU, bit-identical to :func:`generate`.

    The host draws the structural part (a few thousand edges); the device draws the
    Erdos-Renyi pairs, counts them per row (one stream synchronisation to learn the edge count)
    and writes every edge at its shuffled position.  Returns once the edges are written
    (``stream`` is synchronised), so the tensors can be used on any stream."""
    import torch

    dev_lib = _load_dev()
    lib = _load()
    dev = torch.device(device)
    cs = spec._c()
    h = lib.gg_layout_make(ctypes.byref(cs))
    if not h:
        raise ValueError(f"invalid generator spec or out of memory: {spec}")
    try:
        L = h.contents
        with torch.cuda.device(dev):
            st = torch.cuda.current_stream(dev) if stream is None else stream
            sh = ctypes.c_void_p(st.cuda_stream)
            rowoff = torch.empty(int(L.Vc) + 1, dtype=torch.int64, device=dev)
            n_er = ctypes.c_int64(0)
            if dev_lib.ggd_count(h, sh, ctypes.c_void_p(rowoff.data_ptr()), ctypes.byref(n_er)) != 0:
                raise RuntimeError("ggd_count failed")
            ns = int(L.n_struct)
            E = int(n_er.value) + ns
            u = torch.empty(max(E, 1), dtype=torch.int32, device=dev)[:E]
            v = torch.empty(max(E, 1), dtype=torch.int32, device=dev)[:E]
            su = torch.from_numpy(np.ctypeslib.as_array(L.su, shape=(max(ns, 1),))[:ns].copy()).to(dev)
            sv = torch.from_numpy(np.ctypeslib.as_array(L.sv, shape=(max(ns, 1),))[:ns].copy()).to(dev)
            with torch.cuda.stream(st):
                rc = dev_lib.ggd_write(h, sh, ctypes.c_void_p(rowoff.data_ptr()), n_er.value,
                                       ctypes.c_void_p(su.data_ptr()), ctypes.c_void_p(sv.data_ptr()),
                                       ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(v.data_ptr()))
            if rc != 0:
                raise RuntimeError("ggd_write failed")
            st.synchronize()
        npl = int(L.n_planted)
        planted = np.ctypeslib.as_array(L.planted, shape=(max(npl, 1) * 2,))[: 2 * npl].reshape(npl, 2).copy()
        return DeviceGraph(u=u, v=v, V=int(L.V), planted=planted, n_er=int(n_er.value))
    finally:
        lib.gg_layout_free(h)


def generate_device_many(specs, device="cuda", stream=None):
    """The graphs of ``specs`` generated on a GPU together (two stream synchronisations in all),
    each bit-identical to :func:`generate`.  Their edge arrays are views of one device buffer."""
    import torch

    dev_lib = _load_dev()
    lib = _load()
    dev = torch.device(device)
    K = len(specs)
    if K == 0:
        return []
    handles = []
    try:
        for spec in specs:
            cs = spec._c()
            h = lib.gg_layout_make(ctypes.byref(cs))
            if not h:
                raise ValueError(f"invalid generator spec or out of memory: {spec}")
            handles.append(h)
        arr = (ctypes.POINTER(_Layout) * K)(*handles)
        Ls = [h.contents for h in handles]
        n_rows = sum(int(L.Vc) + 1 for L in Ls)
        n_struct = [int(L.n_struct) for L in Ls]
        with torch.cuda.device(dev):
            st = torch.cuda.current_stream(dev) if stream is None else stream
            sh = ctypes.c_void_p(st.cuda_stream)
            rowoff = torch.empty(n_rows + K, dtype=torch.int64, device=dev)
            n_er = (ctypes.c_int64 * K)()
            if dev_lib.ggd_count_many(arr, K, sh, ctypes.c_void_p(rowoff.data_ptr()), n_er) != 0:
                raise RuntimeError("ggd_count_many failed")
            Es = [int(n_er[k]) + n_struct[k] for k in range(K)]
            total = sum(Es)
            ub = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
            vb = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
            parts = []
            for k, L in enumerate(Ls):
                if n_struct[k]:
                    parts.append(np.ctypeslib.as_array(L.su, shape=(n_struct[k],)))
                    parts.append(np.ctypeslib.as_array(L.sv, shape=(n_struct[k],)))
            host = np.concatenate(parts) if parts else np.zeros(1, np.int32)
            sb = torch.from_numpy(host).to(dev)
            with torch.cuda.stream(st):
                rc = dev_lib.ggd_write_many(arr, K, sh, ctypes.c_void_p(rowoff.data_ptr()), n_er,
                                            ctypes.c_void_p(sb.data_ptr()), ctypes.c_void_p(ub.data_ptr()),
                                            ctypes.c_void_p(vb.data_ptr()))
            if rc != 0:
                raise RuntimeError("ggd_write_many failed")
        out, at = [], 0
        for k, L in enumerate(Ls):
            npl = int(L.n_planted)
            planted = np.ctypeslib.as_array(L.planted, shape=(max(npl, 1) * 2,))[: 2 * npl].reshape(npl, 2).copy()
            out.append(DeviceGraph(u=ub[at:at + Es[k]], v=vb[at:at + Es[k]], V=int(L.V), planted=planted,
                                   n_er=int(n_er[k])))
            at += Es[k]
        return out
    finally:
        for h in handles:
            lib.gg_layout_free(h)


WORKLOADS = {
    "small": Spec(seed=0, n_clusters=8, core_vertices=2048, p=0.5, n_pendant=40, n_extra_pairs=20),
    "mid": Spec(seed=1, n_clusters=64, core_vertices=32768, p=0.3, n_paths=1000, path_min=1, path_max=8,
                n_extra=500),
    "large": Spec(seed=2, n_clusters=1, core_vertices=65536, p=0.5, n_trees=256, tree_min=1, tree_max=64,
                  n_two_edge=128),
}


def workload(name: str, **overrides) -> Graph:
    spec = Spec(**{**asdict(WORKLOADS[name]), **overrides})
    return generate(spec)


def workload_spec(kind: str, seed: int, index: int) -> Spec:
    """Per-graph spec of the batched (V in [64, 4096], d in [0.1, 0.9]) or served
    (V in [256, 65536], d in [0.05, 0.6]) workloads."""
    lib = _load()
    out = _Spec()
    if kind == "batched":
        rc = lib.gg_workload_spec(0, seed, index, 64, 6, 0.1, 0.9, ctypes.byref(out))
    elif kind == "served":
        rc = lib.gg_workload_spec(1, seed, index, 256, 8, 0.05, 0.6, ctypes.byref(out))
    else:
        raise ValueError(kind)
    if rc != 0:
        raise ValueError(kind)
    return Spec(**{name: getattr(out, name) for name, _ in _Spec._fields_})


def random_multigraph(seed: int, V: int, E: int):
    """Seeded random multigraph with self-loops and duplicates kept (not normalised)."""
    lib = _load()
    u = np.empty(E, np.int32)
    v = np.empty(E, np.int32)
    if E:
        lib.gg_random_multigraph(seed, V, E, u.ctypes.data, v.ctypes.data)
    return u, v


def rmat(seed: int, scale: int, E: int, a: float = 0.57, b: float = 0.19, c: float = 0.19):
    """Seeded R-MAT graph on 2**scale vertices (skewed degrees; self-loops and repeats kept)."""
    if not 1 <= scale <= 30:
        raise ValueError("scale must be in [1, 30]")
    lib = _load()
    u = np.empty(E, np.int32)
    v = np.empty(E, np.int32)
    if E:
        lib.gg_rmat(seed, scale, E, a, b, c, u.ctypes.data, v.ctypes.data)
    return u, v


def num_threads() -> int:
    return int(_load().gg_num_threads())
