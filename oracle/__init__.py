"""CPU oracle for the sparse-certificate bridge method (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import this package.  It shares no code with the CUDA path.

Every function takes an undirected edge list as two int32 arrays ``u``, ``v`` and the vertex
count ``V`` and returns bridges as an (n, 2) int32 array of (a < b) pairs sorted ascending.
See ``oracle.c`` for the passage of the paper each function follows.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests (hand-derived
fixtures, closed forms, brute force, planted bridges, certificate invariants and, where networkx
is installed, that library's independent routines on random simple graphs); none is "parity
unpinned".
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import build as _build

_lib = None
_I32P = ctypes.c_void_p


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(_build.build())
        for name in ("oracle_dfs_bridges", "oracle_chain_bridges", "oracle_brute_bridges"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int64
            f.argtypes = [_I32P, _I32P, ctypes.c_int64, ctypes.c_int32, _I32P]
        lib.oracle_bridges.restype = ctypes.c_int64
        lib.oracle_bridges.argtypes = [_I32P, _I32P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, _I32P]
        lib.oracle_certificate_stream.restype = ctypes.c_int64
        lib.oracle_certificate_stream.argtypes = [_I32P, _I32P, ctypes.c_int64, ctypes.c_int32, _I32P, _I32P]
        lib.oracle_certificate.restype = ctypes.c_int64
        lib.oracle_certificate.argtypes = [_I32P, _I32P, ctypes.c_int64, ctypes.c_int32, _I32P, _I32P]
        lib.oracle_pipeline_cert.restype = ctypes.c_int64
        lib.oracle_pipeline_cert.argtypes = [_I32P, _I32P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                             _I32P, _I32P, _I32P, _I32P]
        for name in ("oracle_articulation_points", "oracle_brute_articulation"):
            f = getattr(lib, name)
            f.restype = ctypes.c_int64
            f.argtypes = [_I32P, _I32P, ctypes.c_int64, ctypes.c_int32, _I32P]
        lib.oracle_is_articulation.restype = ctypes.c_int32
        lib.oracle_is_articulation.argtypes = [_I32P, _I32P, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32]
        lib.oracle_block_certificate.restype = ctypes.c_int64
        lib.oracle_block_certificate.argtypes = [_I32P, _I32P, ctypes.c_int64, ctypes.c_int32, _I32P, _I32P, _I32P,
                                                 _I32P]
        lib.oracle_two_edge_components.restype = ctypes.c_int32
        lib.oracle_two_edge_components.argtypes = [_I32P, _I32P, ctypes.c_int64, ctypes.c_int32, _I32P]
        lib.oracle_components.restype = ctypes.c_int32
        lib.oracle_components.argtypes = [_I32P, _I32P, ctypes.c_int64, ctypes.c_int32, _I32P]
        _lib = lib
    return _lib


def _edges(u, v):
    u = np.ascontiguousarray(u, dtype=np.int32)
    v = np.ascontiguousarray(v, dtype=np.int32)
    if u.shape != v.shape or u.ndim != 1:
        raise ValueError("u and v must be 1-D arrays of equal length")
    return u, v


def _check(rc):
    if rc == -1:
        raise ValueError("invalid input: vertex id outside [0, V) or negative size")
    if rc == -2:
        raise MemoryError("oracle allocation failed")
    return rc


def _bridge_call(name, u, v, V, *extra):
    u, v = _edges(u, v)
    out = np.empty(2 * max(V, 1), np.int32)
    n = _check(getattr(_load(), name)(u.ctypes.data, v.ctypes.data, u.shape[0], V, *extra, out.ctypes.data))
    return out[: 2 * n].reshape(n, 2).copy()


def bridges(u, v, V: int, M: int = 1) -> np.ndarray:
    """Sec. 3 end to end: M-way partition, certificates, merge phases, then Alg. 1 on X_0."""
    return _bridge_call("oracle_bridges", u, v, V, M)


def dfs_bridges(u, v, V: int) -> np.ndarray:
    """Alg. 1 (iterative Tarjan disc/low) on the whole edge list."""
    return _bridge_call("oracle_dfs_bridges", u, v, V)


def chain_bridges(u, v, V: int) -> np.ndarray:
    """Schmidt's chain decomposition on the whole edge list (independent of Alg. 1)."""
    return _bridge_call("oracle_chain_bridges", u, v, V)


def brute_bridges(u, v, V: int) -> np.ndarray:
    """The definition: an edge is a bridge iff deleting it disconnects its ends (BFS)."""
    return _bridge_call("oracle_brute_bridges", u, v, V)


def certificate(u, v, V: int):
    """Alg. 2 on the whole list: (edge ids of S, F-membership flags)."""
    u, v = _edges(u, v)
    ids = np.empty(max(2 * V, 1), np.int64)
    f1 = np.empty(max(2 * V, 1), np.uint8)
    k = _check(_load().oracle_certificate(u.ctypes.data, v.ctypes.data, u.shape[0], V, ids.ctypes.data,
                                          f1.ctypes.data))
    return ids[:k].copy(), f1[:k].astype(bool)


def certificate_stream(u, v, V: int):
    """Alg. 2 as one streaming pass (F, else F'): (edge ids of S in list order, F flags)."""
    u, v = _edges(u, v)
    ids = np.empty(max(2 * V, 1), np.int64)
    f1 = np.empty(max(2 * V, 1), np.uint8)
    k = _check(_load().oracle_certificate_stream(u.ctypes.data, v.ctypes.data, u.shape[0], V, ids.ctypes.data,
                                                 f1.ctypes.data))
    return ids[:k].copy(), f1[:k].astype(bool)


def pipeline_certificate(u, v, V: int, M: int):
    """Sec. 3 certificate pipeline: (ids of X_0, F flags of X_0, max |X_i| after each phase)."""
    u, v = _edges(u, v)
    ids = np.empty(max(2 * V + 2, 1), np.int64)
    f1 = np.empty(max(2 * V + 2, 1), np.uint8)
    pm = np.zeros(64, np.int64)
    nq = np.zeros(1, np.int32)
    k = _check(_load().oracle_pipeline_cert(u.ctypes.data, v.ctypes.data, u.shape[0], V, M, ids.ctypes.data,
                                            f1.ctypes.data, pm.ctypes.data, nq.ctypes.data))
    return ids[:k].copy(), f1[:k].astype(bool), pm[: int(nq[0])].copy()


def components(u, v, V: int):
    """(number of components, label per vertex = min vertex id of its component)."""
    u, v = _edges(u, v)
    lab = np.empty(max(V, 1), np.int32)
    c = _check(_load().oracle_components(u.ctypes.data, v.ctypes.data, u.shape[0], V, lab.ctypes.data))
    return int(c), lab[:V].copy()


def two_edge_components(u, v, V: int):
    """(number of 2-edge-connected components, label per vertex = min vertex of its component):
    the components of the graph after deleting its bridges."""
    u, v = _edges(u, v)
    lab = np.empty(max(V, 1), np.int32)
    c = _check(_load().oracle_two_edge_components(u.ctypes.data, v.ctypes.data, u.shape[0], V, lab.ctypes.data))
    return int(c), lab[:V].copy()


def _vertex_call(name, u, v, V):
    u, v = _edges(u, v)
    out = np.empty(max(V, 1), np.int32)
    n = _check(getattr(_load(), name)(u.ctypes.data, v.ctypes.data, u.shape[0], V, out.ctypes.data))
    return out[:n].copy()


def articulation_points(u, v, V: int) -> np.ndarray:
    """Articulation points (sorted vertex ids) by Tarjan's DFS low/disc test."""
    return _vertex_call("oracle_articulation_points", u, v, V)


def brute_articulation(u, v, V: int) -> np.ndarray:
    """The definition: vertices whose deletion increases the number of components."""
    return _vertex_call("oracle_brute_articulation", u, v, V)


def is_articulation(u, v, V: int, x: int) -> bool:
    """The definition for one vertex: does deleting x increase the number of components?"""
    u, v = _edges(u, v)
    return bool(_check(_load().oracle_is_articulation(u.ctypes.data, v.ctypes.data, u.shape[0], V, int(x))))


def block_certificate(u, v, V: int):
    """Tree edges T plus the edges that merge fundamental-cycle classes, in input order:
    (edge ids, tree flags, articulation points derived from the classes)."""
    u, v = _edges(u, v)
    ids = np.empty(max(2 * V, 1), np.int64)
    tr = np.empty(max(2 * V, 1), np.uint8)
    pts = np.empty(max(V, 1), np.int32)
    npt = np.zeros(1, np.int64)
    k = _check(_load().oracle_block_certificate(u.ctypes.data, v.ctypes.data, u.shape[0], V, ids.ctypes.data,
                                                tr.ctypes.data, pts.ctypes.data, npt.ctypes.data))
    return ids[:k].copy(), tr[:k].astype(bool), pts[: int(npt[0])].copy()


def rooted_forest(tu, tv, V: int, child_key=None):
    """The rooted, numbered forest that Alg. 1's depth-first search walks, for a spanning forest
    given as edges (tu, tv): every tree is rooted at its minimum vertex, the trees are searched in
    increasing order of their roots, and one global counter numbers the vertices in the order the
    search discovers them (Alg. 1's disc with the global timer of reading 7, counted from 0).
    Siblings are visited in increasing ``child_key`` (default: vertex id).

    Returns (parent, pre, size) as int32 arrays of length V: parent -1 for roots, size = vertices
    in the subtree.  Pure Python (an explicit stack); raises ValueError if the edges contain a
    cycle or an id outside [0, V)."""
    tu = np.asarray(tu, dtype=np.int64).ravel()
    tv = np.asarray(tv, dtype=np.int64).ravel()
    if tu.shape != tv.shape:
        raise ValueError("tu and tv differ in length")
    if tu.size and (min(tu.min(), tv.min()) < 0 or max(tu.max(), tv.max()) >= V):
        raise ValueError("vertex id outside [0, V)")
    key = np.arange(V) if child_key is None else np.asarray(child_key)
    adj = [[] for _ in range(V)]
    for a, b in zip(tu.tolist(), tv.tolist()):
        adj[a].append(b)
        adj[b].append(a)
    parent = np.full(V, -1, np.int32)
    pre = np.full(V, -1, np.int32)
    size = np.zeros(V, np.int32)
    clock = 0
    for r in range(V):  # the first unvisited vertex of a tree is its minimum
        if pre[r] >= 0:
            continue
        pre[r] = clock
        clock += 1
        order = [r]
        # each vertex's unvisited neighbours in key order (its parent's edge left out once)
        stack = [(r, iter(sorted(adj[r], key=lambda y: key[y])))]
        while stack:
            x, it = stack[-1]
            y = next(it, None)
            if y is None:
                stack.pop()
                continue
            if pre[y] >= 0:  # reached twice: a cycle (or a doubled edge)
                raise ValueError("the edges contain a cycle")
            parent[y] = x
            pre[y] = clock
            clock += 1
            order.append(y)
            rest = list(adj[y])
            rest.remove(x)  # the edge to the parent, once
            stack.append((y, iter(sorted(rest, key=lambda z: key[z]))))
        for x in reversed(order):  # subtree sizes, children before parents
            size[x] += 1
            if parent[x] >= 0:
                size[parent[x]] += size[x]
    return parent, pre, size
