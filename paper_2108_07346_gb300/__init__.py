"""Bridges of dense graphs via sparse certificates on one GB300 GPU (arXiv:2108.07346).

A thin ctypes binding over ``libbridges.so`` (C ABI in ``include/bridges.h``).  Every step of
the computation runs in the library's CUDA kernels; this module only marshals arguments.
PyTorch supplies device memory (input/output tensors, optional workspace) and streams.  There
is no CPU fallback: if the library cannot be built or loaded, every call raises.

Functions keep the C names:

* :func:`bridges_find` -- plain call on device tensors (default context, current stream).
* :class:`Context` -- ``find`` (device tensors), ``find_host`` (host tensors, copies inside),
  ``certificate`` (the Sec. 3 certificate), ``from_forest`` (the final stage alone), and the
  introspection calls ``stage_ms``, ``launches``, ``last_config``.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

_lib = None

STATUS = {
    0: "BRIDGES_OK",
    -1: "BRIDGES_EINVAL",
    -2: "BRIDGES_ERANGE",
    -3: "BRIDGES_ENOMEM",
    -4: "BRIDGES_ECUDA",
    -5: "BRIDGES_ETIMEDOUT",
    -6: "BRIDGES_EAGAIN",
    -7: "BRIDGES_EBUSY",
    -8: "BRIDGES_EINTERNAL",
    -9: "BRIDGES_ECANCELED",
}


class BridgesError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = int(code)
        super().__init__(f"{what}: {STATUS.get(self.code, self.code)}")


class Opts(ctypes.Structure):
    _fields_ = [
        ("M", ctypes.c_int32),
        ("fan_in", ctypes.c_int32),
        ("block", ctypes.c_int32),
        ("ctas_per_sm", ctypes.c_int32),
        ("warm_edges", ctypes.c_int64),
        ("profile", ctypes.c_int32),
        ("host_read", ctypes.c_int32),
        ("ap_warm_edges", ctypes.c_int32),
        ("warm_block", ctypes.c_int32),
        ("ap_fused", ctypes.c_int32),
        ("test_barrier_polls", ctypes.c_int32),
        ("test_hold_polls", ctypes.c_int32),
        ("test_fail_alloc", ctypes.c_int32),
    ]


class BatchPlan(ctypes.Structure):
    """bridges_batch_plan: the batched form's per-bucket plan (see include/bridges.h)."""

    _fields_ = [
        ("n", ctypes.c_int32),
        ("vmax", ctypes.c_int32 * 8),
        ("group", ctypes.c_int32 * 8),
        ("warm_per_v", ctypes.c_int32 * 8),
        ("warm_add", ctypes.c_int32 * 8),
        ("split", ctypes.c_int64 * 8),
    ]

    def buckets(self):
        """The plan as a list of per-bucket dicts."""
        return [{"vmax": self.vmax[b], "group": self.group[b], "split": self.split[b],
                 "warm_per_v": self.warm_per_v[b], "warm_add": self.warm_add[b]} for b in range(self.n)]

    @classmethod
    def from_buckets(cls, buckets):
        p = cls()
        p.n = len(buckets)
        for b, d in enumerate(buckets):
            p.vmax[b], p.group[b], p.split[b] = d["vmax"], d["group"], d["split"]
            p.warm_per_v[b], p.warm_add[b] = d["warm_per_v"], d["warm_add"]
        return p


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32

_SIGS = {
    "bridges_ctx_create": (_P, [ctypes.c_int, ctypes.c_size_t, ctypes.POINTER(Opts)]),
    "bridges_ctx_create_ws": (_P, [ctypes.c_int, _P, ctypes.c_size_t, ctypes.POINTER(Opts)]),
    "bridges_ctx_destroy": (None, [_P]),
    "bridges_workspace_bytes": (ctypes.c_size_t, [_P, _I64, _I32, _I32]),
    "bridges_find_ctx": (_I64, [_P, _P, _P, _P, _I64, _I32, _I32, _P, _P]),
    "bridges_find": (_I64, [_P, _P, _I64, _I32, _I32, _P]),
    "bridges_find_host": (_I64, [_P, _P, _P, _P, _I64, _I32, _I32, _P]),
    "bridges_certificate": (_I64, [_P, _P, _P, _P, _I64, _I32, _I32, _P, _P, _P]),
    "bridges_from_forest": (_I64, [_P, _P, _P, _P, _I64, _P, _P, _I64, _I32, _P]),
    "bridges_rooted_forest": (_I64, [_P, _P, _P, _P, _I64, _I32, _P, _P, _P]),
    "bridges_ctx_stage_ms": (_I32, [_P, ctypes.POINTER(ctypes.c_float), _I32]),
    "bridges_ctx_stage_ms_history": (_I32, [_P, ctypes.POINTER(ctypes.c_float), _I32]),
    "bridges_ctx_launches": (_I64, [_P]),
    "bridges_ctx_last_config": (_I32, [_P, ctypes.POINTER(ctypes.c_int64), _I32]),
    "bridges_status_string": (ctypes.c_char_p, [_I32]),
    "bridges_find_noalloc": (_I64, [_P, _P, _P, _I64, _I32, _I32, _P, _P]),
    "bridges_find_batched": (_I64, [_P, _P, _P, _P, _P, _P, _I32, _P, _P]),
    "bridges_ctx_set_batch_split": (_I32, [_P, _I64]),
    "bridges_ctx_set_batch_plan": (_I32, [_P, ctypes.POINTER(BatchPlan)]),
    "bridges_ctx_get_batch_plan": (_I32, [_P, ctypes.POINTER(BatchPlan)]),
    "bridges_batch_autotune": (_I32, [_P, _P, _P, _P, _P, _P, _I32, _I32, ctypes.POINTER(BatchPlan),
                                      ctypes.POINTER(ctypes.c_double)]),
    "bridges_server_create": (_P, [ctypes.c_int, ctypes.c_size_t, _I32, _I32, ctypes.POINTER(Opts)]),
    "bridges_server_submit": (_I32, [_P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "bridges_server_poll": (_I32, [_P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_double)]),
    "bridges_server_wait": (_I32, [_P, ctypes.c_uint64, _I64, ctypes.POINTER(ctypes.c_int64),
                                   ctypes.POINTER(ctypes.c_double)]),
    "bridges_server_stats": (_I32, [_P, ctypes.POINTER(ctypes.c_int64), _I32]),
    "bridges_server_cancel": (_I32, [_P, ctypes.c_uint64]),
    "bridges_server_destroy": (None, [_P]),
    "bridges_autotune": (_I32, [_P, _P, _P, _P, _I64, _I32, _I32, ctypes.POINTER(ctypes.c_int64)]),
    "bridges_ctx_set_opts": (_I32, [_P, ctypes.POINTER(Opts)]),
    "bridges_ctx_get_opts": (_I32, [_P, ctypes.POINTER(Opts)]),
    "bridges_wait_value": (_I32, [_P, _P, _P, _I32, _I64]),
    "bridges_two_edge_components": (_I64, [_P, _P, _P, _P, _I64, _I32, _I32, _P, _P]),
    "bridges_inc_create": (_P, [ctypes.c_int, ctypes.POINTER(Opts)]),
    "bridges_inc_destroy": (None, [_P]),
    "bridges_inc_reset": (_I64, [_P, _P, _P, _P, _I64, _I32, _I32, _P]),
    "bridges_inc_add": (_I64, [_P, _P, _P, _P, _I64, _P]),
    "bridges_inc_two_edge_components": (_I64, [_P, _P, _P]),
    "bridges_inc_certificate_size": (_I64, [_P]),
    "bridges_articulation_points": (_I64, [_P, _P, _P, _P, _I64, _I32, _I32, _P, _P, _P]),
    "bridges_articulation_points_host": (_I64, [_P, _P, _P, _P, _I64, _I32, _I32, _P]),
    "bridges_articulation_workspace_bytes": (_I64, [_P, _I64, _I32, _I32]),
    "bridges_ctx_ap_stage_ms": (_I32, [_P, ctypes.POINTER(ctypes.c_float), _I32]),
    "bridges_ctx_ap_stage_ms_history": (_I32, [_P, ctypes.POINTER(ctypes.c_float), _I32]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Loads libbridges.so (building it from source first if it is missing or stale)."""
    global _lib
    if _lib is None:
        if build_if_missing and _build.needs_build():
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError(f"libbridges.so not found at {_build.LIB}; run __graft_entry__.build()")
        lib = ctypes.CDLL(_build.LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dev_edges(u, v):
    if not (isinstance(u, torch.Tensor) and isinstance(v, torch.Tensor)):
        raise TypeError("edges must be torch tensors")
    if u.dtype != torch.int32 or v.dtype != torch.int32 or u.shape != v.shape or u.dim() != 1:
        raise ValueError("edges_u and edges_v must be 1-D int32 tensors of equal length")
    if not (u.is_cuda and v.is_cuda):
        raise ValueError("edges must be CUDA tensors (use Context.find_host for host input)")
    return u.contiguous(), v.contiguous()


def _check(rc, what):
    rc = int(rc)
    if rc < 0:
        raise BridgesError(rc, what)
    return rc


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Context:
    """A libbridges context on one device.

    ``workspace_bytes``: when given, the workspace is a torch allocation of that size and the
    library never allocates device memory itself (calls that need more raise ENOMEM); otherwise
    the library grows its own workspace up to ``mem_budget`` bytes (0: unlimited).
    """

    def __init__(self, device=None, M=0, fan_in=0, block=0, ctas_per_sm=0, warm_edges=-1, profile=False,
                 mem_budget=0, workspace_bytes=None, host_read=False, ap_warm_edges=0, warm_block=0, ap_fused=0):
        self._lib = load()
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.device = dev
        o = Opts()
        o.M, o.fan_in, o.block, o.ctas_per_sm = M, fan_in, block, ctas_per_sm
        o.warm_edges, o.profile, o.host_read = warm_edges, int(bool(profile)), int(bool(host_read))
        o.ap_warm_edges = int(ap_warm_edges)
        o.warm_block = int(warm_block)
        o.ap_fused = int(ap_fused)
        self._opts = o
        self._ws = None
        with torch.cuda.device(dev):
            if workspace_bytes is not None:
                self._ws = torch.empty(int(workspace_bytes), dtype=torch.uint8, device=dev)
                h = self._lib.bridges_ctx_create_ws(dev.index, _ptr(self._ws), int(workspace_bytes), ctypes.byref(o))
            else:
                h = self._lib.bridges_ctx_create(dev.index, int(mem_budget), ctypes.byref(o))
        if not h:
            raise BridgesError(-4, "bridges_ctx_create")
        self._h = ctypes.c_void_p(h)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bridges_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def workspace_bytes(self, E: int, V: int, M: int = 0) -> int:
        return int(self._lib.bridges_workspace_bytes(self._h, E, V, M))

    def find(self, u, v, V: int, M: int = 0, out=None, stream=None, count_device=None):
        """bridges_find_ctx on device tensors.  Returns an (n, 2) int32 view of ``out``; with
        ``count_device`` (a 1-element int64 CUDA tensor) the call is asynchronous and returns
        ``out`` whole."""
        u, v = _dev_edges(u, v)
        if out is None:
            out = torch.empty(2 * max(V - 1, 1), dtype=torch.int32, device=u.device)
        rc = self._lib.bridges_find_ctx(self._h, _stream(stream), _ptr(u), _ptr(v), u.numel(), V, M, _ptr(out),
                                        _ptr(count_device))
        n = _check(rc, "bridges_find_ctx")
        if count_device is not None:
            return out
        return out[: 2 * n].view(n, 2)

    def find_host(self, u, v, V: int, M: int = 0, out=None, stream=None):
        """bridges_find_host: host (ideally pinned) int32 tensors in, host bridges out."""
        for t in (u, v):
            if t.is_cuda or t.dtype != torch.int32 or t.dim() != 1:
                raise ValueError("find_host takes 1-D int32 host tensors")
        u, v = u.contiguous(), v.contiguous()
        if out is None:
            out = torch.empty(2 * max(V - 1, 1), dtype=torch.int32)
        rc = self._lib.bridges_find_host(self._h, _stream(stream), _ptr(u), _ptr(v), u.numel(), V, M, _ptr(out))
        n = _check(rc, "bridges_find_host")
        return out[: 2 * n].view(n, 2)

    def certificate(self, u, v, V: int, M: int = 0, stream=None):
        """bridges_certificate: (cert_u, cert_v, cert_tree) device tensors of the final certificate."""
        u, v = _dev_edges(u, v)
        cap = 2 * max(V - 1, 1)
        cu = torch.empty(cap, dtype=torch.int32, device=u.device)
        cv = torch.empty(cap, dtype=torch.int32, device=u.device)
        ct = torch.empty(cap, dtype=torch.uint8, device=u.device)
        rc = self._lib.bridges_certificate(self._h, _stream(stream), _ptr(u), _ptr(v), u.numel(), V, M, _ptr(cu),
                                           _ptr(cv), _ptr(ct))
        n = _check(rc, "bridges_certificate")
        return cu[:n], cv[:n], ct[:n].bool()

    def from_forest(self, tu, tv, xu, xv, V: int, stream=None):
        """bridges_from_forest: bridges of forest (tu, tv) plus extra edges (xu, xv)."""
        tu, tv = _dev_edges(tu, tv)
        xu, xv = _dev_edges(xu, xv)
        out = torch.empty(2 * max(V - 1, 1), dtype=torch.int32, device=tu.device)
        rc = self._lib.bridges_from_forest(self._h, _stream(stream), _ptr(tu), _ptr(tv), tu.numel(), _ptr(xu),
                                           _ptr(xv), xu.numel(), V, _ptr(out))
        n = _check(rc, "bridges_from_forest")
        return out[: 2 * n].view(n, 2)

    def rooted_forest(self, tu, tv, V: int, stream=None):
        """bridges_rooted_forest: (parent, pre, size) of forest (tu, tv), each tree rooted at its
        minimum vertex and numbered in preorder (int32 CUDA tensors of length V)."""
        tu, tv = _dev_edges(tu, tv)
        outs = [torch.empty(max(V, 1), dtype=torch.int32, device=tu.device) for _ in range(3)]
        rc = self._lib.bridges_rooted_forest(self._h, _stream(stream), _ptr(tu), _ptr(tv), tu.numel(), V,
                                             *[_ptr(o) for o in outs])
        _check(rc, "bridges_rooted_forest")
        return tuple(o[:V] for o in outs)

    def find_batched(self, u, v, edge_off, Vs, out=None, counts=None, stream=None, sync=True):
        """bridges_find_batched.  ``edge_off`` (G+1) and ``Vs`` (G) are host integer arrays.
        Returns (out, counts, out_off): graph g's bridges are
        out[out_off[g] : out_off[g] + 2*counts[g]] (counts on the device)."""
        import numpy as np

        u, v = _dev_edges(u, v)
        eo = np.ascontiguousarray(edge_off, dtype=np.int64)
        vs = np.ascontiguousarray(Vs, dtype=np.int32)
        G = int(vs.shape[0])
        if eo.shape != (G + 1,):
            raise ValueError("edge_off must have G+1 entries")
        sizes = 2 * np.maximum(vs.astype(np.int64) - 1, 0)
        out_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        if out is None:
            out = torch.empty(max(int(out_off[-1]), 1), dtype=torch.int32, device=u.device)
        if counts is None:
            counts = torch.empty(max(G, 1), dtype=torch.int64, device=u.device)
        rc = self._lib.bridges_find_batched(self._h, _stream(stream), _ptr(u), _ptr(v), eo.ctypes.data, vs.ctypes.data,
                                            G, _ptr(out), _ptr(counts))
        _check(rc, "bridges_find_batched")
        if sync:
            (stream or torch.cuda.current_stream()).synchronize()
        return out, counts, out_off[:-1]

    def autotune(self, u, v, V: int, reps: int = 3, stream=None):
        """bridges_autotune on device tensors; returns the chosen plan (also kept in the context)."""
        u, v = _dev_edges(u, v)
        best = (ctypes.c_int64 * 5)()
        _check(self._lib.bridges_autotune(self._h, _stream(stream), _ptr(u), _ptr(v), u.numel(), V, reps, best),
               "bridges_autotune")
        names = ["M", "fan_in", "warm_edges", "block", "us_per_call"]
        plan = {names[i]: int(best[i]) for i in range(5)}
        plan["warm_block"] = self.get_opts()["warm_block"]
        return plan

    def get_opts(self):
        """bridges_ctx_get_opts: the context's current options as a dict."""
        o = Opts()
        _check(self._lib.bridges_ctx_get_opts(self._h, ctypes.byref(o)), "bridges_ctx_get_opts")
        return {name: getattr(o, name) for name, _ in Opts._fields_}

    def set_opts(self, M=0, fan_in=0, block=0, ctas_per_sm=0, warm_edges=-1, host_read=False, warm_block=0,
                 ap_warm_edges=0, ap_fused=0, test_barrier_polls=0, test_hold_polls=0, test_fail_alloc=0):
        o = Opts()
        o.M, o.fan_in, o.block, o.ctas_per_sm, o.warm_edges = M, fan_in, block, ctas_per_sm, warm_edges
        o.host_read = int(bool(host_read))
        o.warm_block, o.ap_warm_edges = int(warm_block), int(ap_warm_edges)
        o.ap_fused = int(ap_fused)
        o.test_barrier_polls, o.test_hold_polls = int(test_barrier_polls), int(test_hold_polls)
        o.test_fail_alloc = int(test_fail_alloc)
        _check(self._lib.bridges_ctx_set_opts(self._h, ctypes.byref(o)), "bridges_ctx_set_opts")

    def wait_value(self, flag, value: int, max_polls: int, stream=None) -> int:
        """bridges_wait_value on a 1-element int32 CUDA tensor; returns the status code."""
        if not (flag.is_cuda and flag.dtype == torch.int32):
            raise ValueError("flag must be an int32 CUDA tensor")
        return int(self._lib.bridges_wait_value(self._h, _stream(stream), _ptr(flag), int(value), int(max_polls)))

    def two_edge_components(self, u, v, V: int, M: int = 0, stream=None):
        """bridges_two_edge_components: (count, labels (V,) int32 device tensor, bridges (n, 2))."""
        u, v = _dev_edges(u, v)
        labels = torch.empty(max(V, 1), dtype=torch.int32, device=u.device)
        out = torch.empty(2 * max(V - 1, 1), dtype=torch.int32, device=u.device)
        n = _check(self._lib.bridges_two_edge_components(self._h, _stream(stream), _ptr(u), _ptr(v), u.numel(), V, M,
                                                         _ptr(labels), _ptr(out)), "bridges_two_edge_components")
        return n, labels[:V]

    def articulation_points(self, u, v, V: int, M: int = 0, stream=None, with_bridges: bool = False,
                            counts_device=None, out=None):
        """bridges_articulation_points: the cut vertices (sorted int32 device tensor); with
        with_bridges also the bridges as an (n, 2) tensor.  With counts_device (an int64 device
        tensor of 2 elements) the call only enqueues work and returns the full-capacity output
        buffers (counts appear in counts_device)."""
        u, v = _dev_edges(u, v)
        pts = out if out is not None else torch.empty(max(V, 1), dtype=torch.int32, device=u.device)
        br = torch.empty(2 * max(V - 1, 1), dtype=torch.int32, device=u.device) if with_bridges else None
        if counts_device is not None:
            _check(self._lib.bridges_articulation_points(self._h, _stream(stream), _ptr(u), _ptr(v), u.numel(), V, M,
                                                         _ptr(pts), _ptr(br), _ptr(counts_device)),
                   "bridges_articulation_points")
            return (pts, br) if with_bridges else pts
        cnt = torch.zeros(2, dtype=torch.int64, device=u.device) if with_bridges else None
        n = _check(self._lib.bridges_articulation_points(self._h, _stream(stream), _ptr(u), _ptr(v), u.numel(), V, M,
                                                         _ptr(pts), _ptr(br), _ptr(cnt)),
                   "bridges_articulation_points")
        if not with_bridges:
            return pts[:n]
        (stream or torch.cuda.current_stream(u.device)).synchronize()
        na, nb = (int(x) for x in cnt.cpu())
        _check(na, "bridges_articulation_points")
        _check(nb, "bridges_articulation_points")
        return pts[:na], br[: 2 * nb].view(nb, 2)

    def articulation_points_host(self, u, v, V: int, M: int = 0, stream=None, out=None):
        """bridges_articulation_points_host: host int32 edge tensors (pinned for full speed) in,
        a host int32 tensor of the cut vertices out."""
        for t in (u, v):
            if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.int32 or t.dim() != 1:
                raise ValueError("edges must be 1-D int32 host tensors")
        if u.shape != v.shape:
            raise ValueError("edges_u and edges_v must have equal length")
        u, v = u.contiguous(), v.contiguous()
        pts = out if out is not None else torch.empty(max(V, 1), dtype=torch.int32)
        n = _check(self._lib.bridges_articulation_points_host(self._h, _stream(stream), _ptr(u), _ptr(v), u.numel(),
                                                              V, M, _ptr(pts)), "bridges_articulation_points_host")
        return pts[:n]

    def articulation_workspace_bytes(self, E: int, V: int, M: int = 0) -> int:
        return int(self._lib.bridges_articulation_workspace_bytes(self._h, E, V, M))

    def ap_stage_ms(self):
        """Stage times (ms) of the last profiled articulation-point call's block pass."""
        buf = (ctypes.c_float * 5)()
        k = self._lib.bridges_ctx_ap_stage_ms(self._h, buf, 5)
        names = ["warmup", "snapshot", "stream", "mark", "total"]
        return {names[i]: float(buf[i]) for i in range(max(k, 0))}

    def ap_stage_ms_history(self, max_calls: int = 32):
        """Block-pass stage times of the last min(max_calls, 32) profiled calls, oldest first."""
        buf = (ctypes.c_float * (5 * max_calls))()
        k = self._lib.bridges_ctx_ap_stage_ms_history(self._h, buf, max_calls)
        names = ["warmup", "snapshot", "stream", "mark", "total"]
        return [{names[j]: float(buf[5 * i + j]) for j in range(5)} for i in range(k)]

    def batch_autotune(self, u, v, edge_off, Vs, reps: int = 3, stream=None):
        """bridges_batch_autotune on a batch (arguments as for find_batched); keeps the tuned plan
        in the context and returns (per-bucket plan list, microseconds per batch)."""
        import numpy as np

        u, v = _dev_edges(u, v)
        eo = np.ascontiguousarray(edge_off, dtype=np.int64)
        vs = np.ascontiguousarray(Vs, dtype=np.int32)
        G = int(vs.shape[0])
        if eo.shape != (G + 1,):
            raise ValueError("edge_off must have G+1 entries")
        plan, us = BatchPlan(), ctypes.c_double(0)
        _check(self._lib.bridges_batch_autotune(self._h, _stream(stream), _ptr(u), _ptr(v), eo.ctypes.data,
                                                vs.ctypes.data, G, int(reps), ctypes.byref(plan), ctypes.byref(us)),
               "bridges_batch_autotune")
        return plan.buckets(), float(us.value)

    def set_batch_plan(self, buckets):
        """bridges_ctx_set_batch_plan from a per-bucket list (empty: the automatic plan)."""
        _check(self._lib.bridges_ctx_set_batch_plan(self._h, ctypes.byref(BatchPlan.from_buckets(buckets))),
               "bridges_ctx_set_batch_plan")

    def get_batch_plan(self):
        plan = BatchPlan()
        _check(self._lib.bridges_ctx_get_batch_plan(self._h, ctypes.byref(plan)), "bridges_ctx_get_batch_plan")
        return plan.buckets()

    def set_batch_split(self, split_edges: int):
        _check(self._lib.bridges_ctx_set_batch_split(self._h, int(split_edges)), "bridges_ctx_set_batch_split")

    def stage_ms(self):
        buf = (ctypes.c_float * 6)()
        k = self._lib.bridges_ctx_stage_ms(self._h, buf, 6)
        names = ["warmup", "snapshot", "forest", "merge", "final", "total"]
        return {names[i]: float(buf[i]) for i in range(k)}

    def stage_ms_history(self, max_calls: int = 32):
        """Stage times of the last min(max_calls, 32) profiled calls, oldest first."""
        buf = (ctypes.c_float * (6 * max_calls))()
        k = self._lib.bridges_ctx_stage_ms_history(self._h, buf, max_calls)
        names = ["warmup", "snapshot", "forest", "merge", "final", "total"]
        return [{names[j]: float(buf[6 * i + j]) for j in range(6)} for i in range(k)]

    def launches(self) -> int:
        return int(self._lib.bridges_ctx_launches(self._h))

    def last_config(self):
        buf = (ctypes.c_int64 * 8)()
        k = self._lib.bridges_ctx_last_config(self._h, buf, 8)
        names = ["M", "fan_in", "blocks_per_partition", "block", "warm_edges", "ap_warm_edges", "ap_blocks", "ap_fused"]
        return {names[i]: int(buf[i]) for i in range(k)}


class Request(ctypes.Structure):
    _fields_ = [
        ("edges_u", ctypes.c_void_p),
        ("edges_v", ctypes.c_void_p),
        ("E", ctypes.c_int64),
        ("V", ctypes.c_int32),
        ("M", ctypes.c_int32),
        ("out_bridges", ctypes.c_void_p),
    ]


class Server:
    """bridges_server: continuous batching of bridge queries on one GPU (thread-safe).

    ``submit`` keeps references to the request's tensors until its result has been collected."""

    def __init__(self, device=None, mem_budget=0, max_slots=8, max_batch=4096, **opts):
        self._lib = load()
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.device = dev
        o = Opts()
        o.warm_edges = opts.get("warm_edges", -1)
        o.M = opts.get("M", 0)
        o.test_barrier_polls = int(opts.get("test_barrier_polls", 0))
        o.test_hold_polls = int(opts.get("test_hold_polls", 0))
        h = self._lib.bridges_server_create(dev.index, int(mem_budget), max_slots, max_batch, ctypes.byref(o))
        if not h:
            raise BridgesError(-4, "bridges_server_create")
        self._h = ctypes.c_void_p(h)
        self._live = {}

    def submit(self, u, v, V: int, out=None, M: int = 0) -> int:
        u, v = _dev_edges(u, v)
        if out is None:
            out = torch.empty(2 * max(V - 1, 1), dtype=torch.int32, device=u.device)
        r = Request(u.data_ptr(), v.data_ptr(), u.numel(), V, M, out.data_ptr())
        t = ctypes.c_uint64(0)
        _check(self._lib.bridges_server_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "bridges_server_submit")
        self._live[t.value] = (u, v, out)
        return t.value

    def _result(self, ticket, rc, cnt, lat):
        if rc == -7:
            return None
        _check(rc, "bridges_server")
        u, v, out = self._live.pop(ticket)
        n = int(cnt.value)
        if n < 0:
            raise BridgesError(n, "request")
        return out[: 2 * n].view(n, 2), float(lat.value)

    def poll(self, ticket: int):
        """None while pending, else (bridges (n, 2) device view, latency ms)."""
        cnt, lat = ctypes.c_int64(0), ctypes.c_double(0)
        rc = self._lib.bridges_server_poll(self._h, ticket, ctypes.byref(cnt), ctypes.byref(lat))
        return self._result(ticket, rc, cnt, lat)

    def wait(self, ticket: int, timeout_ms: int = 60000):
        cnt, lat = ctypes.c_int64(0), ctypes.c_double(0)
        rc = self._lib.bridges_server_wait(self._h, ticket, timeout_ms, ctypes.byref(cnt), ctypes.byref(lat))
        return self._result(ticket, rc, cnt, lat)

    def cancel(self, ticket: int) -> bool:
        """bridges_server_cancel: True if the queued request was withdrawn (its wait / poll then
        raises BRIDGES_ECANCELED), False if it was already running or done."""
        rc = int(self._lib.bridges_server_cancel(self._h, ticket))
        if rc == -7:
            return False
        _check(rc, "bridges_server_cancel")
        return True

    def stats(self):
        buf = (ctypes.c_int64 * 6)()
        k = self._lib.bridges_server_stats(self._h, buf, 6)
        names = ["completed", "batches", "singles", "max_in_flight", "failures", "queued"]
        return {names[i]: int(buf[i]) for i in range(k)}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bridges_server_destroy(self._h)
            self._h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Incremental:
    """bridges_inc: a resident certificate answering "add these edges" queries."""

    def __init__(self, device=None, **opts):
        self._lib = load()
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.device = dev
        o = Opts()
        o.warm_edges = opts.get("warm_edges", -1)
        o.M = opts.get("M", 0)
        h = self._lib.bridges_inc_create(dev.index, ctypes.byref(o))
        if not h:
            raise BridgesError(-4, "bridges_inc_create")
        self._h = ctypes.c_void_p(h)
        self.V = 0

    def reset(self, u, v, V: int, M: int = 0, stream=None):
        u, v = _dev_edges(u, v)
        out = torch.empty(2 * max(V - 1, 1), dtype=torch.int32, device=u.device)
        n = _check(self._lib.bridges_inc_reset(self._h, _stream(stream), _ptr(u), _ptr(v), u.numel(), V, M, _ptr(out)),
                   "bridges_inc_reset")
        self.V = V
        return out[: 2 * n].view(n, 2)

    def add(self, u, v, stream=None):
        u, v = _dev_edges(u, v)
        out = torch.empty(2 * max(self.V - 1, 1), dtype=torch.int32, device=u.device)
        n = _check(self._lib.bridges_inc_add(self._h, _stream(stream), _ptr(u), _ptr(v), u.numel(), _ptr(out)),
                   "bridges_inc_add")
        return out[: 2 * n].view(n, 2)

    def two_edge_components(self, stream=None):
        labels = torch.empty(max(self.V, 1), dtype=torch.int32, device=self.device)
        n = _check(self._lib.bridges_inc_two_edge_components(self._h, _stream(stream), _ptr(labels)),
                   "bridges_inc_two_edge_components")
        return n, labels[: self.V]

    def certificate_size(self) -> int:
        return _check(self._lib.bridges_inc_certificate_size(self._h), "bridges_inc_certificate_size")

    def close(self):
        if getattr(self, "_h", None):
            self._lib.bridges_inc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bridges_find(u, v, V: int, M: int = 0, out=None):
    """bridges_find: plain synchronous call on device tensors (default context, legacy stream)."""
    lib = load()
    u, v = _dev_edges(u, v)
    if out is None:
        out = torch.empty(2 * max(V - 1, 1), dtype=torch.int32, device=u.device)
    with torch.cuda.device(u.device):
        torch.cuda.current_stream().synchronize()
        rc = lib.bridges_find(_ptr(u), _ptr(v), u.numel(), V, M, _ptr(out))
    n = _check(rc, "bridges_find")
    return out[: 2 * n].view(n, 2)


def bridges_find_noalloc(u, v, V: int, M: int = 0, out=None, stream=None):
    """bridges_find_noalloc: the same result as bridges_find, for callers that must not allocate
    device memory (the library keeps all scratch in a fixed 8 MiB device array; graphs that need
    more raise BridgesError ENOMEM).  Calls that may overlap on the GPU must be serialised."""
    lib = load()
    u, v = _dev_edges(u, v)
    if out is None:
        out = torch.empty(2 * max(V - 1, 1), dtype=torch.int32, device=u.device)
    with torch.cuda.device(u.device):
        rc = lib.bridges_find_noalloc(_stream(stream), _ptr(u), _ptr(v), u.numel(), V, M, _ptr(out), None)
    n = _check(rc, "bridges_find_noalloc")
    return out[: 2 * n].view(n, 2)


def status_string(code: int) -> str:
    return load().bridges_status_string(int(code)).decode()
