"""Benchmark: input edges/s to the exact bridge set on one GB300 (and N replicas under torchrun).

A step is one pass of the whole path -- partition forest pass, label snapshot, merge tree,
Euler tour / range test / sort -- over the large dense workload: an ER(65,536, 0.5) core with
256 pendant trees and 128 two-edge vertices (about 1.07 G edges, 8.6 GB of int32 COO; seed 2).
The inputs (8.6 GB) are larger than L2 (129 MB), so no flush is needed between steps.

Prints one JSON line (rank 0).  On one GPU the default run adds two sub-objects measured after
the large workload: ``batched`` (4,096 graphs per persistent launch) and ``served`` (100,000
Poisson requests at 2,000/s, each a fresh graph generated on the device, against the
continuous-batching server), each with its oracle comparison and plain per-graph calls beside it.
``--impl reference`` times the CPU oracle (the paper's pipeline, single-threaded C) on a bounded
sample of the large workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
import types

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import warnings  # noqa: E402

# the generator's arrays are read-only views of C memory; torch only reads them here
warnings.filterwarnings("ignore", message="The given NumPy array is not writable")

import graphgen  # noqa: E402

METRIC = "input edges/s to exact bridge set"
UNIT = "GE/s"

# DRAM bytes (read + write) per streamed edge, from the ncu captures of the large workload's
# streaming kernels; each is valid only for the kernel sources it was measured on (hash of those
# sources).
#   forest pass, M = 1, at density 1/8 (268 M edges, 2.1 GB: a capture of a few GB, scaled to a
#   full launch by its streamed edges): 2.1402 GB read + 5.5 MB written for 267,444,294 streamed
#   edges; block pass stream and fused stream (articulation points), the same density:
#   2.1471 GB read + 7.6 MB written, and 2.1402 GB read + 0.4 MB written, for 267,444,294
#   streamed edges each
TRAFFIC = {"certify_sha": "245b7bcea88905d1", "bytes_per_edge": 8.0245,
           "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the forest pass at density 1/8 "
                     "(268 M edges), scaled to a full launch by its streamed edges"}
AP_TRAFFIC = {"blocks_sha": "461b023b22eb6faa", "bytes_per_edge": 8.0566,
              "source": "ncu dram bytes of the block pass stream at density 1/8, scaled by streamed edges"}
FUSED_TRAFFIC = {"blocks_sha": "461b023b22eb6faa", "bytes_per_edge": 8.0040,
                 "source": "ncu dram bytes of the fused stream at density 1/8, scaled by streamed edges"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def code_only(text):
    """C++ source without its comments and blank lines: what the compiler sees of it."""
    out, i, n = [], 0, len(text)
    while i < n:
        if text.startswith("//", i):
            i = text.find("\n", i)
            i = n if i < 0 else i
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
        elif text[i] in "\"'":  # a string or character literal: copied as is
            q, j = text[i], i + 1
            while j < n and text[j] != q:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        else:
            out.append(text[i])
            i += 1
    return "\n".join(line.rstrip() for line in "".join(out).splitlines() if line.strip())


def sources_sha(names):
    """Hash of the code (comments left out) of the named sources."""
    h = hashlib.sha256()
    for name in names:
        h.update(code_only(open(os.path.join(ROOT, "paper_2108_07346_gb300", "csrc", name)).read()).encode())
    return h.hexdigest()[:16]


def certify_sha():
    """Hash of the forest pass's sources (the traffic figure is only valid for them)."""
    return sources_sha(("certify.cu", "common.cuh", "forest.cuh", "stream.cuh"))


def blocks_sha():
    """Hash of the block pass's sources."""
    return sources_sha(("blocks.cu", "common.cuh", "forest.cuh", "stream.cuh"))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.5)  # let the sampler come up before the timed region

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = [[x.strip() for x in ln.split(",")] for ln in open(self.f.name).read().strip().splitlines()
                if ln.strip()]
        os.unlink(self.f.name)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        t0, t1 = getattr(self, "t0", None), getattr(self, "t1", None)
        samples = []
        for r in rows:
            if len(r) < 9:
                continue
            try:
                ts = time.mktime(time.strptime(r[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                sm, mx = float(r[1]), float(r[2])
            except ValueError:
                continue
            samples.append((ts, sm, mx, [names[i] for i in range(4) if r[5 + i] == "Active"]))
        if not samples:
            return None
        inside = [x for x in samples if t0 is None or (t0 - 1.0 <= x[0] <= t1 + 1.0)] or samples
        return {"sm_mhz": statistics.median(x[1] for x in inside), "sm_max_mhz": max(x[2] for x in inside),
                "reasons": sorted({n for x in inside for n in x[3]}), "samples": len(inside),
                "window_s": None if t0 is None else round(t1 - t0, 3)}


def reduce_max(value, device=None):
    """Max of a float over the ranks of the default process group (the value itself if none)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed per second (x1e-9): every rank does the same work (replicas)."""
    return world * units_per_rank / seconds / 1e9


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_workload(args):
    over = {}
    if args.density is not None:
        over["p"] = args.density
    return graphgen.workload(args.workload, **over)


def cpu_oracle_rate(g, M, sample_edges):
    """The oracle (Sec. 3 pipeline + Alg. 1, single-threaded C) on the first `sample_edges` edges."""
    import oracle

    n = min(sample_edges, g.E)
    u = np.ascontiguousarray(g.u[:n])
    v = np.ascontiguousarray(g.v[:n])
    t = time.perf_counter()
    oracle.bridges(u, v, g.V, M)
    dt = time.perf_counter() - t
    return n / dt / 1e9, n, dt


def cpu_model():
    """The host CPU's model line (x86 "model name", or an Arm core's implementer and part)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return "unknown"
    for key in ("model name", "Model"):
        for line in info:
            if line.startswith(key):
                return line.split(":", 1)[1].strip()
    parts = {line.split(":")[0].strip(): line.split(":", 1)[1].strip() for line in info if ":" in line}
    return f"Arm implementer {parts.get('CPU implementer', '?')} part {parts.get('CPU part', '?')}"


def cpu_oracle_parallel_rate(g, cores):
    """The paper's scheme on the host's cores: Alg. 2 on one contiguous partition per core (the
    oracle's C certificate, one thread each: the calls release the GIL), one merge (Alg. 2 on
    the union of the partition certificates), then Alg. 1 on the merged certificate."""
    import concurrent.futures

    import oracle

    E = g.E
    cuts = [E * i // cores for i in range(cores + 1)]

    def leaf(i):
        lo, hi = cuts[i], cuts[i + 1]
        ids, _ = oracle.certificate(g.u[lo:hi], g.v[lo:hi], g.V)
        return ids + lo

    t = time.perf_counter()
    with concurrent.futures.ThreadPoolExecutor(cores) as ex:
        ids = np.concatenate(list(ex.map(leaf, range(cores))))
    u1, v1 = g.u[ids], g.v[ids]
    keep, _ = oracle.certificate(u1, v1, g.V)
    br = oracle.dfs_bridges(u1[keep], v1[keep], g.V)
    dt = time.perf_counter() - t
    return E / dt / 1e9, dt, br


def ref_sample_per_step(args, budget_edges):
    """Edges the reference arm times per step: the requested sample, shrunk so that all steps
    together stay near `budget_edges` (about two minutes of the single-threaded oracle)."""
    return max(1_000_000, min(args.ref_sample, budget_edges // max(1, args.steps)))


def workload_name(workload, g):
    """The workload as both arms name it in `config`."""
    if workload in ("large", "articulation"):
        name = (f"large: ER(65536, p={g.spec.p}) core + 256 pendant trees + 128 two-edge vertices, "
                f"seed {g.spec.seed}")
        return name if workload == "large" else "articulation points of " + name
    return workload


def run_reference(args, world, rank):
    if rank != 0:
        return
    if args.workload == "articulation":
        return run_reference_ap(args, world)
    g = make_workload(args)
    M = args.M if args.M > 0 else 5
    per_step = ref_sample_per_step(args, 18_000_000_000)  # 0.15 GE/s: ~2 minutes
    for _ in range(args.warmup):
        cpu_oracle_rate(g, M, max(per_step // 10, 1))
    times = []
    for _ in range(args.steps):
        _, n, dt = cpu_oracle_rate(g, M, per_step)
        times.append(dt)
    tot = sum(times)
    value = n * args.steps / tot / 1e9
    sample = (f"oracle (Sec. 3 pipeline, M={M}, then Alg. 1; single-threaded C) on the first {n} edges of the "
              f"{args.workload} workload per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": workload_name(args.workload, g), "V": g.V, "E": g.E, "sample_edges_per_step": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_ap(args, world):
    g = graphgen.workload("large", **({} if args.density is None else {"p": args.density}))
    per_step = ref_sample_per_step(args, 3_600_000_000)  # 0.03 GE/s: ~2 minutes
    for _ in range(args.warmup):
        cpu_oracle_ap_rate(g, max(per_step // 10, 1))
    times = []
    n = 0
    for _ in range(args.steps):
        _, n, dt = cpu_oracle_ap_rate(g, per_step)
        times.append(dt)
    tot = sum(times)
    value = n * args.steps / tot / 1e9
    sample = (f"oracle Tarjan low/disc articulation points (single-threaded C) on the first {n} edges of the large "
              f"workload per step")
    print(json.dumps({
        "impl": "reference", "metric": AP_METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": workload_name("articulation", g), "V": g.V, "E": g.E, "sample_edges_per_step": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_sharded(args, world, rank, local):
    """N ranks on one graph (strong scaling): rank r holds the contiguous shard r of the list, the
    ranks merge certificates on the paper's schedule (Sec. 3 phases) and rank 0 finds the bridges
    and broadcasts them.  Certificates travel through NCCL on device buffers (NVLS off), or with
    --exchange gloo through host buffers (which also lets several ranks share one GPU for a test
    with --same-device).  A step is one whole sharded call."""
    import torch
    import torch.distributed as dist

    import paper_2108_07346_gb300 as pb
    from paper_2108_07346_gb300.sharded import Certifier, shard_range, sharded_bridges

    os.environ.setdefault("NCCL_NVLS_ENABLE", "0")
    dev = torch.device("cuda", 0 if args.same_device else local)
    torch.cuda.set_device(dev)
    if args.exchange == "gloo":
        dist.init_process_group("gloo")
    else:
        dist.init_process_group("nccl", device_id=dev)
    spec = graphgen.Spec(**{**graphgen.asdict(graphgen.WORKLOADS[args.workload]),
                            **({} if args.density is None else {"p": args.density})})
    g = graphgen.generate_device(spec, dev)
    E, V, planted = g.E, g.V, g.planted
    lo, hi = shard_range(E, rank, world)
    u, v = g.u[lo:hi].clone(), g.v[lo:hi].clone()
    del g
    torch.cuda.empty_cache()
    ctx = pb.Context(device=dev)
    cert = Certifier(ctx)
    res = sharded_bridges(u, v, V, cert).cpu().numpy()
    correct = bool(np.array_equal(res, planted))
    for _ in range(args.warmup):
        sharded_bridges(u, v, V, cert)
    stream = torch.cuda.current_stream(dev)
    dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(dev.index)
    clocks.start()
    clocks.mark("t0")
    l0 = ctx.launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        br = sharded_bridges(u, v, V, cert)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clocks.mark("t1")
    launches = ctx.launches() - l0
    ms_total = reduce_max(e0.elapsed_time(e1), dev if args.exchange == "nccl" else None)
    ck = clocks.stop()
    timed_correct = bool(np.array_equal(br.cpu().numpy(), planted))
    # end to end: each rank's shard from pinned host memory, copied in inside the timed region
    hu, hv = u.cpu().pin_memory(), v.cpu().pin_memory()
    ks = max(1, min(args.steps, args.e2e_steps))
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nb = 0
    for _ in range(ks):
        du, dv = hu.to(dev, non_blocking=True), hv.to(dev, non_blocking=True)
        nb = int(sharded_bridges(du, dv, V, cert).cpu().shape[0])
    torch.cuda.synchronize()
    dt = reduce_max(time.perf_counter() - t0, dev if args.exchange == "nccl" else None)
    if rank == 0:
        line = {
            "metric": METRIC, "value": E * args.steps / (ms_total * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": workload_name(args.workload, types.SimpleNamespace(spec=spec)),
                       "V": V, "E": E, "parallelism": f"sharded x{world}: contiguous shards, certificates merged on "
                                                     f"the paper's log2 N schedule, rank 0 final stage",
                       "exchange": args.exchange, "same_device": bool(args.same_device),
                       "bridges": int(br.shape[0]), "bridges_equal_planted": correct,
                       "timed_output_equal_planted": timed_correct,
                       "l2": "inputs (8E bytes) larger than L2; no flush"},
            "clocks": ck, "gpu_launches": launches,
            "e2e": {"value": E * ks / dt / 1e9, "unit": UNIT, "h2d_bytes_per_step": 8 * E,
                    "d2h_bytes_per_step": 16 + 8 * nb, "steps": ks, "ms_per_step": dt / ks * 1e3},
            "roofline": None, "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)
    dist.destroy_process_group()


def run_native(args, world, rank, local):
    import torch

    import paper_2108_07346_gb300 as pb

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    g = make_workload(args)
    E, V = g.E, g.V
    du = torch.from_numpy(g.u).to(dev)
    dv = torch.from_numpy(g.v).to(dev)
    out = torch.empty(2 * max(V - 1, 1), dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    ctx = pb.Context(device=dev, profile=True, M=args.M)
    stream = torch.cuda.current_stream(dev)
    plan = None
    if args.M <= 0 and not args.no_tune:
        plan = ctx.autotune(du, dv, V, reps=3)  # outside the timed region; kept in the context
    # the merge-tree cost at fixed M (a few steps each, outside the timed region)
    sweep = {}
    if not args.no_sweep:
        for m in (1, 2, 4, 8, 16):
            sctx = pb.Context(device=dev, profile=True, M=m)
            for _ in range(3):
                sctx.find(du, dv, V, m, out=out, count_device=cnt, stream=stream)
            for _ in range(10):
                sctx.find(du, dv, V, m, out=out, count_device=cnt, stream=stream)
            hh = sctx.stage_ms_history(10)
            sweep[str(m)] = {k: round(statistics.median(x[k] for x in hh), 4) for k in hh[0]}
            sweep[str(m)]["GE_per_s"] = round(E / sweep[str(m)]["total"] / 1e6, 1)
            del sctx

    # correctness of what is timed: the planted bridges are exact on this workload
    res = ctx.find(du, dv, V, args.M).cpu().numpy()
    correct = bool(res.shape[0] == len(g.planted) and np.array_equal(res, g.planted))
    for _ in range(args.warmup):
        ctx.find(du, dv, V, args.M, out=out, count_device=cnt, stream=stream)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    clocks.mark("t0")
    l0 = ctx.launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.find(du, dv, V, args.M, out=out, count_device=cnt, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark("t1")
    launches = ctx.launches() - l0
    ms_total = e0.elapsed_time(e1)
    hist = ctx.stage_ms_history(args.steps)
    ck = clocks.stop()
    ms_total = reduce_max(ms_total, dev)
    n_found = int(cnt.item())
    # the last timed call's own output, read back after the timed region
    timed_out = out[: 2 * max(n_found, 0)].view(-1, 2).cpu().numpy()
    timed_correct = bool(n_found == len(g.planted) and np.array_equal(timed_out, g.planted))
    ms_step = ms_total / args.steps
    value = whole_job_rate(E * args.steps, world, ms_total * 1e-3)

    cfg = ctx.last_config()
    forest_ms = statistics.mean(h["forest"] for h in hist) if hist else None
    forest_edges = E - cfg["M"] * max(cfg["warm_edges"], 0) if cfg["warm_edges"] > 0 else None
    peak, peak_kind = peaks()
    roof = None
    if forest_ms and forest_edges:
        achieved = 8.0 * forest_edges / (forest_ms * 1e-3) / 1e9
        traffic = None
        if TRAFFIC["certify_sha"] == certify_sha() and TRAFFIC["bytes_per_edge"]:
            traffic = TRAFFIC["bytes_per_edge"] * forest_edges
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "traffic_source": TRAFFIC["source"] if traffic else None,
                "kernel": "leaf_kernel<cache, vec> (partition forest pass)",
                "algorithmic_bytes": 8 * forest_edges, "peak_kind": peak_kind,
                "frac_of_nominal_7900": achieved / 7900.0,
                "stage_ms_mean": {k: statistics.mean(h[k] for h in hist) for k in hist[0]}}

    # throughput with two calls in flight: two contexts (two workspaces) on two streams take the
    # calls in turn, so one call's latency-bound stages (warm-up, final stage) overlap the other
    # call's forest pass; every call is a whole call (reported beside the headline, not as it)
    pipelined = None
    if world == 1 and not args.no_pipelined:
        pctx = [pb.Context(device=dev, M=args.M) for _ in range(2)]
        if plan is not None:
            for c in pctx:
                c.set_opts(M=plan["M"], fan_in=plan["fan_in"], block=plan["block"], warm_edges=plan["warm_edges"],
                           warm_block=plan.get("warm_block", 0))
        pst = [torch.cuda.Stream(dev) for _ in range(2)]
        pout = [torch.empty_like(out) for _ in range(2)]
        pcnt = [torch.zeros(1, dtype=torch.int64, device=dev) for _ in range(2)]
        for k in range(2 * args.warmup):
            pctx[k % 2].find(du, dv, V, args.M, out=pout[k % 2], count_device=pcnt[k % 2], stream=pst[k % 2])
        torch.cuda.synchronize()
        q0 = torch.cuda.Event(enable_timing=True)
        q1 = torch.cuda.Event(enable_timing=True)
        qb = torch.cuda.Event()
        q0.record(pst[0])
        pst[1].wait_event(q0)
        for k in range(args.steps):
            pctx[k % 2].find(du, dv, V, args.M, out=pout[k % 2], count_device=pcnt[k % 2], stream=pst[k % 2])
        qb.record(pst[1])
        pst[0].wait_event(qb)
        q1.record(pst[0])
        torch.cuda.synchronize()
        pms = q0.elapsed_time(q1)
        pok = all(int(pcnt[k].item()) == len(g.planted) and
                  np.array_equal(pout[k][: 2 * len(g.planted)].view(-1, 2).cpu().numpy(), g.planted) for k in range(2))
        pipelined = {"value": E * args.steps / (pms * 1e-3) / 1e9, "unit": UNIT, "ms_per_call": pms / args.steps,
                     "calls": args.steps, "contexts": 2, "outputs_equal_planted": pok,
                     "note": "two contexts on two streams take the calls in turn: a call's warm-up and final "
                             "stage overlap the other call's forest pass; every call is whole"}
        del pctx, pout

    # end to end through the public API from pinned host buffers (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        hu = torch.from_numpy(g.u).pin_memory()
        hv = torch.from_numpy(g.v).pin_memory()
        hout = torch.empty(2 * max(V - 1, 1), dtype=torch.int32).pin_memory()
        ctx_h = pb.Context(device=dev, M=args.M)
        ctx_h.find_host(hu, hv, V, args.M, out=hout)
        ks = max(1, min(args.steps, args.e2e_steps))
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hres = None
        for _ in range(ks):
            hres = ctx_h.find_host(hu, hv, V, args.M, out=hout)
        torch.cuda.synchronize()
        dt = reduce_max(time.perf_counter() - t0, dev)
        nb = int(hres.shape[0])
        e2e = {"value": whole_job_rate(E * ks, world, dt), "unit": UNIT, "h2d_bytes_per_step": 8 * E,
               "d2h_bytes_per_step": 8 + 8 * nb, "steps": ks, "ms_per_step": dt / ks * 1e3,
               "timed_output_equal_planted": bool(np.array_equal(hres.numpy(), g.planted))}
        del ctx_h
        # the same call with the kernels reading the pinned host buffers in place (opts.host_read):
        # no device copy of the edges at all
        ctx_r = pb.Context(device=dev, M=args.M, host_read=True)
        ctx_r.find_host(hu, hv, V, args.M, out=hout)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rres = None
        for _ in range(ks):
            rres = ctx_r.find_host(hu, hv, V, args.M, out=hout)
        torch.cuda.synchronize()
        dtr = reduce_max(time.perf_counter() - t0, dev)
        e2e["in_place"] = {"value": whole_job_rate(E * ks, world, dtr), "unit": UNIT, "steps": ks,
                           "ms_per_step": dtr / ks * 1e3,
                           "bridges_equal_planted": bool(np.array_equal(rres.numpy(), g.planted)),
                           "note": "kernels read the pinned, mapped host buffers over the host link "
                                   "(opts.host_read); the device holds no copy of the edges"}
        del ctx_r

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, n, dt = cpu_oracle_rate(g, cfg["M"], args.cpu_sample)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"Sec. 3 pipeline + Alg. 1 (single-threaded C) on the first {n} edges of the workload; "
                         f"{dt:.1f} s"}
        cores = os.cpu_count() or 1
        prate, pdt, pbr = cpu_oracle_parallel_rate(g, cores)
        cpu_all = {"value": prate, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "cpu": cpu_model(),
                   "sample": f"the whole graph: Alg. 2 on {cores} partitions in parallel, one merge, Alg. 1 "
                             f"(the oracle's C, one thread per partition); {pdt:.2f} s",
                   "bridges_equal": bool(np.array_equal(pbr, timed_out))}

    # the batched and served workloads on the same GPU, after the large one's buffers are gone
    legs = {}
    if rank == 0 and world == 1 and args.workload == "large":
        del du, dv, ctx
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        if not args.no_batched:
            legs["batched"] = batched_leg(args, dev, with_cpu=not args.no_cpu)
            torch.cuda.empty_cache()
        if not args.no_served:
            legs["served"] = served_leg(args, dev, with_cpu=not args.no_cpu)
            torch.cuda.empty_cache()

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": workload_name(args.workload, g),
                       "V": V, "E": E, "M": cfg["M"], "fan_in": cfg["fan_in"],
                       "blocks_per_partition": cfg["blocks_per_partition"], "block": cfg["block"],
                       "warm_edges": cfg["warm_edges"], "l2": "inputs (8E bytes) larger than L2; no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "bridges": n_found, "bridges_equal_planted": correct,
                       "timed_output_equal_planted": timed_correct,
                       "autotuned_plan": plan, "stage_ms_by_M": sweep},
            "clocks": ck, "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all, "pipelined_two_calls_in_flight": pipelined,
            "per_call_ms": None if not hist else {
                "median": statistics.median(h["total"] for h in hist), "min": min(h["total"] for h in hist),
                "max": max(h["total"] for h in hist), "calls": len(hist),
                "note": "CUDA-event time of each of the last timed calls (stage events)"},
        }
        line.update(legs)
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


AP_METRIC = "input edges/s to exact articulation points and bridges"


def planted_cut_vertices(g):
    """Cut vertices of a generated graph whose blocks are its dense cores and its planted bridges:
    the bridge ends that have another edge (true by construction of the large workload)."""
    loop = g.u == g.v
    deg = np.bincount(np.concatenate([g.u[~loop], g.v[~loop]]), minlength=g.V)
    ends = np.unique(g.planted.ravel())
    return ends[deg[ends] >= 2]


def cpu_oracle_ap_rate(g, sample_edges):
    """The oracle's articulation points (Tarjan low/disc, single-threaded C) on a prefix sample."""
    import oracle

    n = min(sample_edges, g.E)
    u = np.ascontiguousarray(g.u[:n])
    v = np.ascontiguousarray(g.v[:n])
    t = time.perf_counter()
    oracle.articulation_points(u, v, g.V)
    dt = time.perf_counter() - t
    return n / dt / 1e9, n, dt


def run_articulation(args, world, rank, local):
    """Articulation points (and bridges) of the large workload; a step is one
    bridges_articulation_points call: one fused read of the 1.07 G edges for the certificate and
    the block pass (the automatic form for this plan), or the bridge path and then a second pass."""
    import torch

    import paper_2108_07346_gb300 as pb

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    over = {} if args.density is None else {"p": args.density}
    g = graphgen.workload("large", **over)
    E, V = g.E, g.V
    du = torch.from_numpy(g.u).to(dev)
    dv = torch.from_numpy(g.v).to(dev)
    ctx = pb.Context(device=dev, profile=True, M=args.M, ap_fused=-1 if args.ap_two_pass else 0)
    stream = torch.cuda.current_stream(dev)
    plan = ctx.autotune(du, dv, V, reps=3) if args.M <= 0 and not args.no_tune else None
    pts, br = ctx.articulation_points(du, dv, V, args.M, with_bridges=True)
    expect = planted_cut_vertices(g)
    correct = bool(np.array_equal(pts.cpu().numpy(), expect) and np.array_equal(br.cpu().numpy(), g.planted))
    out = torch.empty(max(V, 1), dtype=torch.int32, device=dev)
    cnt = torch.zeros(2, dtype=torch.int64, device=dev)
    for _ in range(args.warmup):
        ctx.articulation_points(du, dv, V, args.M, counts_device=cnt, out=out, stream=stream)
    torch.cuda.synchronize()

    clocks = Clocks(local)
    clocks.start()
    clocks.mark("t0")
    l0 = ctx.launches()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        ctx.articulation_points(du, dv, V, args.M, counts_device=cnt, out=out, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark("t1")
    launches = ctx.launches() - l0
    ms_total = reduce_max(e0.elapsed_time(e1), dev)
    ck = clocks.stop()
    n_pts, n_br = (int(x) for x in cnt.cpu())
    steps_seen = min(args.steps, 32)
    ap_hist = ctx.ap_stage_ms_history(steps_seen)
    br_hist = ctx.stage_ms_history(steps_seen)
    cfg = ctx.last_config()
    warm = cfg["warm_edges"] if cfg["warm_edges"] > 0 else None
    ap_warm = cfg["ap_warm_edges"] if cfg["ap_warm_edges"] >= 0 else None
    peak, peak_kind = peaks()
    kernels = {}
    fused = cfg.get("ap_fused", 0) == 1
    if fused and ap_hist and br_hist:
        # one read of the list: the warm-up prefix (its own launch), then the fused stream over the
        # other E - warm edges for both the certificate and the classes
        fs_bpe = FUSED_TRAFFIC["bytes_per_edge"] if FUSED_TRAFFIC["blocks_sha"] == blocks_sha() else None
        kernels = {"fused stream (ap_fused_kernel<forest, vec>)": (statistics.mean(h["stream"] for h in ap_hist),
                                                                  E - (warm or 0), fs_bpe)}
    elif warm is not None and ap_warm is not None and ap_hist and br_hist:
        fe = E - cfg["M"] * warm
        se = E - ap_warm
        ap_bpe = AP_TRAFFIC["bytes_per_edge"] if AP_TRAFFIC["blocks_sha"] == blocks_sha() else None
        fo_bpe = TRAFFIC["bytes_per_edge"] if TRAFFIC["certify_sha"] == certify_sha() else None
        kernels = {
            "block pass stream (ap_pass_kernel<cache, vec>)": (statistics.mean(h["stream"] for h in ap_hist), se,
                                                               ap_bpe),
            "forest pass (leaf_kernel<cache, vec>)": (statistics.mean(h["forest"] for h in br_hist), fe, fo_bpe),
        }
    roof = None
    if kernels:
        name, (ms, edges, bpe) = max(kernels.items(), key=lambda kv: kv[1][0])
        achieved = 8.0 * edges / (ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None if bpe is None else bpe * edges, "kernel": name, "algorithmic_bytes": 8 * edges, "peak_kind": peak_kind,
                "per_kernel": {k: {"ms": m, "GB_per_s": 8.0 * e / (m * 1e-3) / 1e9,
                                   "frac": 8.0 * e / (m * 1e-3) / 1e9 / peak,
                                   "traffic": None if x is None else x * e} for k, (m, e, x) in kernels.items()},
                "ap_stage_ms_mean": {k: statistics.mean(h[k] for h in ap_hist) for k in ap_hist[0]},
                "bridge_stage_ms_mean": {k: statistics.mean(h[k] for h in br_hist) for k in br_hist[0]}}

    e2e = None
    if not args.no_e2e:
        # the user's call from host memory: bridges_articulation_points_host copies the pinned edges
        # in, runs the path and copies the cut vertices out
        hu = torch.from_numpy(g.u).pin_memory()
        hv = torch.from_numpy(g.v).pin_memory()
        hpts = torch.empty(max(V, 1), dtype=torch.int32).pin_memory()
        ctx_h = pb.Context(device=dev, M=args.M)
        ctx_h.articulation_points_host(hu, hv, V, args.M, out=hpts)
        ks = max(1, min(args.steps, args.e2e_steps))
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        nb = 0
        for _ in range(ks):
            nb = ctx_h.articulation_points_host(hu, hv, V, args.M, out=hpts).shape[0]
        torch.cuda.synchronize()
        dt = reduce_max(time.perf_counter() - t0, dev)
        e2e = {"value": whole_job_rate(E * ks, world, dt), "unit": UNIT, "h2d_bytes_per_step": 8 * E,
               "d2h_bytes_per_step": 8 + 4 * nb, "steps": ks, "ms_per_step": dt / ks * 1e3}
        del ctx_h

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, n, dt = cpu_oracle_ap_rate(g, args.ap_cpu_sample)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"Tarjan low/disc articulation points (single-threaded C) on the first {n} edges of the "
                         f"workload; {dt:.1f} s"}
    if rank == 0:
        line = {
            "metric": AP_METRIC, "value": whole_job_rate(E * args.steps, world, ms_total * 1e-3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": workload_name("articulation", g),
                       "V": V, "E": E, "M": cfg["M"], "warm_edges": cfg["warm_edges"],
                       "form": "one fused read of the list" if fused else "bridge path, then a second pass",
                       "block_pass_prefix_edges": cfg["ap_warm_edges"], "block_pass_blocks": cfg["ap_blocks"],
                       "l2": "inputs (8E bytes) larger than L2; no flush",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "cut_vertices": n_pts, "bridges": n_br, "equal_construction": correct,
                       "autotuned_plan": plan},
            "clocks": ck, "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def make_batch(seed, count):
    """The batched workload: `count` graphs with V log-uniform in [64, 4096], density in
    [0.1, 0.9], 1-32 planted bridges each (pendant vertices and an inter-cluster tree)."""
    us, vs, Vs, planted = [], [], [], []
    for i in range(count):
        g = graphgen.generate(graphgen.workload_spec("batched", seed, i))
        us.append(np.array(g.u))
        vs.append(np.array(g.v))
        Vs.append(g.V)
        planted.append(g.planted)
    off = np.concatenate([[0], np.cumsum([len(x) for x in us])]).astype(np.int64)
    return np.concatenate(us), np.concatenate(vs), off, np.array(Vs, np.int32), planted


def batched_leg(args, dev, with_cpu=True):
    """The batched workload (4,096 graphs, two persistent launches per step) on device `dev`:
    graphs/s, per-step latency, the last timed step's output against the oracle, one plain call
    per graph for comparison.  Returns a dict (the standalone line's body)."""
    import concurrent.futures

    import torch

    import oracle
    import paper_2108_07346_gb300 as pb

    u, v, off, Vs, planted = make_batch(3, args.graphs)
    G, E = len(Vs), int(off[-1])
    du = torch.from_numpy(u).to(dev)
    dv = torch.from_numpy(v).to(dev)
    ctx = pb.Context(device=dev)
    stream = torch.cuda.current_stream(dev)
    out, counts, out_off = ctx.find_batched(du, dv, off, Vs)

    def time_steps(n):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(n):
            ctx.find_batched(du, dv, off, Vs, out=out, counts=counts, sync=False)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / n

    # the automatic plan, then the plan the batched autotuner picks (both outside the timed region)
    for _ in range(args.warmup):
        ctx.find_batched(du, dv, off, Vs, out=out, counts=counts, sync=False)
    auto_ms = time_steps(max(1, args.steps))
    plan, tune_us = (None, None) if args.no_tune else ctx.batch_autotune(du, dv, off, Vs, reps=5)
    for _ in range(args.warmup):
        ctx.find_batched(du, dv, off, Vs, out=out, counts=counts, sync=False)
    torch.cuda.synchronize()
    steps = max(1, args.steps)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    l0 = ctx.launches()
    ev[0].record(stream)
    for i in range(steps):
        ctx.find_batched(du, dv, off, Vs, out=out, counts=counts, sync=False)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    launches = ctx.launches() - l0
    step_ms = np.array([ev[i].elapsed_time(ev[i + 1]) for i in range(steps)])
    ms = float(ev[0].elapsed_time(ev[steps])) / steps
    # the last timed step's output, graph by graph
    cnt = counts.cpu().numpy()
    o = out.cpu().numpy()
    got = [o[out_off[g]:out_off[g] + 2 * max(int(cnt[g]), 0)].reshape(-1, 2) for g in range(G)]
    planted_ok = all({tuple(x) for x in planted[g].tolist()} <= {tuple(x) for x in got[g].tolist()} for g in range(G))
    # one plain call per graph, same GPU, same stream
    plain = pb.Context(device=dev)
    cnt_d = torch.zeros(1, dtype=torch.int64, device=dev)
    outp = torch.empty(2 * 4096, dtype=torch.int32, device=dev)
    for g in range(min(G, 64)):
        plain.find(du[off[g]:off[g + 1]], dv[off[g]:off[g + 1]], int(Vs[g]), 1, out=outp, count_device=cnt_d)
    torch.cuda.synchronize()
    p0 = torch.cuda.Event(enable_timing=True)
    p1 = torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for g in range(G):
        plain.find(du[off[g]:off[g + 1]], dv[off[g]:off[g + 1]], int(Vs[g]), 1, out=outp, count_device=cnt_d)
    p1.record(stream)
    torch.cuda.synchronize()
    ms_plain = p0.elapsed_time(p1)
    cpu = None
    if with_cpu:
        # the oracle (Sec. 3 pipeline + Alg. 1 in C) on every graph, one graph per host core (the C
        # calls release the GIL); its bridges are compared with the timed step's, graph by graph
        cores = os.cpu_count() or 1
        t0 = time.perf_counter()
        with concurrent.futures.ThreadPoolExecutor(cores) as ex:
            ref = list(ex.map(lambda g: oracle.bridges(u[off[g]:off[g + 1]], v[off[g]:off[g + 1]], int(Vs[g]), 1),
                              range(G)))
        dt = time.perf_counter() - t0
        equal = sum(int(np.array_equal(ref[g], got[g])) for g in range(G))
        cpu = {"value": G / dt, "unit": "graphs/s", "cores": cores, "kind": "oracle",
               "sample": f"all {G} graphs, one per host thread ({dt:.1f} s)",
               "graphs_equal_to_timed_step": equal, "graphs": G}
    peak, kind = peaks()
    del du, dv, ctx, plain
    return {
        "metric": "graphs/s (batched bridge queries)", "value": G / (ms * 1e-3), "unit": "graphs/s",
        "steps": steps, "warmup": args.warmup, "ms_per_step": ms,
        "step_latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                            "max": float(step_ms.max())},
        "config": {"workload": f"batched: {G} graphs, V log-uniform [64, 4096], density U[0.1, 0.9], 1-32 planted "
                               f"bridges each, seed 3", "graphs": G, "E_total": E,
                   "planted_subset_found": planted_ok, "launches_per_step": launches / steps,
                   "tuned_plan": plan, "automatic_plan_ms_per_step": auto_ms,
                   "l2": "inputs (8E bytes, 4.3 GB) larger than L2; no flush"},
        "input_GE_per_s": E / (ms * 1e-3) / 1e9,
        "roofline": {"bound": "hbm", "achieved": 8.0 * E / (ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": 8.0 * E / (ms * 1e-3) / 1e9 / peak, "peak_kind": kind,
                     "kernel": "certify_kernel + bridge_kernel (whole step)"},
        "plain_per_graph": {"value": G / (ms_plain * 1e-3), "unit": "graphs/s", "ms_total": ms_plain,
                            "note": "one bridges_find_ctx call per graph on the same stream"},
        "speedup_vs_plain": ms_plain / ms,
        "cpu_baseline": cpu,
    }


def run_batched(args, world, rank, local):
    import torch

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    leg = batched_leg(args, dev, with_cpu=not args.no_cpu)
    line = {"metric": leg.pop("metric"), "value": leg.pop("value"), "unit": leg.pop("unit"), "n_gpus": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic"}
    line.update(leg)
    print(json.dumps(line), flush=True)


class RequestStream:
    """The served workload's requests, each a fresh seeded graph (workload_spec("served", 4, i)),
    generated on the device in batches of `batch` consecutive requests (one batch per call of the
    generator: two stream synchronisations per batch; 8 graphs, about 64 MB of edges, stay in L2
    while the generator scatters them to their shuffled positions) by `threads` producer threads,
    each on its own stream, up to `ahead` requests (and `max_bytes` of edges) ahead of the
    consumer, which takes them in order.  Generation time is ingest, reported apart."""

    def __init__(self, dev, first, count, ahead=512, max_bytes=6 << 30, variant="primary", threads=3, batch=8):
        import threading

        self.dev, self.first, self.count = dev, first, count
        self.ahead, self.max_bytes, self.batch = ahead, max_bytes, batch
        self.bytes = 0
        self.ready = {}
        self.next = first  # the next request the consumer takes
        self.cv = threading.Condition()
        self.gen_s = 0.0
        self.error = None
        self.variant = variant
        self.threads = [threading.Thread(target=self._run, args=(k, threads), daemon=True) for k in range(threads)]
        for t in self.threads:
            t.start()

    def spec(self, i):
        import dataclasses

        s = graphgen.workload_spec("served", 4, i)
        return dataclasses.replace(s, n_clusters=1, n_extra=0) if self.variant == "stress" else s

    def _run(self, k, n):
        import torch

        try:
            st = torch.cuda.Stream(self.dev) if torch.device(self.dev).type == "cuda" else None
            end = self.first + self.count
            for b0 in range(self.first + k * self.batch, end, n * self.batch):
                b1 = min(end, b0 + self.batch)
                with self.cv:  # stay within `ahead` requests and `max_bytes` of the consumer
                    while b1 - 1 - self.next >= self.ahead or (self.bytes > self.max_bytes and b0 > self.next):
                        self.cv.wait()
                t0 = time.perf_counter()
                gs = graphgen.generate_device_many([self.spec(i) for i in range(b0, b1)], self.dev, stream=st)
                dt = time.perf_counter() - t0
                with self.cv:
                    self.gen_s += dt
                    for i, g in zip(range(b0, b1), gs):
                        self.bytes += 8 * g.E
                        self.ready[i] = g
                    self.cv.notify_all()
        except Exception as e:  # surfaced to the consumer
            with self.cv:
                self.error = e
                self.cv.notify_all()

    def qsize(self):
        with self.cv:
            return len(self.ready)

    def get(self):
        with self.cv:
            while self.next not in self.ready:
                if self.error is not None:
                    raise RuntimeError(f"request generation failed: {self.error!r}")
                self.cv.wait()
            i = self.next
            g = self.ready.pop(i)
            self.next += 1
            self.cv.notify_all()
            return i, g

    def release(self, g):
        with self.cv:
            self.bytes -= 8 * g.E
            self.cv.notify_all()


class PoolStream:
    """The stress variant's requests: one ER(V, d) core per request (the served workload's V and
    d draws, no clusters) averages about 60 M edges, too many to generate afresh at 2,000 requests
    per second, so `pool` of them are generated once and request i is pool graph i mod pool
    (the graphs stay resident; the same interface as RequestStream)."""

    def __init__(self, dev, first, count, pool=24):
        import dataclasses

        self.first, self.error, self.gen_s = first, None, 0.0
        self.next = first
        t0 = time.perf_counter()
        self.pool = []
        for k in range(pool):
            s = graphgen.workload_spec("served", 4, k)
            self.pool.append(graphgen.generate_device(dataclasses.replace(s, n_clusters=1, n_extra=0), dev))
        self.gen_s = time.perf_counter() - t0

    def spec(self, i):
        import dataclasses

        s = graphgen.workload_spec("served", 4, (i - self.first) % len(self.pool))
        return dataclasses.replace(s, n_clusters=1, n_extra=0)

    def qsize(self):
        return len(self.pool)

    def get(self):
        i = self.next
        self.next += 1
        return i, self.pool[(i - self.first) % len(self.pool)]

    def release(self, g):
        pass


def served_leg(args, dev, with_cpu=True):
    """The served workload as configured: args.requests Poisson arrivals (mean args.rate per s),
    each a fresh seeded graph generated on the device, against the continuous-batching server
    under a args.budget_gb device-memory budget; p50 / p99 latency (submit to completion), a
    seeded 1% of the results against the oracle, and plain per-graph calls and the saturated
    server on fresh requests for comparison.  Returns a dict."""
    import concurrent.futures

    import torch

    import oracle
    import paper_2108_07346_gb300 as pb

    stress = args.served_variant == "stress"
    N = args.requests
    rng = np.random.default_rng(4)
    arrival = np.cumsum(rng.exponential(1.0 / args.rate, N))
    vrng = np.random.default_rng(41)
    check = set(int(i) for i in vrng.choice(N, max(1, N // 100), replace=False))
    srv = pb.Server(device=dev, mem_budget=int(args.budget_gb * (1 << 30)), max_slots=args.slots)
    # warm-up: a few requests past the measured range (kernels loaded, graphs captured)
    if stress:
        reqs = PoolStream(dev, 0, N)
        warm = reqs
    else:
        warm = RequestStream(dev, N + 1_000_000, 32, variant=args.served_variant)
    for _ in range(32):
        _, g = warm.get()
        srv.wait(srv.submit(g.u, g.v, g.V))
        warm.release(g)
    if stress:
        reqs.next = 0
    else:
        reqs = RequestStream(dev, 0, N, variant=args.served_variant)
    ring = 256
    live = [None] * ring  # (ticket, graph, out)
    lat = np.zeros(N)
    late = np.zeros(N)
    results = {}
    edges = 0
    # the ingest of the first requests is not part of the arrival schedule
    while not stress and reqs.qsize() < min(64, N) and reqs.error is None:
        time.sleep(0.01)

    def finish(j):
        t, g, o = live[j % ring]
        got, ms = srv.wait(t)
        lat[j] = ms
        if j in check:
            results[j] = got.cpu().numpy()
        reqs.release(g)
        live[j % ring] = None

    t0 = time.perf_counter()
    for i in range(N):
        if i >= ring:
            finish(i - ring)
        _, g = reqs.get()
        due = t0 + arrival[i]
        now = time.perf_counter()
        if due > now:
            time.sleep(due - now)
        late[i] = max(0.0, time.perf_counter() - due)
        o = torch.empty(2 * max(g.V - 1, 1), dtype=torch.int32, device=dev)
        live[i % ring] = (srv.submit(g.u, g.v, g.V, out=o), g, o)
        edges += g.E
    for j in range(max(0, N - ring), N):
        finish(j)
    wall = time.perf_counter() - t0
    gen_s = reqs.gen_s
    st = srv.stats()
    # saturation and plain calls on fresh requests past the measured range (same distribution):
    # each chunk is generated first (nothing else on the GPU), then submitted back to back or
    # called one by one, and only that part is timed
    nsat = min(N, args.plain * 2)
    chunk = 128

    def gen_chunk(i0, n):
        if stress:  # the pool's graphs again
            return [reqs.pool[(i - N) % len(reqs.pool)] for i in range(i0, i0 + n)]
        return graphgen.generate_device_many([reqs.spec(i) for i in range(i0, i0 + n)], dev)

    sat_s = 0.0
    for c0 in range(0, nsat, chunk):
        gs = gen_chunk(N + c0, min(chunk, nsat - c0))
        torch.cuda.synchronize()
        ts = time.perf_counter()
        tk = [srv.submit(g.u, g.v, g.V) for g in gs]
        for t in tk:
            srv.wait(t)
        sat_s += time.perf_counter() - ts
        del gs, tk
    srv.close()
    ctx = pb.Context(device=dev)
    cnt = torch.zeros(1, dtype=torch.int64, device=dev)
    outp = torch.empty(2 * 200_000, dtype=torch.int32, device=dev)
    plain_s = 0.0
    for c0 in range(0, args.plain, chunk):
        gs = gen_chunk(N + nsat + c0, min(chunk, args.plain - c0))
        if c0 == 0:
            for g in gs[:8]:
                ctx.find(g.u, g.v, g.V, 0, out=outp, count_device=cnt)
        torch.cuda.synchronize()
        tp = time.perf_counter()
        for g in gs:
            ctx.find(g.u, g.v, g.V, 0, out=outp, count_device=cnt)
        torch.cuda.synchronize()
        plain_s += time.perf_counter() - tp
        del gs
    cpu = None
    if with_cpu:
        # the oracle (Sec. 3 pipeline + Alg. 1 in C) on the seeded 1% of the requests, regenerated
        # on the host, one per host thread (the C calls release the GIL); its bridges must equal
        # what the server returned for them
        cores = os.cpu_count() or 1
        picks = sorted(check)
        tc = time.perf_counter()

        def one(i):
            g = graphgen.generate(reqs.spec(i))
            return oracle.bridges(g.u, g.v, g.V, 1), g.E

        with concurrent.futures.ThreadPoolExecutor(cores) as ex:
            ref = dict(zip(picks, ex.map(one, picks)))
        dtc = time.perf_counter() - tc
        cpu = {"value": len(picks) / dtc, "unit": "graphs/s", "cores": cores, "kind": "oracle",
               "sample": f"a seeded 1% of the requests ({len(picks)} graphs, {sum(e for _, e in ref.values())} "
                         f"edges), regenerated on the host; {dtc:.1f} s including generation",
               "requests_equal_to_served": sum(int(np.array_equal(ref[i][0], results[i])) for i in picks),
               "requests_checked": len(picks)}
    del ctx
    return {
        "metric": "served graphs/s with p50/p99 latency", "value": N / wall, "unit": "graphs/s",
        "requests": N, "ms_per_request": wall / N * 1e3,
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                       "max": float(lat.max()), "from": "submit to completion, measured by the server"},
        "config": {"workload": (f"served{' (stress)' if stress else ''}: Poisson arrivals {args.rate:g}/s, {N} "
                                f"requests, each a fresh graph, V log-uniform [256, 65536], density U[0.05, 0.6], "
                                + ("one ER(V, d) core per request with pendant paths" if stress else
                                   "clusters of 512 with pendant paths and extra inter-cluster edges") + ", seed 4"),
                   "variant": args.served_variant, "budget_gb": args.budget_gb, "slots": args.slots,
                   "mean_edges": edges / N,
                   "ingest": {"where": ("a pool of 24 graphs generated on the device once, request i is graph "
                                        "i mod 24" if stress else
                                        "generated on the device, 8 requests per generator call, by 3 producer "
                                        "threads ahead of arrival"),
                              "thread_s": gen_s, "per_request_thread_ms": gen_s / N * 1e3},
                   "late_submits": {"over_1ms": int((late > 1e-3).sum()), "p99_ms": float(np.percentile(late, 99) * 1e3)}},
        "served_GE_per_s": edges / wall / 1e9, "offered_per_s": args.rate, "server_stats": st,
        "plain_per_graph": {"value": args.plain / plain_s, "unit": "graphs/s", "requests": args.plain,
                            "note": "one bridges_find_ctx call per fresh request, back to back"},
        "saturation": {"value": nsat / sat_s, "unit": "graphs/s", "requests": nsat,
                       "note": f"fresh requests submitted {chunk} at a time back to back"},
        "speedup_saturated_vs_plain": (nsat / sat_s) / (args.plain / plain_s),
        "cpu_baseline": cpu,
    }


def run_served(args, world, rank, local):
    """Poisson arrivals of bridge queries against the continuous-batching server."""
    import torch

    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    leg = served_leg(args, dev, with_cpu=not args.no_cpu)
    line = {"metric": leg.pop("metric"), "value": leg.pop("value"), "unit": leg.pop("unit"), "n_gpus": 1,
            "steps": leg["requests"], "warmup": 32, "ms_per_step": leg["ms_per_request"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic"}
    line.update(leg)
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=["large", "mid", "small", "batched", "served", "articulation"],
                    default="large")
    ap.add_argument("--requests", type=int, default=100_000, help="served: requests")
    ap.add_argument("--rate", type=float, default=2000.0, help="served: mean arrivals per second")
    ap.add_argument("--slots", type=int, default=8, help="served: concurrent units of work")
    ap.add_argument("--budget-gb", type=float, default=40.0, help="served: device-memory budget")
    ap.add_argument("--plain", type=int, default=1000, help="served: plain calls timed for comparison")
    ap.add_argument("--served-variant", choices=["primary", "stress"], default="primary",
                    help="served: clusters of 512 per request (primary) or one ER core per request (stress)")
    ap.add_argument("--graphs", type=int, default=4096, help="graphs of the batched workload")
    ap.add_argument("--density", type=float, default=None, help="override the ER density (profiling)")
    ap.add_argument("--M", type=int, default=0, help="partitions (0: automatic)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (use --M or the default plan)")
    ap.add_argument("--no-sweep", action="store_true", help="skip the per-M stage timings")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--exchange", choices=["nccl", "gloo"], default="nccl",
                    help="N > 1: certificates through NCCL device buffers or gloo host buffers")
    ap.add_argument("--same-device", action="store_true",
                    help="N > 1 with gloo: every rank on cuda:0 (a test of the sharded path on one GPU)")
    ap.add_argument("--no-batched", action="store_true", help="large workload: skip the batched leg")
    ap.add_argument("--no-pipelined", action="store_true", help="large workload: skip the two-calls-in-flight figure")
    ap.add_argument("--no-served", action="store_true", help="large workload: skip the served leg")
    ap.add_argument("--ap-two-pass", action="store_true",
                    help="articulation workload: the bridge path, then a second pass (not the fused read)")
    ap.add_argument("--cpu-sample", type=int, default=2_000_000_000, help="oracle sample (edges; whole graph)")
    ap.add_argument("--ref-sample", type=int, default=150_000_000, help="reference arm sample per step (edges)")
    ap.add_argument("--ap-cpu-sample", type=int, default=100_000_000,
                    help="articulation: oracle sample for cpu_baseline (edges)")
    args = ap.parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batched":
        run_batched(args, world, rank, local)
    elif args.workload == "served":
        run_served(args, world, rank, local)
    elif args.workload == "articulation":
        run_articulation(args, world, rank, local)
    elif world > 1:
        run_sharded(args, world, rank, local)
    else:
        run_native(args, world, rank, local)


if __name__ == "__main__":
    main()
