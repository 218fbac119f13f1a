#!/usr/bin/env python
"""All-nodes closeness estimation throughput on one GB300.

Workload (the configuration the headline metric is quoted on): undirected
R-MAT scale 20, edge factor 16 (a=0.57, b=c=0.19, graph seed 1), self-loops
and duplicates removed, largest connected component, k = 256 sources (sample
seed 2) in one bit-packed multi-source traversal (4 uint64 words per node),
sampling, pivoting, pivoting-upper-bound and hybrid estimates (eps = 1/16)
for every node.

A step = one cc_estimate call (every estimator for every node) with the
graph resident in HBM.  value = k * m / step time in GTEPS (m = undirected
edges of the kept component, each counted once).  e2e = the same call with
pinned host output buffers (sample upload and result download inside the
timed region).  The L2 is flushed (256 MB write) before every timed step.

--impl reference times the CPU oracle (breadth-first searches with O(1)
running state per node, one source per host thread on every core) on a
bounded sample of the same workload.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SCALE, EF, GSEED, SSEED, K = 20, 16, 1, 2, 256
WORKLOAD = "rmat-s20-ef16-lcc-k256"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=SCALE)
    ap.add_argument("--k", type=int, default=K)
    ap.add_argument("--cpu-sources", type=int, default=12,
                    help="sources in the bounded CPU-oracle sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=100,
                    help="serve workload: requests in each Poisson stream")
    ap.add_argument("--slots", type=int, default=4, help="serve workload: slots")
    ap.add_argument("--pool", default="paper", choices=["small", "paper"],
                    help="serve workload: graph pool (paper: R-MAT scales 12..22, grids "
                         "256^2..4096^2, the serving configuration; small: R-MAT to scale "
                         "20, grids to 2048^2)")
    ap.add_argument("--road-nodes", type=int, default=4 << 20,
                    help="road4m workload: points of the road-like graph (a smaller "
                         "graph for profiling runs)")
    ap.add_argument("--workload", default="rmat20",
                    choices=["rmat20", "config1", "batch64", "road4m", "rt22", "serve", "adaptive",
                             "nodeweighted", "reach", "grid"],
                    help="rmat20 is the headline; the others print their own line")
    return ap.parse_args()


def max_over_ranks(x, device=None):
    """Largest value of x over the ranks of the default process group (x
    itself when there is none): the slowest rank's time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world_size, units_per_rank, seconds):
    """Units all ranks processed per second of the slowest rank: every rank
    runs its own replica of the workload (weak scaling)."""
    return world_size * units_per_rank / seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def config(args, n, m):
    return {"workload": f"rmat-s{args.scale}-ef{EF}-lcc-k{args.k}",
            "graph": f"undirected R-MAT scale {args.scale}, edge factor {EF}, "
                     f"a=0.57 b=c=0.19, seed {GSEED}, LCC",
            "n": n, "m": m, "k": args.k, "sample_seed": SSEED,
            "estimators": ["sampling", "pivoting", "pivot_upper", "hybrid"],
            "eps": f"1/{round(args.k ** 0.5)}",
            "l2": "flushed before every timed step (256 MB write)",
            "parallelism": "replicas"}


# --------------------------------------------------------------- CPU oracle

def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return os.cpu_count() or 1, model


def streaming_pass_threads(og, sources, threads):
    """The oracle's streaming pass (one BFS per source with O(1) running
    state per node) with the sources split into `threads` contiguous runs,
    one host thread each (the oracle's C routine runs without the
    interpreter lock), each with its own accumulators; merged afterwards:
    sums added, the pivot the nearest source with ties to the smaller
    sample index, S of the sampled nodes concatenated."""
    from concurrent.futures import ThreadPoolExecutor
    import numpy as np
    from oracle import oracle as orc
    src = np.ascontiguousarray(sources, dtype=np.int32)
    runs = [r for r in np.array_split(np.arange(src.size), max(1, threads)) if r.size]
    with ThreadPoolExecutor(len(runs)) as ex:
        parts = list(ex.map(lambda r: orc.streaming_pass(og, src[r]), runs))
    tot = parts[0]["sum"].copy()
    piv = parts[0]["pivot"].copy()
    dl = parts[0]["delta"].copy()
    for r, p in zip(runs[1:], parts[1:]):
        tot += p["sum"]
        better = p["delta"] < dl
        piv[better] = p["pivot"][better] + r[0]
        dl[better] = p["delta"][better]
    return dict(sum=tot, pivot=piv, delta=dl,
                S_samp=np.concatenate([p["S_samp"] for p in parts]))


def cpu_oracle_gteps(edges, k_all, nsrc, seed=SSEED):
    """Time the oracle's streaming pass on one core over `nsrc` of the k
    sampled sources, and over all k sources split across every host core;
    returns (single-core GTEPS, its seconds, all-core GTEPS, its seconds,
    cores, CPU model)."""
    from oracle import oracle as orc
    n, s, d = edges
    og = orc.csr_from_edges(n, s, d)
    C = orc.choose_sample(og.n, k_all, seed)
    t0 = time.perf_counter()
    orc.streaming_pass(og, C[:nsrc])
    dt1 = time.perf_counter() - t0
    cores, model = host_cpu()
    t0 = time.perf_counter()
    streaming_pass_threads(og, C, cores)
    dtn = time.perf_counter() - t0
    return nsrc * og.m / dt1 / 1e9, dt1, k_all * og.m / dtn / 1e9, dtn, cores, model


def run_reference(args):
    import synth
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    edges = synth.rmat_edges(args.scale, EF, seed=GSEED)
    from oracle import oracle as orc
    n, s, d = edges
    og = orc.csr_from_edges(n, s, d)
    C = orc.choose_sample(og.n, args.k, SSEED)
    cores, model = host_cpu()
    per_step = min(args.k, cores)           # one source per host thread
    for i in range(args.warmup):
        streaming_pass_threads(og, C[:per_step], cores)
    times = []
    for i in range(args.steps):
        lo = (i * per_step) % args.k
        sub = C[lo:lo + per_step]
        t0 = time.perf_counter()
        streaming_pass_threads(og, sub, cores)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    val = len(sub) * og.m * args.steps / tot / 1e9
    sample = (f"{per_step} of the {args.k} sampled sources per step, one per host "
              f"thread on {cores} cores ({model}); streaming pass: BFS + running "
              f"sum/pivot per node, per-thread accumulators merged")
    line = {"impl": "reference", "metric": "source-edge traversals/s (GTEPS)",
            "value": val, "unit": "GTEPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic",
            "config": config(args, og.n, og.m),
            "cpu_baseline": {"value": val, "unit": "GTEPS", "cores": cores,
                             "kind": "oracle", "sample": sample, "cpu_model": model},
            "e2e": {"value": val, "unit": "GTEPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- GPU arm

class Clocks:
    """nvidia-smi sampler running during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi missing"]}
        time.sleep(0.15)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for row in self.f.read().splitlines():
            parts = [x.strip() for x in row.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_sha():
    """sha256 over the traversal kernel's sources (with the header of its
    build-time constants)."""
    h = hashlib.sha256()
    for f in ("msbfs_dev.cuh", "msbfs.cu", "cc_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1409_0035_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def kernel_traffic(path_md):
    """Per-launch DRAM bytes from the committed ncu summary, only while the
    kernel source is unchanged since the capture."""
    meta = {}
    try:
        for line in open(path_md):
            if ":" in line and line.strip().startswith(("source_sha256", "dram_bytes_per_launch")):
                k, v = line.split(":", 1)
                meta[k.strip()] = v.strip().strip("`")
    except OSError:
        return None
    if meta.get("source_sha256") != kernel_source_sha():
        return None
    try:
        return float(meta["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1409_0035_gb300 import build as ccbuild
    ccbuild.build()
    import paper_1409_0035_gb300 as cc
    import synth

    edges = synth.rmat_edges(args.scale, EF, seed=GSEED)
    g, _ = cc.cc_graph_from_edges(*edges)
    n, arcs, _, _ = cc.cc_graph_info(g)
    m = arcs // 2
    k = args.k
    C = cc.cc_sample_choose(g, k, SSEED)
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", local)

    # device outputs
    shat = torch.empty((4, n), dtype=torch.float64, device=dev)
    clo = torch.empty((4, n), dtype=torch.float64, device=dev)
    piv = torch.empty(n, dtype=torch.int32, device=dev)
    dl = torch.empty(n, dtype=torch.int32, device=dev)
    ssum = torch.empty(n, dtype=torch.int64, device=dev)
    hyb = torch.empty((n, 6), dtype=torch.int64, device=dev)
    o = cc.cc_out()
    for e in range(4):
        o.s_hat[e] = shat[e].data_ptr()
        o.closeness[e] = clo[e].data_ptr()
    o.pivot, o.delta, o.sample_sum, o.hyb_int = (piv.data_ptr(), dl.data_ptr(),
                                                 ssum.data_ptr(), hyb.data_ptr())
    opts = cc.cc_opts_default(k)
    opts.device_outputs = 1
    opts.stream = stream.cuda_stream
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        cc.cc_estimate(g, C, opts, o)

    for _ in range(max(3, args.warmup)):
        step()
    stats = cc.cc_last_pass_stats(g)
    trace = cc.cc_last_pass_trace(g)

    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    t_total, kms, kbytes, klaunch, kall, replays = 0.0, 0.0, 0.0, 0, 0, 0
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    for _ in range(args.steps):
        flush.zero_()
        ev0.record(stream)
        step()
        ev1.record(stream)
        ev1.synchronize()
        t_total += ev0.elapsed_time(ev1)
        nl, ms, b, nk = cc.cc_last_call_timing(g)
        replays += int(cc.cc_last_call_graph(g))
        kall += nk
        klaunch += nl
        kms += ms
        kbytes += b
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    t_total = max_over_ranks(t_total, dev)
    ms_step = t_total / args.steps
    value = whole_job_rate(ws, k * m * args.steps, t_total / 1e3) / 1e9

    # End to end: pinned host outputs, result download inside the region.
    host = {"s_hat": torch.empty((4, n), dtype=torch.float64, pin_memory=True),
            "closeness": torch.empty((4, n), dtype=torch.float64, pin_memory=True),
            "pivot": torch.empty(n, dtype=torch.int32, pin_memory=True),
            "delta": torch.empty(n, dtype=torch.int32, pin_memory=True),
            "sum": torch.empty(n, dtype=torch.int64, pin_memory=True),
            "hyb": torch.empty((n, 6), dtype=torch.int64, pin_memory=True)}
    oh = cc.cc_out()
    for e in range(4):
        oh.s_hat[e] = host["s_hat"][e].data_ptr()
        oh.closeness[e] = host["closeness"][e].data_ptr()
    oh.pivot, oh.delta = host["pivot"].data_ptr(), host["delta"].data_ptr()
    oh.sample_sum, oh.hyb_int = host["sum"].data_ptr(), host["hyb"].data_ptr()
    opts_h = cc.cc_opts_default(k)
    opts_h.stream = stream.cuda_stream
    d2h = sum(t.numel() * t.element_size() for t in host.values())
    h2d = k * 4
    cc.cc_estimate(g, C, opts_h, oh)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e2e_t = 0.0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cc.cc_estimate(g, C, opts_h, oh)
        e2e_t += time.perf_counter() - t0
    if ws > 1:
        torch.distributed.barrier()
    e2e_t = max_over_ranks(e2e_t, dev)
    e2e = whole_job_rate(ws, k * m * args.steps, e2e_t) / 1e9

    # One source per launch: the same traversal with one bit, k launches.
    nsingle = 16
    t0 = time.perf_counter()
    cc.cc_sampling_sums_single(g, C[:nsingle])
    single_t = time.perf_counter() - t0
    single_gteps = nsingle * m / single_t / 1e9

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    per_launch_bytes = kbytes / max(1, klaunch)
    per_launch_ms = kms / max(1, klaunch)
    achieved = per_launch_bytes / (per_launch_ms / 1e3) / 1e9
    traffic = kernel_traffic(os.path.join(ROOT, "profiles", "msbfs_rmat20_k256.md"))
    gpu_launches = kall

    line = {"metric": "source-edge traversals/s (GTEPS)", "value": value,
            "unit": "GTEPS", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": config(args, n, m),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                         "kernel": "msbfs_kernel<4>", "peak_source": peak_src,
                         "alg_bytes_per_launch": per_launch_bytes,
                         "ms_per_launch": per_launch_ms,
                         "launches_per_step": klaunch / args.steps},
            "e2e": {"value": e2e, "unit": "GTEPS", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": gpu_launches,
            "steps_replaying_captured_graph": replays,
            "clocks": clk,
            "single_source_per_launch": {"value": single_gteps, "unit": "GTEPS",
                                         "sources": nsingle,
                                         "speedup": value / single_gteps},
            "pass_stats": stats,
            "level_trace": [{"level": l, "us": ns / 1e3, "top_down": td, "frontier": fr,
                             "frontier_arcs": fa, "words": wd}
                            for (l, ns, td, fr, fa, wd) in trace],
            "estimates_per_s": n / (ms_step / 1e3)}

    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        g1, dt1, gn, dtn, cores, model = cpu_oracle_gteps(edges, k, args.cpu_sources)
        line["cpu_baseline"] = {
            "value": gn, "unit": "GTEPS", "cores": cores, "kind": "oracle",
            "cpu_model": model,
            "sample": f"all {k} sources (streaming BFS pass), one contiguous run of "
                      f"sources per host thread on {cores} cores, {dtn:.1f} s wall",
            "single_core": {"value": g1, "unit": "GTEPS", "cores": 1,
                            "sample": f"{args.cpu_sources} of the {k} sources, "
                                      f"{dt1:.1f} s"}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    cc.cc_graph_free(g)
    if ws > 1:
        torch.distributed.destroy_process_group()


# --------------------------------------------------------------- other configs

def _time_steps(fn, steps, warmup, flush=None):
    """Device time (ms) of `steps` calls of fn after `warmup` calls, CUDA
    events on the current stream, L2 flushed before each timed call."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot = 0.0
    for _ in range(steps):
        if flush is not None:
            flush.zero_()
        e0.record(st)
        fn()
        e1.record(st)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    return tot / steps


def batch64_graphs(master=7):
    """32 R-MAT (scale 10..18, edge factor 8..16), 16 square grids (side
    64..1024), 16 Watts-Strogatz (n = 2^12..2^16, degree 10, p = 0.05); per
    graph k in {16, 64, 256, 512}; all draws from splitmix64(master, i)."""
    import synth
    u = lambda i: float(synth.uniform_at(master, [i])[0])
    out = []
    for g in range(64):
        kind = "rmat" if g < 32 else ("grid" if g < 48 else "ws")
        k = (16, 64, 256, 512)[min(3, int(u(4 * g) * 4))]
        if kind == "rmat":
            scale = 10 + min(8, int(u(4 * g + 1) * 9))
            ef = 8 + min(8, int(u(4 * g + 2) * 9))
            e = synth.rmat_edges(scale, ef, seed=1000 + g)
            desc = f"rmat s{scale} ef{ef}"
        elif kind == "grid":
            side = 64 + int(u(4 * g + 1) * (1024 - 64 + 1))
            e = synth.grid_edges(side, side)
            desc = f"grid {side}"
        else:
            ln = 12 + min(4, int(u(4 * g + 1) * 5))
            e = synth.watts_strogatz_edges(1 << ln, 10, 0.05, seed=2000 + g)
            desc = f"ws 2^{ln}"
        out.append((desc, e, k))
    return out


def serve_pool(paper=False):
    """40 resident graphs: R-MAT scale 12 + (i mod 9), edge factor 16, for
    i < 20; square grids with side 256 * 2^(i mod 4) for the other 20.  With
    `paper`, R-MAT scales 12 + (i mod 11) (up to 22) and grid sides
    256 * 2^(i mod 5) (up to 4096)."""
    import synth
    pool = []
    for i in range(40):
        if i < 20:
            scale = 12 + (i % (11 if paper else 9))
            pool.append((f"rmat s{scale}", synth.rmat_edges(scale, 16, seed=500 + i)))
        else:
            side = 256 << (i % (5 if paper else 4))
            pool.append((f"grid {side}", synth.grid_edges(side, side)))
    return pool


def _serve_stream(cc, srv, R, rate, seed, ns, ms_, start=0):
    """Submit R Poisson arrivals at `rate` requests/s (counter-based draws
    of stream `seed`, from request `start` on) and wait for all; returns
    (latencies ms, source-edges, estimates, wall s)."""
    import numpy as np
    import synth
    c = np.arange(4 * start, 4 * (start + R), dtype=np.uint64)
    u = synth.uniform_at(seed, c)
    gaps = -np.log1p(-u[0::4]) / rate
    gsel = np.minimum((u[1::4] * len(ns)).astype(int), len(ns) - 1)
    est = (0, 1, 3)  # sampling, pivoting, hybrid
    esel = [est[min(2, int(x * 3))] for x in u[2::4]]
    ksel = [(64, 128, 256, 512, 1024)[min(4, int(x * 5))] for x in u[3::4]]
    t0 = time.perf_counter()
    ids, t_next = [], t0
    for i in range(R):
        t_next += gaps[i]
        dt = t_next - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        k = min(ksel[i], ns[gsel[i]])
        # the sample of (graph, k) is fixed (seed SSEED): a repeated request
        # finds its first pass resident
        ids.append((cc.cc_server_submit(srv, int(gsel[i]), esel[i], k, SSEED), i, k))
    work, est_nodes, lat, failed = 0, 0, [], []
    for rid, i, k in ids:
        st = cc.cc_server_wait(srv, rid, 3600000)
        if st != cc.CC_OK:
            failed.append((i, cc.cc_strerror(st)))
            continue
        r = cc.cc_server_result(srv, rid, ns[gsel[i]])
        lat.append(r["latency_ms"])
        work += k * ms_[gsel[i]]
        est_nodes += ns[gsel[i]]
    if failed:
        raise RuntimeError(f"{len(failed)} requests failed, first: {failed[0]}")
    return lat, work, est_nodes, time.perf_counter() - t0


def run_serve(args, cc):
    """Poisson arrivals of (graph, estimator, k) requests over the resident
    pool, continuous batching in the server: first at the offered 200
    requests/s (seed 3), then at 80 % of the rate the server sustained
    there (seed 4), each reporting p50 / p99 latency and throughput."""
    import numpy as np
    pool = serve_pool(paper=args.pool == "paper")
    handles, ns, ms_ = [], [], []
    for desc, (n, s, d) in pool:
        g, _ = cc.cc_graph_from_edges(n, s, d)
        nn, arcs, _, _ = cc.cc_graph_info(g)
        handles.append(g)
        ns.append(nn)
        ms_.append(arcs // 2)
    R = args.requests
    srv = cc.cc_server_create(handles, slots=args.slots)
    try:
        lat, work, est_nodes, wall = _serve_stream(cc, srv, R, 200.0, 3, ns, ms_)
        stats = cc.cc_server_stats(srv)
        cache = cc.cc_server_cache_stats(srv)
        cap = R / wall
        lat2, work2, _, wall2 = _serve_stream(cc, srv, R, 0.8 * cap, 4, ns, ms_, start=R)
        cache2 = cc.cc_server_cache_stats(srv)
    finally:
        cc.cc_server_free(srv)
        for g in handles:
            cc.cc_graph_free(g)
    return {"value": work / wall / 1e9, "ms_per_step": wall * 1e3 / R,
            "requests": R, "wall_s": wall, "requests_per_s": R / wall,
            "offered_requests_per_s": 200.0, "estimates_per_s": est_nodes / wall,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "server_stats": stats, "resident_state": cache, "slots": args.slots,
            "sustainable": {"offered_requests_per_s": 0.8 * cap, "requests": R,
                            "requests_per_s": R / wall2,
                            "p50_ms": float(np.percentile(lat2, 50)),
                            "p99_ms": float(np.percentile(lat2, 99)),
                            "GTEPS": work2 / wall2 / 1e9,
                            "resident_state_hits": cache2["hits"] - cache["hits"]},
            "config": {"workload": "serve", "pool": [d for d, _ in pool],
                       "arrivals": "Poisson 200/s (seed 3), then 80 % of the sustained "
                                   "rate (seed 4)",
                       "k": [64, 128, 256, 512, 1024], "sample_seed": SSEED,
                       "estimators": ["sampling", "pivoting", "hybrid"]}}


def run_extra(args):
    import numpy as np
    import torch
    from paper_1409_0035_gb300 import build as ccbuild
    ccbuild.build()
    import paper_1409_0035_gb300 as cc
    import synth
    torch.cuda.set_device(0)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    line = {"metric": "source-edge traversals/s (GTEPS)", "unit": "GTEPS",
            "higher_is_better": True, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "data": "synthetic", "workload": args.workload}
    if args.workload == "serve":
        line.update(run_serve(args, cc))
    elif args.workload == "adaptive":
        # The headline graph and sample under the error estimate (one eps)
        # and the adaptive hybrid (seven eps values), against the plain
        # hybrid: what SqErrEst and Hyb.-ad cost on top of eq. (4).
        n, s, d = synth.rmat_edges(SCALE, EF, seed=GSEED)
        g, _ = cc.cc_graph_from_edges(n, s, d)
        nn, arcs, _, _ = cc.cc_graph_info(g)
        m = arcs // 2
        C = cc.cc_sample_choose(g, K, SSEED)
        # Device outputs throughout: the hybrid estimate and closeness, its
        # error estimate, the adaptive choice.
        dev = torch.device("cuda", 0)
        st = torch.cuda.current_stream()
        shat = torch.empty(nn, dtype=torch.float64, device=dev)
        clo = torch.empty(nn, dtype=torch.float64, device=dev)
        sqe = torch.empty(nn, dtype=torch.float64, device=dev)
        choice = torch.empty(nn, dtype=torch.int32, device=dev)
        o = cc.cc_opts_default(K)
        o.device_outputs = 1
        o.stream = st.cuda_stream
        out_plain = cc.cc_out()
        out_plain.s_hat[3], out_plain.closeness[3] = shat.data_ptr(), clo.data_ptr()
        out_sq = cc.cc_out()
        out_sq.s_hat[3], out_sq.closeness[3] = shat.data_ptr(), clo.data_ptr()
        out_sq.sq_err = sqe.data_ptr()
        plain = _time_steps(lambda: cc.cc_estimate(g, C, o, out_plain), args.steps,
                            args.warmup, flush)
        sq = _time_steps(lambda: cc.cc_estimate(g, C, o, out_sq), args.steps, args.warmup,
                         flush)
        Cd = np.ascontiguousarray(C, dtype=np.int32)

        def adaptive():
            cc._chk(cc.lib().cc_estimate_adaptive(
                g, Cd.ctypes.data_as(cc.ctypes.c_void_p), K, cc.ctypes.byref(o), 0, None,
                None, shat.data_ptr(), clo.data_ptr(), sqe.data_ptr(), choice.data_ptr()),
                "cc_estimate_adaptive")

        ad = _time_steps(adaptive, args.steps, args.warmup, flush)
        ch = choice.cpu().numpy()
        line.update(metric="all-node estimates/s", unit="estimates/s",
                    value=nn / (ad / 1e3), ms_per_step=ad,
                    plain_hybrid_ms=plain, with_sqerr_ms=sq, adaptive_ms=ad,
                    eps_chosen={str(e): int((ch == i).sum())
                                for i, e in enumerate(cc.ADAPTIVE_EPS)},
                    note="device outputs (hybrid estimate and closeness, error, choice)",
                    config={"workload": "adaptive", "graph": f"R-MAT scale {SCALE}, edge "
                            f"factor {EF}, seed {GSEED}, LCC", "n": nn, "m": m, "k": K})
        cc.cc_graph_free(g)
    elif args.workload == "nodeweighted":
        # Node-weighted closeness (section 5) on the headline graph with
        # Pareto node weights: the weighted sample, then the sampling and
        # hybrid estimates of S_beta (device outputs), beside the unweighted
        # estimate of the same k.
        n, s, d = synth.rmat_edges(SCALE, EF, seed=GSEED)
        g, _ = cc.cc_graph_from_edges(n, s, d)
        nn, arcs, _, _ = cc.cc_graph_info(g)
        m = arcs // 2
        beta = synth.pareto_node_weights(nn, seed=GSEED)
        cc.cc_graph_set_node_weights(g, beta)
        dev = torch.device("cuda", 0)
        st = torch.cuda.current_stream()
        bufs = [torch.empty(nn, dtype=torch.float64, device=dev) for _ in range(4)]
        Sd = torch.empty(K, dtype=torch.int64, device=dev)
        box = {}

        def sample():
            box["C"], box["tau"] = cc.cc_sample_varopt(g, K, SSEED)

        t_sample = _time_steps(sample, args.steps, args.warmup, flush)
        C, tau = box["C"], box["tau"]
        o = cc.cc_opts_default(K)
        o.device_outputs = 1
        o.stream = st.cuda_stream
        w = cc.cc_wout()
        for e in range(2):
            w.s_hat[e], w.closeness[e] = bufs[2 * e].data_ptr(), bufs[2 * e + 1].data_ptr()
        w.S_sampled = Sd.data_ptr()
        t_w = _time_steps(lambda: cc.cc_estimate_node_weighted(g, C, tau, o, out=w),
                          args.steps, args.warmup, flush)
        o.want_hybrid = 0
        t_ws = _time_steps(lambda: cc.cc_estimate_node_weighted(g, C, tau, o, out=w),
                           args.steps, args.warmup, flush)
        o.want_hybrid = 1
        Cu = cc.cc_sample_choose(g, K, SSEED)
        ou = cc.cc_out()
        ou.s_hat[3], ou.closeness[3] = bufs[0].data_ptr(), bufs[1].data_ptr()
        t_u = _time_steps(lambda: cc.cc_estimate(g, Cu, o, ou), args.steps, args.warmup, flush)
        line.update(value=K * m / (t_w / 1e3) / 1e9, ms_per_step=t_w,
                    sample_ms=t_sample, weighted_hybrid_ms=t_w, weighted_sampling_only_ms=t_ws,
                    unweighted_hybrid_ms=t_u, tau=list(tau),
                    certain=int((beta[C].astype(np.uint64) * tau[1] >= tau[0]).sum()),
                    note="value = k m / weighted-hybrid time; the weighted estimate runs "
                         "on chunks of distance rows (two sweeps for the hybrid)",
                    config={"workload": "nodeweighted", "graph": f"R-MAT scale {SCALE}, "
                            f"edge factor {EF}, seed {GSEED}, LCC", "n": nn, "m": m, "k": K,
                            "node_weights": "Pareto(1.2) x 10 + 1, capped at 10^6",
                            "total_weight": int(beta.astype(np.uint64).sum())})
        cc.cc_graph_free(g)
    elif args.workload == "reach":
        # Outbound and inbound estimates (section 6.2) on a directed R-MAT
        # graph kept whole (not strongly connected): every node's bottom-k
        # reachability sample, k = 64.
        kr = 64
        n, s, d = synth.rmat_edges(SCALE, EF, seed=GSEED)
        g, _ = cc.cc_graph_from_edges(n, s, d, directed=True, keep_component=False)
        nn, arcs, _, _ = cc.cc_graph_info(g)
        res = {}
        for name, inb in (("outbound", False), ("inbound", True)):
            t = _time_steps(lambda: cc.cc_reach_estimate(g, kr, SSEED, inb), args.steps,
                            args.warmup, flush)
            r = cc.cc_reach_estimate(g, kr, SSEED, inb)
            lv = cc.cc_last_pass_stats(g)["levels"]
            res[name] = dict(ms=t, levels_total=int(lv), full_samples=int((r["count"] == kr).sum()),
                             empty=int((r["count"] == 0).sum()))
        tot = res["outbound"]["ms"] + res["inbound"]["ms"]
        line.update(metric="node samples/s", unit="nodes/s", value=2 * nn / (tot / 1e3),
                    ms_per_step=tot, outbound=res["outbound"], inbound=res["inbound"],
                    note="value = 2 n / (outbound + inbound time); host outputs",
                    config={"workload": "reach", "graph": f"directed R-MAT scale {SCALE}, edge "
                            f"factor {EF}, seed {GSEED}, all nodes", "n": nn, "arcs": arcs,
                            "k": kr})
        cc.cc_graph_free(g)
    elif args.workload == "batch64":
        specs = batch64_graphs()
        handles, samples, work, kinds = [], [], 0, []
        for i, (desc, (n, s, d), k) in enumerate(specs):
            g, _ = cc.cc_graph_from_edges(n, s, d)
            nn, arcs, _, _ = cc.cc_graph_info(g)
            k = min(k, nn)
            handles.append(g)
            samples.append(cc.cc_sample_choose(g, k, 3000 + i))
            work += k * (arcs // 2)
            kinds.append(desc)
        b = cc.cc_batch_create(handles, samples, autotune=True)
        ms = _time_steps(lambda: cc.cc_batch_run(b), args.steps, args.warmup, flush)
        info = cc.cc_batch_info(b)
        plans = [cc.cc_batch_plan(b, i) for i in range(len(handles))]
        classes = {}
        for p in plans:
            classes.setdefault(p["words"], {"graphs": 0, "teams": p["class_teams"],
                                            "ctas": p["class_ctas"],
                                            "ctas_per_sm": p["ctas_per_sm"], "alpha": {}})
            c = classes[p["words"]]
            c["graphs"] += 1
            c["alpha"][str(p["alpha"])] = c["alpha"].get(str(p["alpha"]), 0) + 1
        seq = 0.0
        per = []
        single_src = 0.0
        for g, C, desc in zip(handles, samples, kinds):
            t = _time_steps(lambda: cc.cc_estimate(g, C), 1, 1)
            seq += t
            per.append((t, desc, len(C), cc.cc_last_pass_stats(g)["levels"]))
        # one source per launch (the traversal alone, no estimates): the
        # same sources on every graph, timed on a bounded share of them
        nsrc = 2
        for g, C in zip(handles, samples):
            t0 = time.perf_counter()
            cc.cc_sampling_sums_single(g, C[:nsrc])
            single_src += (time.perf_counter() - t0) * 1e3 * len(C) / min(nsrc, len(C))
        per.sort(reverse=True)
        by_kind = {}
        for t, desc, k, lv in per:
            by_kind[desc.split()[0]] = by_kind.get(desc.split()[0], 0.0) + t
        line.update(value=work / (ms / 1e3) / 1e9, ms_per_step=ms,
                    sequential={"value": work / (seq / 1e3) / 1e9, "ms": seq},
                    speedup_vs_sequential=seq / ms, plan=info, plan_by_word_width=classes,
                    single_source_per_launch={
                        "ms": single_src, "value": work / (single_src / 1e3) / 1e9,
                        "note": f"{nsrc} sources per graph timed, scaled to its k",
                        "speedup": single_src / ms},
                    sequential_ms_by_kind=by_kind,
                    slowest=[{"graph": d, "k": k, "levels": lv, "ms": t}
                             for t, d, k, lv in per[:6]],
                    config={"workload": "batch64", "graphs": kinds,
                            "source_edges": work})
        cc.cc_batch_free(b)
        for g in handles:
            cc.cc_graph_free(g)
    elif args.workload == "grid":
        # The high-diameter case of the batch and serving pools: a 1024^2
        # grid (stand-in for the paper's grid20), k = 256, every estimator
        # with the hybrid at eps = 1/16 (device outputs).
        side, kg = 1024, 256
        n, s, d = synth.grid_edges(side, side)
        g, _ = cc.cc_graph_from_edges(n, s, d)
        nn, arcs, _, _ = cc.cc_graph_info(g)
        C = cc.cc_sample_choose(g, kg, SSEED)
        dev = torch.device("cuda", 0)
        shat = torch.empty((4, nn), dtype=torch.float64, device=dev)
        o = cc.cc_out()
        for e in range(4):
            o.s_hat[e] = shat[e].data_ptr()
        opts = cc.cc_opts_default(kg)
        opts.device_outputs = 1
        opts.stream = torch.cuda.current_stream().cuda_stream
        ms = _time_steps(lambda: cc.cc_estimate(g, C, opts, o), args.steps, args.warmup, flush)
        st = cc.cc_last_pass_stats(g)
        nl, kms, kb, nk = cc.cc_last_call_timing(g)
        line.update(value=kg * (arcs // 2) / (ms / 1e3) / 1e9, ms_per_step=ms,
                    traversal_launches=nl, traversal_ms=kms, levels=st["levels"],
                    td_levels=st["td_levels"], bu_levels=st["bu_levels"],
                    config={"workload": "grid", "graph": f"{side} x {side} grid", "n": nn,
                            "m": arcs // 2, "k": kg, "eps": "1/16"})
        cc.cc_graph_free(g)
    elif args.workload in ("road4m", "rt22", "config1"):
        if args.workload == "road4m":
            n, s, d, length = synth.road_like_edges(args.road_nodes, seed=1)
            variants = [("round(1000 len)+1", synth.edge_lengths_to_weights(length, 1e3)),
                        ("round(1e6 len)+1", synth.edge_lengths_to_weights(length, 1e6))]
            k, directed = 64, False
        elif args.workload == "rt22":
            n, s, d = synth.rmat_edges(22, 16, seed=1)
            variants = [("unit", None)]
            k, directed = 128, True
        else:
            n, s, d = synth.rmat_edges(12, 8, seed=1)
            variants = [("unit", None)]
            k, directed = 64, False
        results = []
        dev = torch.device("cuda", 0)
        for name, w in variants:
            g, _ = cc.cc_graph_from_edges(n, s, d, w, directed=directed)
            nn, arcs, _, _ = cc.cc_graph_info(g)
            m = arcs if directed else arcs // 2
            C = cc.cc_sample_choose(g, k, 2)
            o = cc.cc_opts_default(k)
            o.roundtrip = int(directed)
            # device outputs (every estimator's estimate and closeness), as
            # the headline line; the same call with host outputs is e2e
            outs = [torch.empty(nn, dtype=torch.float64, device=dev) for _ in range(8)]
            od = cc.cc_out()
            for e in range(4):
                od.s_hat[e], od.closeness[e] = outs[2 * e].data_ptr(), outs[2 * e + 1].data_ptr()
            o.device_outputs = 1
            o.stream = torch.cuda.current_stream().cuda_stream
            ms = _time_steps(lambda: cc.cc_estimate(g, C, o, od), args.steps, args.warmup, flush)
            tr = cc.cc_last_call_timing(g)
            ps = cc.cc_last_pass_stats(g)
            oh = cc.cc_opts_default(k)
            oh.roundtrip = int(directed)
            e2e_ms = _time_steps(lambda: cc.cc_estimate(g, C, oh), 1, 1, flush)
            units = k * m * (2 if directed else 1)
            r = {"weights": name, "n": nn, "m": m, "k": k, "ms_per_step": ms,
                 "value": units / (ms / 1e3) / 1e9,
                 "traversal_ms": tr[1], "kernel_launches": tr[0],
                 "levels_or_rounds": ps["levels"],
                 "e2e_ms_host_outputs": e2e_ms}
            if args.workload == "config1":
                t0 = time.perf_counter()
                cc.cc_exact(g)
                r["exact_all_pairs_s"] = time.perf_counter() - t0
            results.append(r)
            cc.cc_graph_free(g)
        line.update(value=results[0]["value"], ms_per_step=results[0]["ms_per_step"],
                    variants=results, config={"workload": args.workload})
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "rmat20":
        run_extra(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
