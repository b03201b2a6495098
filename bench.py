#!/usr/bin/env python
"""Benchmark of the GB300-native TIMEST hot path.

One step = one pass of the whole path over one synthetic input: load the
device-resident edge arrays, build the temporal CSR, compute the weights of
the motif's spanning tree (windows, DP, prefix sums, root CDF) and draw,
validate and count k samples.  `value` is samples per second of whole steps
(k / step time), timed with CUDA events on the library's stream; L2 is
flushed (a 512 MB write) before every timed step, outside its events.  The
default workload is the largest single-GPU one: a Chung-Lu graph of 5e7
edges, the 5-cycle with a chord, delta = 3,600 and k = 1e7.

Extra keys: per-phase times and launch counts from the library's event
timers, per-kernel live times (an event pair around every launch), the weight
pass's bandwidth against its byte model, a roofline object for the kernel
that leads the live per-kernel list, an end-to-end figure through the C ABI
with host buffers (pinned), and the CPU oracle timed on a bounded sample of
the same workload (a slice of its time span, scaled to a whole step).

`--impl reference` times the CPU oracle alone (the reference arm).
Under torchrun each rank samples its own range of sample ids on a replica of
the graph; the ranks' integer sums are combined by one all-reduce and checked
against a single-rank run of the same ids.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "cl50m_cycle5chord"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--k", type=int, default=0, help="override the sample count")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-ablation", action="store_true")
    ap.add_argument("--serve-queries", type=int, default=100)
    ap.add_argument("--serve-rate", type=float, default=50.0)
    ap.add_argument("--serve-workload", default="",
                    help="also serve the motif pool on this workload's graph (e.g. cl200m) in a fresh context")
    ap.add_argument("--serve-large-queries", type=int, default=300)
    ap.add_argument("--serve-large-rates", default="50",
                    help="comma-separated Poisson arrival rates (q/s) for --serve-workload")
    ap.add_argument("--serve-budget-frac", type=float, default=0.8,
                    help="weight budget for --serve-workload as a fraction of free device memory after the build")
    ap.add_argument("--alloc", choices=["native", "torch"], default="native",
                    help="device memory: the library's stream-ordered pool or PyTorch's caching allocator")
    ap.add_argument("--cpu-slice", type=float, default=0.1,
                    help="fraction of the time span the CPU baseline's oracle runs on (then scaled)")
    ap.add_argument("--ref-slice", type=float, default=0.02,
                    help="fraction of the time span of each reference-arm step")
    ap.add_argument("--ref-samples", type=int, default=200_000,
                    help="samples the oracle draws per reference-arm step (scaled to k)")
    return ap.parse_args()


# ---------------------------------------------------------------- clocks ----
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.gpu)], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


KERNEL_SOURCES = {
    "k_sample": ["sampler.cu", "tm_device.cuh", "tm_internal.h"],
    "k_dp": ["weights.cu", "tm_device.cuh", "tm_internal.h"],
    "k_gather2_pair": ["csr.cu", "tm_internal.h"],
    "k_gather2": ["csr.cu", "tm_internal.h"],
    "k_rs_scatter": ["csr.cu", "tm_internal.h"],
    "k_segscan2": ["scan.cuh", "weights.cu", "tm_device.cuh", "tm_internal.h"],
}


def kernel_source_hash(kernel):
    """sha256 over the sources that define a kernel (the files in order)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, []):
        with open(os.path.join(ROOT, "paper_2507_20441_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def profiled_traffic(kernel, workload):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum)
    from the committed ncu summary profiles/<kernel>_<workload>.md, or None
    when there is none or the kernel's sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if kernel not in KERNEL_SOURCES or not os.path.exists(path):
        return None
    fields = {}
    with open(path) as f:
        for line in f:
            line = line.strip().strip("`")
            for key in ("traffic_bytes_per_launch:", "source_sha256:"):
                if line.startswith(key):
                    fields[key[:-1]] = line[len(key):].strip()
    if fields.get("source_sha256") != kernel_source_hash(kernel):
        return None
    try:
        return int(fields["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


# ------------------------------------------------ algorithmic byte models ----
def dp_bytes_per_edge(plan_children):
    """Bytes one weight-DP launch must move per edge for a tree node with the
    given children (list of leaf flags), both layers: the edge record (t,
    src, dst, pair) and the reverse-pair id, read once; per layer and child
    the two list bounds (2 x 4 B offsets) and, for a non-leaf child, the four
    prefix values that bound the candidate range and its exclusion (4 x 8 B);
    per layer the 8 B weight written."""
    b = 16 + 4
    for _ in range(2):
        for leaf in plan_children:
            b += 8
            if not leaf:
                b += 32
        b += 8
    return b


def tree_children(order, parent):
    ntree = len(order)
    children = {q: [] for q in range(ntree)}
    for q in range(1, ntree):
        children[int(parent[q])].append(q)
    return children


def weight_pass_bytes_per_edge(children):
    """The weight pass's byte model per edge, both layers (the survey's
    per-layer formula for this tree): for each non-leaf node a 16 B edge
    record, 32 B of candidate- and exclusion-list bounds per child, 32 B of
    prefix reads per non-leaf child and an 8 B weight write; for each
    non-root, non-leaf node two prefix orders of (4 B map + 8 B read + 8 B
    write); for the root 8 B write + 8 B read + 8 B CDF write."""
    per_layer = 0
    for q, ch in children.items():
        if not ch:
            continue
        per_layer += 16 + 32 * len(ch) + 32 * sum(1 for c in ch if children[c]) + 8
    per_layer += sum(1 for q, ch in children.items() if q != 0 and ch) * 2 * (4 + 8 + 8)
    per_layer += 24
    return 2 * per_layer


def graph_stats(gr):
    """Edge-weighted mean list lengths of the workload graph: the out/in-list
    length and the multi-edge-list length seen from a uniformly random edge
    (sum of squares over sum)."""
    import numpy as np
    outd = np.bincount(gr.src, minlength=gr.n).astype(np.float64)
    ind = np.bincount(gr.dst, minlength=gr.n).astype(np.float64)
    key = gr.src.astype(np.uint64) * np.uint64(gr.n) + gr.dst.astype(np.uint64)
    _, sig = np.unique(key, return_counts=True)
    sig = sig.astype(np.float64)
    m = float(len(gr.src))
    return {"list_len": float(((outd ** 2).sum() + (ind ** 2).sum()) / (2 * m)),
            "pair_len": float((sig ** 2).sum() / m), "m": m}


def sampler_bytes_per_sample(ntree, nontree, stats, nwin):
    """The per-sample effective-bytes model of the sampler, every probe of
    every search counted at 8 B: the window search over the window totals
    (16 B entries) and the root search over the root CDF, 16 B for the root
    edge record; per non-root tree edge a 16 B record and five searches of the
    meeting vertex's list (two window bounds, two exclusion bounds, the
    inverse-CDF pick); per non-tree edge one search of its multi-edge list."""
    import math
    lg = lambda x: max(1, math.ceil(math.log2(max(x, 2.0))))
    b = lg(nwin) * 16 + lg(2 * stats["m"]) * 8 + 16
    b += (ntree - 1) * (16 + lg(stats["list_len"]) * 8 * 5)
    b += nontree * lg(stats["pair_len"]) * 8
    return b


def kernel_family(name):
    for fam in ("k_sample", "k_dp", "k_gather2_pair", "k_gather2", "k_rs_scatter", "k_segscan2"):
        if name.startswith(fam):
            return fam
    return name.split("<")[0]


def kernel_model(name, launches_per_step, ctx_m, k, children, per_sample):
    """Algorithmic bytes per launch of a kernel the live per-kernel list can
    put first, with the model's wording; None for a kernel without one."""
    fam = kernel_family(name)
    if fam == "k_sample":
        return k * per_sample, f"effective bytes (every search probe at 8 B): {per_sample} B/sample x k"
    if fam == "k_dp":
        per_step = sum(ctx_m * dp_bytes_per_edge([not children[c] for c in ch]) for ch in children.values() if ch)
        return per_step / max(launches_per_step, 1), \
            "streamed edge record, list bounds, prefix reads and weight writes per edge (averaged over the DP launches)"
    if fam == "k_gather2_pair":
        return 40 * ctx_m, "two sets x (4 B index + two 4 B gathered reads + two 4 B writes) per edge"
    if fam == "k_gather2":
        return 20 * ctx_m, "4 B index + two 4 B gathered reads + two 4 B writes per edge"
    return None, None


# ------------------------------------------------------- rank combining ----
def combine_across_ranks(res, device=None):
    """Sum the integer results of all ranks (disjoint sample-id ranges):
    hits2 (128-bit, as 16-bit limbs) and the four counters, one all-reduce.
    `res` has hits2, valid, rej_vertex, rej_delta, rej_order."""
    from paper_2507_20441_gb300.shard import all_reduce_counts
    return all_reduce_counts(res.hits2, res.valid, res.rej_vertex, res.rej_delta, res.rej_order, device=device)


def workload_config(args, gr, mo, k, tree, root):
    """The workload as both arms name it (identical dictionaries)."""
    return {"workload": args.workload, "n": int(gr.n), "m": int(gr.m), "motif": mo.name, "delta": int(mo.delta),
            "k": int(k), "tree": sorted(int(x) for x in tree), "root": int(root),
            "l2": "flushed (512 MB write) before every timed step", "alloc": args.alloc,
            "graph": "Chung-Lu bursty" if "cl" in args.workload else "uniform"}


# ------------------------------------------------------------------ ours ----
def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import paper_2507_20441_gb300 as tg
    from paper_2507_20441_gb300 import synth

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    gr = synth.make_graph(args.workload)
    mo = synth.make_motif(args.workload)
    k = args.k or mo.k
    tree, root = reference_tree(mo)
    stream = torch.cuda.Stream(device=dev)
    ctx = tg.Context(device=local_rank, stream=stream.cuda_stream, profile=2,
                     torch_allocator=(args.alloc == "torch"))
    src_d = torch.from_numpy(gr.src.view(np.int32)).to(dev)
    dst_d = torch.from_numpy(gr.dst.view(np.int32)).to(dev)
    t_d = torch.from_numpy(gr.t).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    torch.cuda.synchronize()

    state = {}

    def step(i, host=False):
        # rank r of N draws ids [(i N + r) k, (i N + r + 1) k): the ranks of one
        # step cover one contiguous range of N k sample ids
        first = (i * world + rank) * k
        if host:
            ctx.load_graph(gr.n, state["src_h"], state["dst_h"], state["t_h"], flags=tg.TM_HOST)
        else:
            ctx.load_graph(gr.n, src_d, dst_d, t_d, flags=tg.TM_DEVICE)
        m = ctx.motif(mo.nv, mo.edges, mo.rank, mo.delta)
        W = m.weights()
        res = m.sample(k, args.seed, first)
        if "plan" not in state:   # reporting metadata, read once (a warm-up step)
            state["plan"] = m.plan()
        state["W"] = W
        m.free()
        return res

    def timed(nsteps, host=False, base=0):
        times = []
        for i in range(nsteps):
            with torch.cuda.stream(stream):
                flush.fill_(i)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = step(base + i, host)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return times, res

    for i in range(args.warmup):
        step(10_000 + i)
    ctx.phase_times()
    ctx.kernel_times()
    ctx.io_bytes()
    clocks = ClockSampler(local_rank)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times, res = timed(args.steps)
    torch.cuda.synchronize()
    clk = clocks.stop()
    phases = ctx.phase_times()
    ktimes = ctx.kernel_times()
    ctx.io_bytes()
    my_ms = sum(times)
    if world > 1:
        t = torch.tensor([my_ms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.barrier()
        my_ms = float(t.item())
    ms_per_step = my_ms / args.steps
    value = world * k * args.steps / (my_ms / 1e3)
    # sub-phases ("csr.out") nest inside their phase: count top-level phases only
    launches = sum(n for name, (_, n) in phases.items() if "." not in name)

    # ---- the ranks' results of the last timed step combined (one all-reduce);
    # with N > 1 rank 0 checks them against one run over the same N k ids
    last = args.steps - 1
    hits2, valid, rv, rd, ro = combine_across_ranks(res, dev) if world > 1 else \
        (res.hits2, res.valid, res.rej_vertex, res.rej_delta, res.rej_order)
    combined = {"ranks": world, "samples": world * k, "first_id": last * world * k, "hits2": hits2, "valid": valid,
                "rej_vertex": rv, "rej_delta": rd, "rej_order": ro,
                "estimate": state["W"] * hits2 / (2.0 * world * k) if k else 0.0}
    if world > 1 and rank == 0:
        m = ctx.motif(mo.nv, mo.edges, mo.rank, mo.delta)
        m.weights()
        one = m.sample(world * k, args.seed, last * world * k)
        m.free()
        combined["equals_single_rank_run"] = (one.hits2, one.valid, one.rej_vertex, one.rej_delta,
                                              one.rej_order) == (hits2, valid, rv, rd, ro)
    ctx.phase_times()
    ctx.kernel_times()

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        state["src_h"] = torch.from_numpy(gr.src.view(np.int32)).pin_memory().numpy().view(np.uint32)
        state["dst_h"] = torch.from_numpy(gr.dst.view(np.int32)).pin_memory().numpy().view(np.uint32)
        state["t_h"] = torch.from_numpy(gr.t).pin_memory().numpy()
        for i in range(2):   # warm-up: first touches of the pinned buffers
            step(20_000 + i, host=True)
        ctx.phase_times(); ctx.io_bytes(); ctx.kernel_times()
        n_e2e = max(5, args.steps // 4)
        t_e2e, _ = timed(n_e2e, host=True, base=30_000)
        h2d, d2h = ctx.io_bytes()
        ph_e2e = ctx.phase_times()
        ctx.kernel_times()
        e2e = {"value": world * k * n_e2e / (sum(t_e2e) / 1e3), "unit": "samples/s",
               "h2d_bytes_per_step": h2d // n_e2e, "d2h_bytes_per_step": d2h // n_e2e,
               "ms_per_step": sum(t_e2e) / n_e2e,
               "phases_ms_per_step": {nm: round(v / n_e2e, 4) for nm, (v, _) in ph_e2e.items()
                                      if "." not in nm and v > 0}}

    # ---- roofline of the kernel that leads the live per-kernel list
    peak, peak_kind = measured_peaks()
    per = {name: (ms / args.steps, n / args.steps) for name, (ms, n) in phases.items() if n}
    order, parent = state["plan"]
    assert sorted(int(x) for x in order) == sorted(tree) and int(order[0]) == root, "default tree mismatch"
    ntree = len(order)
    children = tree_children(order, parent)
    m_edges = ctx.m
    gst = graph_stats(gr)
    nwin = 2 * (ctx.T // mo.delta + 1)
    per_sample = sampler_bytes_per_sample(ntree, len(mo.edges) - ntree, gst, nwin)
    kern = sorted(((name, ms / args.steps, n / args.steps) for name, (ms, n) in ktimes.items()),
                  key=lambda x: -x[1])
    top_name, top_ms, top_n = kern[0]
    algo, model = kernel_model(top_name, top_n, m_edges, k, children, per_sample)
    kern_ms = top_ms / max(top_n, 1)
    achieved = algo / (kern_ms / 1e3) / 1e9 if (algo and kern_ms > 0) else None
    roofline = {"bound": "hbm", "kernel": top_name, "achieved": round(achieved, 1) if achieved else None,
                "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                "frac": round(achieved / peak, 4) if achieved else None,
                "traffic": profiled_traffic(kernel_family(top_name), args.workload),
                "algorithmic_bytes_per_launch": int(algo) if algo else None, "model": model,
                "launch_ms": round(kern_ms, 4), "launches_per_step": top_n,
                "share_of_step": round(top_ms / ms_per_step, 4),
                "timing": "CUDA events around every launch on the library stream, timed steps"}
    step_kernels = [{"kernel": nm, "ms_per_step": round(ms, 4), "launches_per_step": n,
                     "share": round(ms / ms_per_step, 4)} for nm, ms, n in kern[:12]]

    # ---- weight pass against its byte model
    weight_ms = sum(per.get(p, (0.0, 0))[0] for p in ("windows", "dp", "prefix", "root"))
    wp_bytes = m_edges * weight_pass_bytes_per_edge(children)
    dp_bytes = sum(m_edges * dp_bytes_per_edge([not children[c] for c in ch]) for ch in children.values() if ch)
    dp_ms = per.get("dp", (0.0, 0))[0]
    wp_gbps = wp_bytes / (weight_ms / 1e3) / 1e9 if weight_ms else None
    weight_pass = {"ms": round(weight_ms, 4), "edges_per_s": m_edges / (weight_ms / 1e3) if weight_ms else None,
                   "model_bytes": int(wp_bytes), "model_bytes_per_edge": weight_pass_bytes_per_edge(children),
                   "GBps": round(wp_gbps, 1) if wp_gbps else None,
                   "frac_of_peak": round(wp_gbps / peak, 4) if wp_gbps else None,
                   "dp_GBps": round(dp_bytes / (dp_ms / 1e3) / 1e9, 1) if dp_ms else None,
                   "dp_frac_of_peak": round(dp_bytes / (dp_ms / 1e3) / 1e9 / peak, 4) if dp_ms else None,
                   "model": "windows + DP + prefix sums + root CDF; per layer: non-leaf nodes 16 B record + 32 B "
                            "bounds per child + 32 B prefix reads per non-leaf child + 8 B write; prefix nodes "
                            "2 x (4 + 8 + 8) B; root 24 B"}

    ablation = None if args.no_ablation else run_ablation(ctx, mo, k, args.seed, stream)
    batched = None if args.no_batch else run_batched(ctx, tg, synth, stream)
    served = None if args.no_serve else run_served(ctx, tg, synth, args.serve_queries, args.serve_rate,
                                                   compare_plain=True)

    out = {
        "metric": "samples/s", "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": workload_config(args, gr, mo, k, tree, root),
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": roofline,
        "kernels_per_step": step_kernels,
        "phases_ms_per_step": {k_: round(v[0], 4) for k_, v in per.items()},
        "weight_pass": weight_pass,
        "estimate": combined["estimate"], "W": state["W"], "hits2": hits2, "valid": valid,
        "combined": combined,
        "ablation": ablation,
        "batched": batched,
        "served": served,
    }
    ctx.close()
    if args.serve_workload:
        out["served_large"] = run_served_large(args, tg, synth, dev, stream)
    state["graph"] = gr
    return out, gr


# ------------------------------------------------------ batched / served ----
def run_batched(ctx, tg, synth, stream, reps=3):
    """32-query pool (3-7 vertices; delta in {600, 3600, 86400}; k log-uniform
    in [1e4, 1e7]) on the bench graph: one persistent batched launch against
    32 separate tm_sample calls, same weights and seeds; results must be
    identical.  Weights are computed once beforehand for both."""
    import torch
    pool = synth.motif_pool(seed=7, count=32)
    motifs = []
    for mo in pool:
        m = ctx.motif(mo.nv, mo.edges, mo.rank, mo.delta)
        m.weights()
        motifs.append(m)
    ks = [mo.k for mo in pool]
    seeds = [1000 + i for i in range(len(pool))]

    def timed(fn):
        best = None
        out = None
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        return best, out

    ms_plain, plain = timed(lambda: [m.sample(k, s) for m, k, s in zip(motifs, ks, seeds)])
    t0 = time.perf_counter()
    tuned, table = ctx.autotune(motifs, ks, seeds)      # picks tile / threads / record staging
    tune_s = time.perf_counter() - t0
    ms_batch, batch = timed(lambda: ctx.batch_run(motifs, ks, seeds))
    same = all((a.hits2, a.valid, a.rej_vertex, a.rej_delta, a.rej_order) ==
               (b.hits2, b.valid, b.rej_vertex, b.rej_delta, b.rej_order) for a, b in zip(plain, batch))
    ctx.phase_times()
    ctx.kernel_times()
    for m in motifs:
        m.free()
    return {"queries": len(pool), "samples": int(sum(ks)), "k_range": [int(min(ks)), int(max(ks))],
            "plain_ms": round(ms_plain, 3), "batched_ms": round(ms_batch, 3),
            "plain_qps": round(len(pool) / (ms_plain / 1e3), 1), "batched_qps": round(len(pool) / (ms_batch / 1e3), 1),
            "speedup": round(ms_plain / ms_batch, 3), "identical_results": bool(same),
            "autotuned_shape": {k_: tuned[k_] for k_ in tuned if k_ != "ms"},
            "autotune_s": round(tune_s, 3), "shapes_tried": len(table),
            "timing": "best of %d, CUDA events on the library stream, weights precomputed" % reps}


def run_ablation(ctx, mo, k, seed, stream):
    """The paper's constraint ablation on the bench workload: Constraint 1
    alone, 1+2 and 1+2+3 (the method), same motif, tree and k; per setting
    W, the invalid-sample rates by reason, the valid rate, the estimate and
    the weight-pass and sampler times (CUDA events)."""
    import torch
    out = {}
    for name, c2, c3 in (("C1", False, False), ("C1+2", True, False), ("C1+2+3", True, True)):
        m = ctx.motif(mo.nv, mo.edges, mo.rank, mo.delta).set_constraints(c2, c3)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        W = m.weights()
        e1.record(stream)
        r = m.sample(k, seed)
        e2.record(stream)
        e2.synchronize()
        out[name] = {"W": W, "valid_rate": r.valid / k, "invalid_vertex_map": r.rej_vertex / k,
                     "invalid_delta": r.rej_delta / k, "invalid_order": r.rej_order / k,
                     "estimate": r.estimate, "weights_ms": round(e0.elapsed_time(e1), 3),
                     "sample_ms": round(e1.elapsed_time(e2), 3)}
        m.free()
    ctx.phase_times()
    ctx.kernel_times()
    return out


def _pct(xs, p):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(p * (len(xs) - 1) + 0.5))] if xs else None


def run_plain_queries(ctx, pool, picks, arrivals, seeds):
    """The same arrival trace served the plain way: one query at a time in
    arrival order, each with its own weight pass (tm_weights) and one
    tm_sample launch; latency is arrival-to-result on the host clock."""
    t0 = time.perf_counter()
    lat, results = [], []
    for i, (q, a) in enumerate(zip(picks, arrivals)):
        now = time.perf_counter() - t0
        if a > now:
            time.sleep(a - now)
        mo = pool[int(q)]
        m = ctx.motif(mo.nv, mo.edges, mo.rank, mo.delta)
        m.weights()
        r = m.sample(mo.k, seeds[i])
        m.free()
        lat.append((time.perf_counter() - t0 - a) * 1e3)
        results.append(r)
    wall = time.perf_counter() - t0
    return results, {"p50_ms": round(_pct(lat, 0.5), 3), "p99_ms": round(_pct(lat, 0.99), 3),
                     "mean_ms": round(sum(lat) / len(lat), 3), "qps": round(len(lat) / wall, 2),
                     "wall_s": round(wall, 3)}


def run_served(ctx, tg, synth, nq, rate, weight_budget=0, compare_plain=False):
    """Poisson arrivals at `rate` queries/s drawn from the 32-motif pool (k
    log-uniform in [1e4, 1e7]), served by continuous batching with cached
    weights; latency is submit-to-result on the host clock.  With
    compare_plain the same trace is then run the plain way (one weight pass
    and one sampler launch per query, in arrival order) and both latency
    profiles and the share of identical results are reported."""
    import numpy as np
    pool = synth.motif_pool(seed=7, count=32)
    rng = np.random.default_rng(17)
    gaps = rng.exponential(1.0 / rate, size=nq)
    picks = rng.integers(0, len(pool), size=nq)
    arrivals = np.cumsum(gaps)
    seeds = [5000 + i for i in range(nq)]
    ctx.serve_start(max_active=64, weight_budget=weight_budget)
    tickets = []
    t0 = time.perf_counter()
    for i in range(nq):
        now = time.perf_counter() - t0
        if arrivals[i] > now:
            time.sleep(arrivals[i] - now)
        mo = pool[int(picks[i])]
        tickets.append(ctx.submit(mo.nv, mo.edges, mo.rank, mo.delta, mo.k, seeds[i]))
    served = []
    for t in tickets:
        r = ctx.poll(t, timeout_ms=600_000)
        assert r is not None
        served.append(r)
    wall = time.perf_counter() - t0
    st = ctx.serve_stats()
    ctx.serve_stop()
    out = {"queries": nq, "arrival_rate_qps": rate, "wall_s": round(wall, 3),
           "completed": st["completed"], "p50_ms": round(st["p50_ms"], 3), "p99_ms": round(st["p99_ms"], 3),
           "mean_ms": round(st["mean_ms"], 3), "qps": round(st["qps"], 2), "cache_hits": st["cache_hits"],
           "cache_misses": st["cache_misses"], "evictions": st["evictions"], "rounds": st["rounds"],
           "nomem_retries": st["nomem_retries"]}
    if compare_plain:
        plain, pst = run_plain_queries(ctx, pool, picks, arrivals, seeds)
        same = sum((a.W, a.hits2, a.valid, a.rej_vertex, a.rej_delta, a.rej_order) ==
                   (b.W, b.hits2, b.valid, b.rej_vertex, b.rej_delta, b.rej_order) for a, b in zip(served, plain))
        out["plain"] = pst
        out["identical_results"] = f"{same}/{nq}"
        out["p50_speedup_vs_plain"] = round(pst["p50_ms"] / out["p50_ms"], 3) if out["p50_ms"] else None
        out["p99_speedup_vs_plain"] = round(pst["p99_ms"] / out["p99_ms"], 3) if out["p99_ms"] else None
    ctx.phase_times()
    ctx.kernel_times()
    return out


def run_served_large(args, tg, synth, dev, stream):
    """The serving workload on its own graph: build the graph in a fresh
    context (the CSR build timed with CUDA events), then serve the pool at
    each requested arrival rate with a weight budget of a fraction of the
    device memory left after the build."""
    import numpy as np
    import torch
    t0 = time.perf_counter()
    gr = synth.make_graph(args.serve_workload)
    gen_s = time.perf_counter() - t0
    ctx = tg.Context(device=dev.index or 0, stream=stream.cuda_stream, torch_allocator=(args.alloc == "torch"))
    src_d = torch.from_numpy(gr.src.view(np.int32)).to(dev)
    dst_d = torch.from_numpy(gr.dst.view(np.int32)).to(dev)
    t_d = torch.from_numpy(gr.t).to(dev)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.load_graph(gr.n, src_d, dst_d, t_d, flags=tg.TM_DEVICE)
    e1.record(stream)
    e1.synchronize()
    build_ms = e0.elapsed_time(e1)
    del src_d, dst_d, t_d
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free, total = torch.cuda.mem_get_info(dev)
    budget = int(free * args.serve_budget_frac)
    runs = []
    for rate in [float(x) for x in args.serve_large_rates.split(",") if x]:
        r = run_served(ctx, tg, synth, args.serve_large_queries, rate, weight_budget=budget)
        runs.append(r)
    out = {"workload": args.serve_workload, "n": gr.n, "m": int(ctx.m), "generate_s": round(gen_s, 1),
           "build_ms": round(build_ms, 2), "weight_budget_bytes": budget,
           "free_bytes_after_build": int(free), "runs": runs}
    ctx.close()
    return out


# ------------------------------------------------------------- oracle ----
def oracle_slice_step(gr, mo, tree, root, k, frac, offset, k_sample, seed, threads):
    """One oracle step on a bounded sample of the workload: the edges whose
    time lies in [offset, offset + frac) of the span (a time slice keeps the
    per-window list lengths, the burstiness and every vertex of the full
    graph, since delta is far below the span).  The oracle's graph build and
    weight pass are timed in full on the slice and scaled by m / m_slice; its
    sampler draws k_sample samples with OpenMP, scaled to k."""
    import oracle
    t = gr.t
    t0, t1 = int(t.min()), int(t.max())
    span = t1 - t0 + 1
    if frac >= 1.0:
        src, dst, tt = gr.src, gr.dst, t
    else:
        lo = t0 + int(offset * span)
        hi = t0 + int(min(1.0, offset + frac) * span)
        sel = (t >= lo) & (t < hi)
        src, dst, tt = gr.src[sel], gr.dst[sel], t[sel]
    ms = len(src)
    a = time.perf_counter()
    G = oracle.Graph(gr.n, src, dst, tt)
    b = time.perf_counter()
    G.set_motif(mo.nv, mo.edges, mo.rank, mo.delta, sorted(tree), root)
    G.weights()
    c = time.perf_counter()
    ks = min(k, k_sample)
    G.sample(ks, seed, 0, threads=threads)
    d = time.perf_counter()
    G.close()
    scale = gr.m / max(ms, 1)
    step_s = ((b - a) + (c - b)) * scale + (d - c) * (k / max(ks, 1))
    return {"step_s": step_s, "m_slice": ms, "graph_s": b - a, "weights_s": c - b, "sample_s": d - c,
            "k_sample": ks, "scale": scale}


def slice_fraction(frac, m):
    """At least 1e6 edges (or the whole graph) per oracle slice."""
    return 1.0 if m <= 1_000_000 else min(1.0, max(frac, 1_000_000 / m))


def cpu_baseline(gr, mo, tree, root, k, frac, seed):
    threads = os.cpu_count() or 1
    frac = slice_fraction(frac, gr.m)
    r = oracle_slice_step(gr, mo, tree, root, k, frac, 0.0, 200_000, seed, threads)
    return {"value": k / r["step_s"], "unit": "samples/s", "cores": threads, "kind": "oracle",
            "sample": (f"edges in the first {frac:.0%} of the time span ({r['m_slice']} of {gr.m}): graph build "
                       f"and weights timed in full and scaled by m/m_slice = {r['scale']:.2f}; "
                       f"{r['k_sample']} samples (OpenMP) scaled to k = {k}"),
            "graph_s": round(r["graph_s"], 3), "weights_s": round(r["weights_s"], 3),
            "sample_s": round(r["sample_s"], 3), "step_s_scaled": round(r["step_s"], 3)}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle
    from paper_2507_20441_gb300 import synth
    oracle.build()
    gr = synth.make_graph(args.workload)
    mo = synth.make_motif(args.workload)
    k = args.k or mo.k
    tree, root = reference_tree(mo)
    threads = os.cpu_count() or 1
    frac = slice_fraction(args.ref_slice, gr.m)
    nslices = max(1, int(1.0 / frac))
    vals = []
    for i in range(args.warmup + args.steps):
        off = (i % nslices) * frac if frac < 1.0 else 0.0
        r = oracle_slice_step(gr, mo, tree, root, k, frac, off, args.ref_samples, args.seed + i, threads)
        if i >= args.warmup:
            vals.append(r)
    step_s = statistics.mean(v["step_s"] for v in vals)
    value = k / step_s
    sample = (f"per step the edges of one {frac:.0%} slice of the time span (about {vals[0]['m_slice']} of "
              f"{gr.m}; slices rotate over the span): oracle graph build and weights timed in full and scaled "
              f"by m/m_slice, {vals[0]['k_sample']} samples (OpenMP) scaled to k = {k}")
    return {"impl": "reference", "metric": "samples/s", "value": value, "unit": "samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": workload_config(args, gr, mo, k, tree, root),
            "cpu_baseline": {"kind": "oracle", "cores": threads, "value": value, "unit": "samples/s",
                             "sample": sample},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def reference_tree(mo):
    """Default spanning tree and root, computed on the host exactly as
    tm_set_motif documents: least looseness (pairs of tree edges at a
    vertex, |pi(e1)-pi(e2)|-1), lexicographically first, rooted at the edge
    of least eccentricity (ties: lower id)."""
    import itertools
    nv, edges, rank = mo.nv, mo.edges, mo.rank
    best = None
    for comb in itertools.combinations(range(len(edges)), nv - 1):
        comp = list(range(nv)); ok = True
        for e in comb:
            a, b = edges[e]; ca, cb = comp[a], comp[b]
            if ca == cb:
                ok = False; break
            comp = [ca if c == cb else c for c in comp]
        if not ok:
            continue
        L = 0
        for v in range(nv):
            inc = [e for e in comb if v in edges[e]]
            for i in range(len(inc)):
                for j in range(i + 1, len(inc)):
                    L += abs(rank[inc[i]] - rank[inc[j]]) - 1
        if best is None or L < best[0]:
            best = (L, list(comb))
    tree = best[1]

    def adj(x, y):
        return bool(set(edges[x]) & set(edges[y]))
    bestr = None
    for r in tree:
        dist = {r: 0}; frontier = [r]
        while frontier:
            nxt = []
            for x in frontier:
                for y in tree:
                    if y not in dist and adj(x, y):
                        dist[y] = dist[x] + 1; nxt.append(y)
            frontier = nxt
        ecc = max(dist.values())
        if bestr is None or ecc < bestr[0]:
            bestr = (ecc, r)
    return tree, bestr[1]


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    out, gr = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            import oracle
            from paper_2507_20441_gb300 import synth
            oracle.build()
            mo = synth.make_motif(args.workload)
            c = out["config"]
            out["cpu_baseline"] = cpu_baseline(gr, mo, c["tree"], c["root"], c["k"], args.cpu_slice, args.seed)
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
