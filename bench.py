#!/usr/bin/env python
"""Throughput of exact k-bisimulation refinement on one GB300.

Workload: the power-law graph with 10M vertices and 100M edges (out-degree
exponent 2.1 capped at 1M, targets preferential by in-degree, 1000 Zipf edge
labels, 200 Zipf vertex labels, 10% untyped), refined to the fixpoint with a
cap of 10 rounds. One step is one pass of the whole path over that graph:
summarize_init_coo (CSR build by radix sort, label partition), bisim_iterate
(refinement rounds until the block count stops changing, at most 10) and
get_partition, through the C-ABI.

  value  = edges x rounds executed / step time, COO already resident in HBM
  e2e    = the same metric with the COO and labels in pinned host memory and
           the partition copied back to pinned host memory inside the timed
           region, two requests in flight (one request at a time beside it)
  roofline = the kernel with the largest event-timed share of the timed steps:
           its algorithmic bytes / its summed launch time, against the measured
           HBM copy bandwidth

  rounds_roofline = per refinement round: the algorithmic bytes of the rows and
           vertices that round processed (12 B per row entry + 44 B per listed
           vertex, counted on the device) over the round's event time
  cpu_baseline = the oracle (exact signatures in an ordered map) on the same
           graph: one thread on a range of the vertices, and the same round
           on all host cores

--impl reference times the CPU oracle on the same graph: each step is one
exact refinement round over the next 1/K of the vertices, so K steps cover one
whole round. --gpus N > 1 runs N independent replicas (the refinement of one
graph has no sharded form here), one per rank.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "k-bisim edge-iterations/sec (1 GB300, bit-exact); update-batch p50/p99 latency"
UNIT = "edge-iterations/s"
WORKLOAD = dict(n=10_000_000, m=100_000_000, exponent=2.1, dmax=1_000_000, n_elabels=1000, n_vlabels=200,
                untyped=0.1, k="fixpoint", cap=10, seed=2)
# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per unit of work of the
# kernels that can be the dominant one, each from one ncu --set full capture of one launch
# on the generator's 3M-vertex / 30M-edge instance (bench.py --scale 0.3, inputs larger
# than L2); a launch's traffic is this times the units it processed. Entries are removed
# when their kernel changes.
NCU_TRAFFIC_PER_UNIT = {
    # k_place_sorted: 420.1 MB read + 205.7 MB written for 30M edges (algorithmic 24 B per edge)
    "csr_place": ((420.07e6 + 205.74e6) / 30e6, "edges"),
    # k_dense_verify, round 1 (all 3M positions listed): 214.7 MB read + 18.3 MB written
    # (algorithmic 20 B per listed vertex); later rounds list scattered positions, whose
    # sectors serve fewer bytes, so this is a lower bound for them
    "dense_verify": ((214.7e6 + 18.3e6) / 3e6, "vertices"),
    # k_dense_insert, round 1: 145.1 MB read + 30.0 MB written (algorithmic 24 B per vertex)
    "dense_insert": ((145.1e6 + 30.0e6) / 3e6, "vertices"),
}
# Per-round algorithmic bytes of a refinement round (the row entries and vertices it processed).
ROUND_EDGE_BYTES = 12.0     # packed (label, target) word 8 + gathered block id 4
ROUND_VERTEX_BYTES = 44.0   # row offset 4 + own block 4 + new block written 4 + two 16-byte table accesses
SIG_SITES = ("dense_thread_sig_8", "dense_thread_sig_16", "dense_thread_sig_32", "dense_warp_sig",
             "dense_mid_512", "dense_mid_1024", "dense_mid_2048", "dense_mid_4096", "dense_mid_8192",
             "hub_insert", "dense_hub_finalize")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=float, default=1.0, help="shrink the workload (smoke runs only)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the update-batch latency section")
    ap.add_argument("--serving-batches", type=int, default=40)
    ap.add_argument("--no-autotune", action="store_true", help="keep the default class thresholds")
    ap.add_argument("--profile-updates", type=int, default=0, metavar="K",
                    help="profiler capture window only: run the 1k-op update batches of the serving section "
                         "alone and bracket K incremental batches (after eight) with cudaProfilerStart/Stop, "
                         "for ncu --profile-from-start off; prints the batches' latencies, not a bench line")
    ap.add_argument("--literal-alg4", action="store_true",
                    help="diagnostic only: on each of the five configurations, the partition of Algorithm 4 taken "
                         "literally (no edge labels in its last round) against the definition's; prints one JSON "
                         "line per configuration, not a bench line")
    ap.add_argument("--union-rounds", action="store_true",
                    help="batched workload: run the union through the single-graph round kernels instead of the "
                         "persistent per-graph kernel")
    ap.add_argument("--batch-split", type=int, default=None, metavar="V",
                    help="batched workload: graphs of at most V vertices go to the persistent kernel (default: "
                         "the library's, or the autotuner's choice)")
    ap.add_argument("--workload", default="powerlaw", choices=["powerlaw", "chain", "paths", "batched"],
                    help="powerlaw: 10M/100M to the fixpoint (the headline); chain: 1000 paths of 1000 "
                         "+ 2M random edges to the fixpoint; paths: 1000 paths of 1000 with one vertex and one "
                         "edge label (999 rounds, every vertex listed in each); batched: 4096 graphs in one "
                         "context, k=3")
    return ap.parse_args()


def workload_graph(scale):
    from paper_2111_12493_gb300 import graphgen
    n = max(1000, int(WORKLOAD["n"] * scale))
    m = max(10_000, int(WORKLOAD["m"] * scale))
    return graphgen.powerlaw_graph(n=n, m=m, exponent=WORKLOAD["exponent"], dmax=min(WORKLOAD["dmax"], m // 10),
                                   n_elabels=WORKLOAD["n_elabels"], n_vlabels=WORKLOAD["n_vlabels"],
                                   untyped_frac=WORKLOAD["untyped"], seed=WORKLOAD["seed"])


class Workload:
    """Inputs, one step of the path and its accounting for one benchmark configuration."""

    def __init__(self, name, scale):
        from paper_2111_12493_gb300 import graphgen
        self.name = name
        self.batched = name == "batched"
        if name == "powerlaw":
            g = workload_graph(scale)
            self.k, self.cap = -1, WORKLOAD["cap"]
            self.arrays = [g[k] for k in ("src", "dst", "elabel", "vlabel")]
            self.graph = g
        elif name == "chain":
            paths = max(10, int(1000 * scale))
            g = graphgen.chain_graph(n_paths=paths, path_len=1000, extra=int(2_000_000 * scale), seed=3)
            self.k, self.cap = -1, 10_000
            self.arrays = [g[k] for k in ("src", "dst", "elabel", "vlabel")]
            self.graph = g
        elif name == "paths":
            paths = max(10, int(1000 * scale))
            g = graphgen.chain_graph(n_paths=paths, path_len=1000, extra=0, n_elabels=1, n_vlabels=1, seed=3)
            self.k, self.cap = -1, 10_000
            self.arrays = [g[k] for k in ("src", "dst", "elabel", "vlabel")]
            self.graph = g
        else:
            b = graphgen.batched_graphs(n_graphs=max(8, int(4096 * scale)), seed=4)
            self.k, self.cap = 3, 0
            self.arrays = [b["vertex_offsets"], b["edge_offsets"], b["src_local"], b["dst_local"], b["elabel"],
                           b["vlabel"]]
            self.graph = b
        self.n = int(self.arrays[-1].shape[0])
        self.m = int(self.arrays[-4 if self.batched else 0].shape[0])

    def config(self, extra=None):
        g = self.graph
        if self.name == "powerlaw":
            return config_dict(self.n, self.m, g, extra)
        if self.name == "chain":
            d = {"workload": f"{self.n // 1000:,} directed paths of 1000 vertices (path-major ids) + "
                             f"{self.m - (self.n // 1000) * 999:,} uniform extra edges, 16 uniform edge labels, "
                             f"2 vertex labels; refine to the fixpoint (cap 10000)",
                 "n_vertices": self.n, "n_edges": self.m, "k": "fixpoint", "cap": 10_000,
                 "l2": "inputs smaller than L2 (36 MB COO): a latency-bound many-round workload"}
        elif self.name == "paths":
            d = {"workload": f"{self.n // 1000:,} directed paths of 1000 vertices (path-major ids), one vertex "
                             f"label and one edge label; refine to the fixpoint (cap 10000): every round splits "
                             f"one vertex off each path and every vertex stays listed, 999 rounds (the long "
                             f"k-chaining regime; a supplement to the chains configuration, whose random extra "
                             f"edges separate the paths by round 4)",
                 "n_vertices": self.n, "n_edges": self.m, "k": "fixpoint", "cap": 10_000,
                 "l2": "inputs smaller than L2 (12 MB COO): a latency-bound many-round workload"}
        else:
            ng = np.diff(g["vertex_offsets"])
            d = {"workload": f"{g['n_graphs']:,} independent graphs in one context, vertex counts log-uniform "
                             f"[100, 100k] (realised {int(ng.min()):,}-{int(ng.max()):,}), power-law out-degree "
                             f"(2.3) with mean 5, uniform in-graph targets, 64 Zipf(1.1) edge labels, 16 vertex "
                             f"labels; k=3",
                 "n_graphs": int(g["n_graphs"]), "n_vertices": self.n, "n_edges": self.m, "k": 3,
                 "round_path": "union through the single-graph round kernels" if self.union_rounds else
                           "graphs up to batch_split vertices: one persistent kernel, a CTA per graph from a "
                           "largest-first queue; larger graphs: the union's round kernels on the same GPU at "
                           "the same time",
                 "l2": "inputs larger than L2"}
        if extra:
            d.update(extra)
        return d

    options = None
    union_rounds = False

    def step(self, bisim, tensors, out):
        ctx = self.init_only(bisim, tensors)
        rounds, blocks = bisim.bisim_iterate(ctx, self.k, self.cap)
        bisim.get_partition(ctx, out=out)
        executed = bisim.bisim_get_stats(ctx)["rounds_executed"]
        bisim.summarize_destroy(ctx)
        return rounds, blocks, executed

    def init_only(self, bisim, tensors):
        if self.batched:
            return bisim.summarize_init_batched(*tensors, options=self.options)
        return bisim.summarize_init_coo(self.n, *tensors, options=self.options)


def config_dict(n, m, g=None, extra=None):
    d = {"workload": f"power-law digraph {n:,} vertices / {m:,} edges, out-degree exponent 2.1 (max 1M), "
                     f"copy-model targets, 1000 Zipf(1.1) edge labels, 200 Zipf(1.0) vertex labels + 10% untyped; "
                     f"refine to the fixpoint, cap 10 rounds",
         "n_vertices": int(n), "n_edges": int(m), "k": "fixpoint", "cap": 10,
         "l2": "inputs larger than L2 (COO 1.2 GB, CSR 0.8 GB)"}
    if g is not None:
        d["max_out_degree"] = int(np.bincount(g["src"], minlength=g["n"]).max())
        d["max_in_degree"] = int(np.bincount(g["dst"], minlength=g["n"]).max())
    if extra:
        d.update(extra)
    return d


# ----------------------------------------------------------------------------- distributed plumbing

def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, x):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------- end to end

def e2e_run(bisim, torch, W, h_in, steps, slots, local, world):
    """`steps` requests from host buffers, `slots` of them in flight at a time
    (request i on host thread i mod slots, each thread with its own stream and
    pinned output). summarize_init_coo copies the edge arrays of different
    contexts one after the other, so one request's upload overlaps the other's
    build, refinement and download. Returns (edge-iterations, the timed
    region in ms, outputs)."""
    import threading
    torch.cuda.set_device(local)
    streams = [torch.cuda.Stream() for _ in range(slots)]
    outs = [torch.empty(W.n, dtype=torch.int32).pin_memory() for _ in range(slots)]
    done = [0] * slots
    errors = []

    def worker(t, count):
        try:
            torch.cuda.set_device(local)
            with torch.cuda.stream(streams[t]):
                for _ in range(count):
                    _, _, ex = W.step(bisim, h_in, outs[t])
                    streams[t].synchronize()     # the partition is in host memory now
                    done[t] += W.m * ex
        except BaseException as e:  # noqa: BLE001 - re-raised below
            errors.append(e)

    def run(total):
        threads = [threading.Thread(target=worker, args=(t, len(range(t, total, slots)))) for t in range(slots)]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        if errors:
            raise errors[0]

    run(slots)                                   # warm-up: one request per slot
    torch.cuda.synchronize()
    done[:] = [0] * slots
    barrier(world)
    t0 = time.perf_counter()
    run(steps)
    torch.cuda.synchronize()
    wall_ms = (time.perf_counter() - t0) * 1e3
    return sum(done), max_over_ranks(world, wall_ms), outs



# ----------------------------------------------------------------------------- per-round roofline

def _iterate_ms(bisim, torch, ctx, k, stream, reps=3):
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bisim.bisim_iterate(ctx, k, 0)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1)
        best = t if best is None else min(best, t)
    return best


def _round_work(bisim, ctx, k):
    """Listed vertices and row entries processed by k rounds from P_0 (device-counted)."""
    bisim.bisim_profile_reset()
    bisim.bisim_profile_enable(True)
    bisim.bisim_iterate(ctx, k, 0)
    bisim.bisim_profile_enable(False)
    prof = {p["name"]: p for p in bisim.bisim_profile_read()}
    listed = prof.get("dense_verify", {}).get("vertices", 0)
    entries = sum(prof.get(n, {}).get("edges", 0) for n in SIG_SITES)
    return listed, entries


def rounds_roofline(bisim, torch, W, d_in, stream, peak, executed):
    """Per round i: survey bytes of the rows and vertices it processed / its event time.

    Round i's time is T(i) - T(i-1), T(k) the best event time of bisim_iterate(k)
    on a resident context (captured device-side loop); its work is counted on the
    device in an eager profiled run of the same k. Workloads with many rounds
    report rounds 1-3 and the mean of the rest."""
    ctx = W.init_only(bisim, d_in)
    bisim.bisim_iterate(ctx, W.k, W.cap)            # captures the round graph
    ks = list(range(0, executed + 1)) if executed <= 12 else [0, 1, 2, 3, executed]
    T = {k: _iterate_ms(bisim, torch, ctx, k, stream) for k in ks}
    work = {0: (0, 0)}
    for k in ks[1:]:
        work[k] = _round_work(bisim, ctx, k)
    bisim.summarize_destroy(ctx)
    out = []
    for a, b in zip(ks[:-1], ks[1:]):
        ms = T[b] - T[a]
        listed = work[b][0] - work[a][0]
        entries = work[b][1] - work[a][1]
        byts = ROUND_EDGE_BYTES * entries + ROUND_VERTEX_BYTES * listed
        gbs = byts / (ms / 1e3) / 1e9 if ms > 0 else None
        out.append({"rounds": f"{a + 1}" if b == a + 1 else f"{a + 1}-{b} (mean)", "ms": round(ms / (b - a), 4),
                    "listed_vertices": int(listed / (b - a)), "row_entries": int(entries / (b - a)),
                    "alg_bytes": byts / (b - a), "GB/s": round(gbs, 1) if gbs else None,
                    "frac": round(gbs / peak, 4) if gbs else None})
    plain = ROUND_EDGE_BYTES * W.m + ROUND_VERTEX_BYTES * W.n
    total_ms = T[ks[-1]] - T[0]
    return {"per_round": out, "unit": "GB/s", "peak": peak,
            "bytes_formula": "12 B per row entry processed + 44 B per listed vertex (counted on the device)",
            "plain_round_effective": {
                "GB/s": round(plain * executed / (total_ms / 1e3) / 1e9, 1),
                "note": "every executed round credited with a plain round's bytes (12 B per edge + 44 B per "
                        "vertex), although rounds after the first skip the vertices alone in their block: an "
                        "effective rate, not achieved bandwidth"}}


# ----------------------------------------------------------------------------- our arm

def run_ours(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    from paper_2111_12493_gb300 import bisim

    W = Workload(args.workload, args.scale)
    W.union_rounds = bool(args.union_rounds)
    g = W.graph
    n, m = W.n, W.m
    dev = torch.device("cuda", local)
    d_in = [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in W.arrays]
    d_out = torch.empty(n, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step(*tensors):
        return W.step(bisim, tensors[:-1], tensors[-1])

    tuned = None
    if not args.no_autotune:
        # class thresholds and hub chunk timed on this graph, once, before the warm-up
        ctx = W.init_only(bisim, d_in)
        tuned = bisim.bisim_autotune(ctx, rounds=2)
        bisim.summarize_destroy(ctx)
        W.options = bisim.default_options(**{k: tuned[k] for k in ("small_max_degree", "mid_max_degree",
                                                                   "hub_chunk", "batch_split")})
    if W.batched and args.batch_split is not None:
        W.options = W.options or bisim.default_options()
        W.options.batch_split = args.batch_split

    if W.batched and args.union_rounds:
        W.options = W.options or bisim.default_options()
        W.options.flags |= bisim.FLAG_UNION_ROUNDS

    for _ in range(args.warmup):
        rounds, blocks, executed = step(*d_in, d_out)
    torch.cuda.synchronize()

    # timed region: K steps, inputs resident in HBM
    clocks = ClockSampler(local)
    launches0 = bisim.bisim_launch_count()
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    edge_iters = 0
    for _ in range(args.steps):
        rounds, blocks, executed = step(*d_in, d_out)
        edge_iters += m * executed
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clock_info = clocks.stop()
    launches = bisim.bisim_launch_count() - launches0
    t_ms = max_over_ranks(world, ev0.elapsed_time(ev1))
    total_edge_iters = sum_over_ranks(world, edge_iters)
    value = total_edge_iters / (t_ms / 1e3)

    # the same steps with every launch timed by CUDA events on its stream (the
    # rounds then run as host-driven launch sequences instead of the graph)
    bisim.bisim_profile_reset()
    bisim.bisim_profile_enable(True)
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        step(*d_in, d_out)
    p1.record(stream)
    torch.cuda.synchronize()
    bisim.bisim_profile_enable(False)
    prof = bisim.bisim_profile_read()
    profiled_ms = p0.elapsed_time(p1)

    # rounds only, on a resident context (the first call also captures the round graph)
    ctx = W.init_only(bisim, d_in)
    bisim.bisim_iterate(ctx, W.k, W.cap)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r2, _ = bisim.bisim_iterate(ctx, W.k, W.cap)
    e1.record(stream)
    torch.cuda.synchronize()
    it_exec = bisim.bisim_get_stats(ctx)["rounds_executed"]
    iterate_only = m * it_exec / (e0.elapsed_time(e1) / 1e3)
    stats = bisim.bisim_get_stats(ctx)
    bisim.summarize_destroy(ctx)

    # sanity of the result that was timed: canonical ids (block id = its smallest member)
    P = d_out.cpu().numpy()
    if W.batched:   # graph-local ids: the block id is the smallest local id in the block
        local = np.arange(n) - np.repeat(g["vertex_offsets"][:-1], np.diff(g["vertex_offsets"]))
        glob = P + (np.arange(n) - local)
        assert (P >= 0).all() and (P <= local).all() and (glob[glob] == glob).all(), "non-canonical partition"
    else:
        assert (P >= 0).all() and (P <= np.arange(n)).all() and (P[P] == P).all(), "non-canonical partition"
        assert len(np.unique(P)) == blocks

    # end to end through the C-ABI with host buffers: one request at a time, and
    # two in flight (each on its own host thread and stream, as the request
    # loop runs them), so that one request's upload overlaps the other's rounds
    e2e = None
    if not args.no_e2e:
        h_in = [torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in W.arrays]
        runs = {}
        for slots in (1, 2):
            ei, e_ms, outs = e2e_run(bisim, torch, W, h_in, args.steps, slots, local, world)
            for o in outs:
                assert np.array_equal(o.numpy(), P), "host-buffer run differs from the device run"
            runs[slots] = sum_over_ranks(world, ei) / (e_ms / 1e3)
        e2e = {"value": runs[2], "unit": UNIT,
               "h2d_bytes_per_step": int(sum(t.numel() * t.element_size() for t in h_in)),
               "d2h_bytes_per_step": int(4 * n), "requests_in_flight": 2,
               "one_at_a_time": {"value": runs[1], "unit": UNIT},
               "note": "each step is one request through the public calls (summarize_init_coo from pinned host "
                       "COO and labels, bisim_iterate, get_partition into pinned host memory, summarize_destroy); "
                       "every step's uploads and its partition's download are inside the timed region; with two "
                       "requests in flight the library copies their edge arrays one after the other and one "
                       "request's upload overlaps the other's build, refinement and download"}

    # roofline of the dominant kernel (largest event-timed share of the timed steps)
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    total_kernel_ms = sum(p["total_ms"] for p in prof)
    top = max(prof, key=lambda p: p["total_ms"]) if prof else None
    roofline = None
    kernels = None
    if top and top["total_ms"] > 0:
        achieved = top["alg_bytes"] / (top["total_ms"] / 1e3) / 1e9
        per_unit = NCU_TRAFFIC_PER_UNIT.get(top["name"]) if W.name == "powerlaw" else None
        traffic = None
        if per_unit is not None:
            units = top.get(per_unit[1], 0) / max(1, top["launches"])
            traffic = per_unit[0] * units if units > 0 else None
        roofline = {"bound": "hbm", "kernel": top["name"], "achieved": round(achieved, 1), "peak": peak,
                    "unit": "GB/s", "frac": round(achieved / peak, 4), "peak_source": peak_src,
                    "traffic": traffic, "alg_bytes_per_launch": top["alg_bytes"] / max(1, top["launches"]),
                    "avg_launch_ms": top["total_ms"] / max(1, top["launches"]),
                    "share_of_kernel_time": round(top["total_ms"] / total_kernel_ms, 4)}
        if traffic is not None:
            roofline["traffic_vs_alg"] = round(traffic / roofline["alg_bytes_per_launch"], 3)
            unit1 = {"vertices": "listed vertex", "edges": "edge"}[per_unit[1]]
            roofline["traffic_note"] = (f"ncu DRAM bytes per {unit1} of one launch on the 30M-edge "
                                        f"instance ({per_unit[0]:.1f} B) x the {per_unit[1]} an average launch "
                                        f"processed here")
        kernels = sorted(({"name": p["name"], "launches": p["launches"], "ms": round(p["total_ms"], 3),
                           "share": round(p["total_ms"] / total_kernel_ms, 4),
                           "GB/s": round(p["alg_bytes"] / (p["total_ms"] / 1e3) / 1e9, 1) if p["total_ms"] else None}
                          for p in prof if p["launches"]), key=lambda x: -x["ms"])[:12]

    rr = None
    if not W.batched:
        rr = rounds_roofline(bisim, torch, W, d_in, stream, peak, int(it_exec))

    serving_info = None
    if not args.no_serving and W.name == "powerlaw":
        serving_info = run_serving(args, local)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(W)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32 ids, u64 hashes (integer only)",
            "data": "synthetic (seeded generator; stands in for the paper's BSBM/DyLDO graphs)",
            "config": W.config({"parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                                "rounds": int(rounds), "rounds_executed": int(executed), "blocks": int(blocks),
                                "edge_iterations": f"edges x rounds_executed ({int(executed)}) per step; r = "
                                                   f"{int(rounds)} is the result, the round after it confirms "
                                                   f"the fixpoint and is counted because it runs",
                                "autotuned": None if tuned is None else
                                {k: tuned[k] for k in ("small_max_degree", "mid_max_degree", "hub_chunk")
                                 + (("batch_split",) if W.batched else ())},
                                **({"batch_split": int(W.options.batch_split) if W.options else None}
                                   if W.batched else {})}),
            "iterate_only": {"value": iterate_only, "unit": UNIT, "rounds_executed": int(it_exec),
                             "note": "bisim_iterate alone on a resident context (round graph already captured)"},
            "profiled_steps": {"ms_per_step": profiled_ms / args.steps,
                               "note": "the timed steps again with per-launch CUDA events (rounds run eagerly); "
                                       "kernels and roofline come from these"},
            "e2e": e2e, "roofline": roofline, "rounds_roofline": rr, "kernels": kernels, "cpu_baseline": cpu,
            "gpu_launches": int(launches), "clocks": clock_info,
            "buckets": {"small": stats["n_small"], "mid": stats["n_mid"], "hub": stats["n_hub"]},
            "collision_levels": stats["collision_levels"], "serving": serving_info}
    if rank == 0:
        print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- update-batch latency

SERVING = dict(n=5_000_000, m=50_000_000, k=2, rate_hz=200.0, min_ops=1000, max_ops=1_000_000, seed=5)


def _pct(xs, q):
    return float(np.percentile(np.asarray(xs) * 1e3, q)) if len(xs) else None


def run_serving(args, local):
    """Resident 5M/50M graph at k=2 under update batches: incremental vs full recompute.

    closed loop: fixed 1k-op batches, each applied and its partition read back
    before the next; latency = apply_updates + get_partition, ops staged from
    pinned host memory inside the timed call. Full recompute = the same batch
    applied to a second resident context that recomputes all k rounds over the
    whole edited graph (BISIM_FLAG_FULL_RECOMPUTE).
    open loop: batches of log-uniform size in [1k, 1M] ops arriving as a
    Poisson process at 200/s, submitted to the request loop as they arrive;
    latency = result time - arrival time (queueing included).
    """
    import torch
    from paper_2111_12493_gb300 import bisim, graphgen, serving
    n = max(1000, int(SERVING["n"] * args.scale))
    m = max(10_000, int(SERVING["m"] * args.scale))
    g = graphgen.powerlaw_graph(n=n, m=m, exponent=WORKLOAD["exponent"], dmax=min(WORKLOAD["dmax"], m // 10),
                                n_elabels=WORKLOAD["n_elabels"], n_vlabels=WORKLOAD["n_vlabels"],
                                untyped_frac=WORKLOAD["untyped"], seed=SERVING["seed"])
    dev = torch.device("cuda", local)
    d = {k: torch.from_numpy(g[k]).to(dev) for k in ("src", "dst", "elabel", "vlabel")}
    empty = torch.zeros((0, 4), dtype=torch.int32, device=dev)
    out = {"workload": f"power-law digraph {n:,} vertices / {m:,} edges (generator as above), k=2 maintained "
                       f"under update batches of 70% edge adds / 25% edge deletes / 5% vertex deletes"}

    def ctx_for(flags):
        c = bisim.summarize_init_coo(n, d["src"], d["dst"], d["elabel"], d["vlabel"],
                                     options=bisim.default_options(k_incremental=SERVING["k"], flags=flags))
        bisim.apply_updates(c, empty)
        return c

    # closed loop, 1k-op batches
    fixed = graphgen.update_batches(g, 33, fixed_size=1000, seed=51)
    pinned = [torch.from_numpy(b["ops"]).pin_memory() for b in fixed]
    res = {}
    for mode, flags in (("incremental", 0), ("full_recompute", bisim.FLAG_FULL_RECOMPUTE)):
        ctx = ctx_for(flags)
        part = torch.empty(n, dtype=torch.int32, device=dev)
        lat, fr = [], []
        for i, ops in enumerate(pinned):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bisim.apply_updates(ctx, ops)
            bisim.get_partition(ctx, out=part)
            torch.cuda.synchronize()
            if i >= 3:                          # the first three batches are warm-up
                lat.append(time.perf_counter() - t0)
                fr.append(bisim.bisim_get_stats(ctx)["last_frontier"])
        res[mode] = dict(p50_ms=_pct(lat, 50), p99_ms=_pct(lat, 99), batches=len(lat),
                         mean_frontier=float(np.mean(fr)))
        res[mode + "_P"] = part.cpu().numpy()
        bisim.summarize_destroy(ctx)
    same = bool(np.array_equal(res.pop("incremental_P"), res.pop("full_recompute_P")))
    out["batch_1k"] = dict(res, identical_partitions=same,
                           p99_speedup=res["full_recompute"]["p99_ms"] / res["incremental"]["p99_ms"])

    out["overlap"] = serving_overlap(torch, serving, graphgen, args.scale)

    # open loop through the request loop, log-uniform sizes, Poisson arrivals
    batches = graphgen.update_batches(g, args.serving_batches, min_ops=SERVING["min_ops"],
                                      max_ops=int(SERVING["max_ops"] * min(1.0, args.scale)),
                                      rate_hz=SERVING["rate_hz"], seed=52)
    pinned = [torch.from_numpy(b["ops"]).pin_memory() for b in batches]
    srv = serving.Server(slots=2)
    srv.summarize("g", n, d["src"], d["dst"], d["elabel"], d["vlabel"], k=SERVING["k"], keep=True,
                  k_incremental=SERVING["k"]).result()
    futs = []
    t_start = time.perf_counter()
    for b, ops in zip(batches, pinned):
        wait = t_start + b["arrival_s"] - time.perf_counter()
        if wait > 0:
            time.sleep(wait)
        futs.append(srv.update("g", ops))
    for f in futs:
        f.result()
    span = time.perf_counter() - t_start
    reqs = [r for r in srv.scheduler.completed if r.kind == "update"]
    srv.close()
    lat = [r.finished - r.arrival for r in reqs]
    svc = [r.finished - r.started for r in reqs]
    n_ops = int(sum(len(b["ops"]) for b in batches))
    # the same batches as full recomputes (service time only)
    ctx = ctx_for(bisim.FLAG_FULL_RECOMPUTE)
    part = torch.empty(n, dtype=torch.int32, device=dev)
    full = []
    for ops in pinned:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bisim.apply_updates(ctx, ops)
        bisim.get_partition(ctx, out=part)
        torch.cuda.synchronize()
        full.append(time.perf_counter() - t0)
    bisim.summarize_destroy(ctx)
    out["open_loop"] = dict(batches=len(reqs), ops=n_ops, sizes="log-uniform [1k, 1M] ops",
                            arrival_rate_hz=SERVING["rate_hz"], wall_s=span,
                            latency_p50_ms=_pct(lat, 50), latency_p99_ms=_pct(lat, 99),
                            service_p50_ms=_pct(svc, 50), service_p99_ms=_pct(svc, 99),
                            full_recompute_service_p50_ms=_pct(full, 50),
                            full_recompute_service_p99_ms=_pct(full, 99),
                            utilisation=sum(svc) / span)
    return out


def serving_overlap(torch, serving, graphgen, scale):
    """Two independent summarizations (400k / 4M power-law graphs) on two
    slots of the request loop's executor: each alone, then both at once from
    two threads. Device spans from CUDA events on each slot's stream."""
    import threading
    n, m = max(1000, int(400_000 * scale)), max(10_000, int(4_000_000 * scale))
    gs = [graphgen.powerlaw_graph(n=n, m=m, dmax=max(100, m // 100), n_elabels=100, n_vlabels=20, seed=s)
          for s in (25, 26)]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    reqs = [serving.Request("summarize", i, dict(n=g["n"], src=t(g["src"]), dst=t(g["dst"]), edge_label=t(g["elabel"]),
                                                 vertex_label=t(g["vlabel"]), k=-1, cap=10, keep=False))
            for i, g in enumerate(gs)]
    ex = serving.GpuExecutor(slots=2)
    for r in reqs:
        ex(r, 0)
    torch.cuda.synchronize()

    def timed(slot, r, out):
        st = ex.streams[slot]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ex(r, slot)
        e1.record(st)
        out[slot] = (e0, e1)

    solo = []
    for i, r in enumerate(reqs):
        o = {}
        timed(i, r, o)
        torch.cuda.synchronize()
        solo.append(o[i][0].elapsed_time(o[i][1]))
    best = None
    for _ in range(5):
        o = {}
        th = [threading.Thread(target=timed, args=(i, r, o)) for i, r in enumerate(reqs)]
        for x in th:
            x.start()
        for x in th:
            x.join()
        torch.cuda.synchronize()
        (a0, a1), (b0, b1) = o[0], o[1]
        ea, sb, eb = a0.elapsed_time(a1), a0.elapsed_time(b0), a0.elapsed_time(b1)
        together, overlap = max(ea, eb) - min(0.0, sb), min(ea, eb) - max(0.0, sb)
        if best is None or together < best[0]:
            best = (together, overlap)
    return {"graphs": f"two power-law graphs of {n:,} vertices / {m:,} edges, summarized to the fixpoint",
            "solo_ms": [round(x, 3) for x in solo], "together_ms": round(best[0], 3),
            "overlap_ms": round(best[1], 3), "speedup_vs_serial": round(sum(solo) / best[0], 3)}


# ----------------------------------------------------------------------------- oracle on the host cores

def oracle_graph(W):
    """The graph the CPU baselines run on: the workload's own graph (for the
    batched workload, the union of its first 512 graphs)."""
    from paper_2111_12493_gb300 import graphgen
    if W.batched:
        b = graphgen.batched_graphs(n_graphs=min(512, int(W.graph["n_graphs"])), seed=4)
        return graphgen.batched_union(b), f"the union of the first {b['n_graphs']} graphs of the generator"
    return W.graph, "the same graph"


def _ranges(n, parts):
    cuts = [n * i // parts for i in range(parts + 1)]
    return list(zip(cuts[:-1], cuts[1:]))


def _range_edges(g, ranges):
    """Edges whose source lies in each vertex range (the edges one range's round processes)."""
    cnt = np.bincount(g["src"], minlength=g["n"]).astype(np.int64)
    pre = np.concatenate([[0], np.cumsum(cnt)])
    return [int(pre[b] - pre[a]) for a, b in ranges]


def time_oracle_range(g, P0, v0, v1, out):
    import oracle
    t0 = time.perf_counter()
    oracle.refine_round_range(g["n"], g["src"], g["dst"], g["elabel"], g["vlabel"], P0, v0, v1, out=out,
                              graph=g.get("graph"))
    return time.perf_counter() - t0


def cpu_baseline(W):
    """The oracle as it stands on the host cores: one thread over 1/8 of the
    vertices of one exact round, and the same round over all vertices on every
    host thread (the multi-threaded restatement, pinned to the oracle)."""
    import oracle
    g, what = oracle_graph(W)
    n = g["n"]
    P0 = oracle.label_partition(n, g["vlabel"], graph=g.get("graph"))
    parts = 8 if n >= 1_000_000 else 1
    (v0, v1), = _ranges(n, parts)[:1]
    m_range = _range_edges(g, [(v0, v1)])[0]
    out = np.empty(n, np.int32)
    dt = time_oracle_range(g, P0, v0, v1, out)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.refine_round_threads(n, g["src"], g["dst"], g["elabel"], P0, threads=threads, graph=g.get("graph"))
    dt_all = time.perf_counter() - t0
    m = len(g["src"])
    return {"value": m_range / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "host_cores": threads,
            "sample": f"one exact refinement round P_0 -> P_1 over vertices [{v0:,}, {v1:,}) of {what} "
                      f"({n:,} vertices / {m:,} edges; {m_range:,} edges in the range), single-threaded C++ "
                      f"oracle, {dt:.1f} s",
            "all_cores": {"value": m / dt_all, "unit": UNIT, "cores": threads, "kind": "oracle, threaded",
                          "sample": f"the whole round P_0 -> P_1 of {what} on {threads} host threads "
                                    f"(the oracle's round with signatures gathered and maps built per shard in "
                                    f"parallel), {dt_all:.1f} s"}}


def run_reference(args, world, rank):
    """The CPU oracle on the same workload: step j is one exact refinement round
    P_0 -> P_1 over the j-th of `steps` consecutive vertex ranges, so the timed
    steps together cover one whole round of the full graph; warm-up steps repeat
    the first range."""
    if rank != 0:
        return
    import oracle
    W = Workload(args.workload, args.scale)
    g, what = oracle_graph(W)
    n = g["n"]
    P0 = oracle.label_partition(n, g["vlabel"], graph=g.get("graph"))
    ranges = _ranges(n, max(1, args.steps))
    medges = _range_edges(g, ranges)
    out = np.empty(n, np.int32)
    for _ in range(args.warmup):
        time_oracle_range(g, P0, ranges[0][0], ranges[0][1], out)
    t = [time_oracle_range(g, P0, a, b, out) for a, b in ranges]
    total = sum(t)
    value = sum(medges) / total
    extra = {"parallelism": "single CPU thread",
             "note": f"the oracle on {what}; each step one exact round over 1/{len(ranges)} of the vertices"}
    config = W.config(extra)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(ranges),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "int32 ids (exact signatures, no hashing)", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "host_cores": os.cpu_count(),
                             "sample": f"one exact refinement round P_0 -> P_1 per step over consecutive vertex "
                                       f"ranges of {what} ({n:,} vertices / {len(g['src']):,} edges); the "
                                       f"{len(ranges)} steps cover the whole round"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profile_updates(args, local):
    """The serving section's closed loop of 1k-op batches, incremental only, with a
    profiler window around K batches (launch lists of the update path)."""
    import torch
    from paper_2111_12493_gb300 import bisim, graphgen
    n, m = SERVING["n"], SERVING["m"]
    g = graphgen.powerlaw_graph(n=n, m=m, exponent=WORKLOAD["exponent"], dmax=min(WORKLOAD["dmax"], m // 10),
                                n_elabels=WORKLOAD["n_elabels"], n_vlabels=WORKLOAD["n_vlabels"],
                                untyped_frac=WORKLOAD["untyped"], seed=SERVING["seed"])
    dev = torch.device("cuda", local)
    d = {k: torch.from_numpy(g[k]).to(dev) for k in ("src", "dst", "elabel", "vlabel")}
    ctx = bisim.summarize_init_coo(n, d["src"], d["dst"], d["elabel"], d["vlabel"],
                                   options=bisim.default_options(k_incremental=SERVING["k"]))
    bisim.apply_updates(ctx, torch.zeros((0, 4), dtype=torch.int32, device=dev))
    batches = graphgen.update_batches(g, 8 + args.profile_updates, fixed_size=1000, seed=51)
    part = torch.empty(n, dtype=torch.int32, device=dev)
    lat = []
    for i, b in enumerate(batches):
        ops = torch.from_numpy(b["ops"]).pin_memory()
        torch.cuda.synchronize()
        if i == 8:
            torch.cuda.profiler.start()
        t0 = time.perf_counter()
        bisim.apply_updates(ctx, ops)
        bisim.get_partition(ctx, out=part)
        torch.cuda.synchronize()
        lat.append(1e3 * (time.perf_counter() - t0))
    torch.cuda.profiler.stop()
    bisim.summarize_destroy(ctx)
    print(json.dumps({"profile_updates": args.profile_updates, "batch_ms": lat}))


def literal_alg4_diagnostic(args, local):
    """Per configuration: blocks of P_k by the definition and by Algorithm 4
    taken literally, and the vertices whose literal class spans several of the
    definition's blocks (the literal algorithm merged them)."""
    import torch
    from paper_2111_12493_gb300 import bisim, graphgen
    dev = torch.device("cuda", local)
    sc = args.scale
    cases = [
        ("uniform 10k/50k, k=2", graphgen.uniform_graph(seed=1), 2),
        ("power-law 10M/100M, k=4 (its fixpoint round)", workload_graph(sc), 4),
        ("chains 1000x1000 + 2M random edges, k=4 (its fixpoint round)",
         graphgen.chain_graph(n_paths=max(10, int(1000 * sc)), path_len=1000, extra=int(2_000_000 * sc), seed=3), 4),
        ("4096 batched graphs as one union (graph id folded into the vertex label), k=3", None, 3),
        ("power-law 5M/50M (update base graph), k=2",
         graphgen.powerlaw_graph(n=max(1000, int(5_000_000 * sc)), m=max(10_000, int(50_000_000 * sc)),
                                 exponent=2.1, dmax=min(1_000_000, int(50_000_000 * sc) // 10), n_elabels=1000,
                                 n_vlabels=200, untyped_frac=0.1, seed=5), 2)]
    for name, g, k in cases:
        if g is None:
            b = graphgen.batched_graphs(n_graphs=max(8, int(4096 * sc)), seed=4)
            u = graphgen.batched_union(b)
            g = dict(u, vlabel=(u["graph"].astype(np.int64) * 16 + u["vlabel"]).astype(np.int32))
        t = [torch.from_numpy(np.ascontiguousarray(g[x])).to(dev) for x in ("src", "dst", "elabel", "vlabel")]
        ctx = bisim.summarize_init_coo(g["n"], *t)
        _, blocks = bisim.bisim_iterate(ctx, k, 0)
        P = bisim.get_partition(ctx).cpu().numpy()
        t0 = time.perf_counter()
        lit, lblocks = bisim.bisim_literal_alg4(ctx, k)
        dt = time.perf_counter() - t0
        lit = lit.cpu().numpy()
        bisim.summarize_destroy(ctx)
        # literal classes that hold more than one of the definition's blocks
        pairs = np.unique(np.stack([lit, P]).T, axis=0)
        per_lit = np.bincount(pairs[:, 0], minlength=g["n"])
        merged = per_lit[lit] > 1
        print(json.dumps({"literal_alg4": name, "k": k, "n_vertices": int(g["n"]), "n_edges": int(len(g["src"])),
                          "blocks_definition": int(blocks), "blocks_literal": int(lblocks),
                          "definition_blocks_merged": int(blocks - lblocks),
                          "vertices_in_merged_classes": int(merged.sum()),
                          "fraction_of_vertices": float(merged.mean()), "literal_s": round(dt, 2)}), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_init()
    if args.profile_updates > 0:
        profile_updates(args, local)
        return
    if args.literal_alg4:
        literal_alg4_diagnostic(args, local)
        return
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
