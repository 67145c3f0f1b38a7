#!/usr/bin/env python
"""Throughput of the GB300 PI-RRT# exploitation path (edge relaxations/s).

One step = the whole Batched-Extension schedule of one roadmap (Alg. 3):
starting from an empty graph, insert block after block (vertices plus the
edges whose other endpoint is present) and exploit to convergence after each
(Alg. 2: Improve / Evaluate until no parent switches).  The default workload
is the 6-D roadmap: [-pi, pi]^6 with 64 hyperspheres, N = 4,000,000
collision-free samples, k = 30 nearest neighbours, 16-point edge checks, FP32
costs, FP64 g, blocks of 50,000 vertices (80 exploitation rounds per step).

value      = edge relaxations (CSR entries scanned by Improve) / device time,
             inputs resident in HBM, summed over ranks (replicas).
e2e        = the same through the C ABI with pinned host inputs: every step
             copies the COO blocks host->device inside insert_batch and reads
             g and the parents back to the host.
roofline   = the dominant kernel's algorithmic bytes / its CUDA-event time,
             against the measured HBM copy bandwidth.
cpu_baseline / --impl reference = the CPU oracle (serial policy iteration,
             Alg. 2, one core) on a bounded prefix of the same schedule.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2003_04920_gb300 import workloads as W  # noqa: E402

METRIC = "edge relaxations/sec and ms to converged exploitation per batch; % of HBM roofline"
UNIT = "relaxations/s"
L2_BYTES = 129 * 1024 * 1024

WORKLOADS = {
    "c3": ("roadmap_c3", "6-D [-pi,pi]^6, 64 hyperspheres r~U[0.3,0.8], N=4e6, k=30, "
                         "16-point edge check, FP32 costs, FP64 g, blocks of 5e4"),
    "c3-gpu": ("roadmap_c3_gpu", "6-D [-pi,pi]^6, 64 hyperspheres r~U[0.3,0.8], N=4e6, k=30, "
                                 "16-point edge check, FP32 costs, FP64 g, blocks of 5e4; the "
                                 "same law built by the GPU generator (Philox samples, grid "
                                 "k-NN; another instance, another x_init)"),
    "c2": ("roadmap_c2", "2-D unit square, 200 circles r~U[0.02,0.08], N=1e6, k=76, FP32 costs, "
                         "FP64 g, blocks of 1e4"),
    "c2-companion": ("roadmap_c2", "2-D unit square, 200 circles r~U[0.01,0.04], N=1e6, k=76, "
                                   "FP32 costs, FP64 g, blocks of 1e4"),
}


def load_roadmap(name: str, n: int | None, block: int | None, trial: int):
    """The workload's roadmap; ``block`` (the Batched-Extension block size S)
    only changes how its edge list is cut, not the graph (Alg. 3: the final
    graph does not depend on S)."""
    fn_name, _ = WORKLOADS[name]
    kw = dict(trial=trial)
    if n:
        kw["n"] = n
    if fn_name == "roadmap_c3_gpu":
        # seconds on the device, no on-disk cache; host copies for the pinned
        # end-to-end pass and the oracle legs
        import torch

        from paper_2003_04920_gb300.workloads import gpu as GG
        GG.build()
        GG.load()
        if block:
            kw["block"] = int(block)
        drm = GG.roadmap_c3_gpu(**kw)
        rm = drm.to_host()
        del drm
        torch.cuda.empty_cache()
        return rm
    if name == "c2-companion":
        kw["companion"] = True
    rm = W.cached(name, getattr(W, fn_name), **kw)
    if block:
        rm.block = int(block)
    return rm


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, busy_sm_floor: float = 0.0) -> dict:
        rows = []
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    rows.append(dict(sm=float(parts[1]), smax=float(parts[2]),
                                     hw=parts[5], hwt=parts[6], swt=parts[7], pcap=parts[8]))
                except ValueError:
                    continue
            os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        reasons = set()
        for r in rows:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows),
                "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def improve_bytes(prof: dict, entry_bytes: int, cost_bytes: int, offers: bool) -> float:
    """Algorithmic (compulsory) HBM bytes of all Improve launches.  Every CSR
    entry scanned (col + cost); per vertex of a dense sweep its row offsets,
    parent, parent-edge cost, the parent's g and its own g; per listed vertex
    the list id, parent, parent-edge cost and the parent's g, plus its row
    offsets (full scans) or its best offer (candidate offers, where only the
    deciding vertices -- at least every switch -- read their row offsets);
    the parent / cost writes and the switch-list id of each switch.  Gathers
    of g(u) for scanned entries are not counted (a lower bound)."""
    entries = prof["improve_entries"]
    verts = prof["improve_vertices"]
    dense_v = prof["improve_dense_vertices"]
    sparse_v = verts - dense_v
    sw = prof["improve_switches"]
    dense = dense_v * (8 + 4 + cost_bytes + 8 + 8)
    if offers:
        sparse = sparse_v * (4 + 4 + cost_bytes + 8 + 8) + sw * 8
    else:
        sparse = sparse_v * (4 + 8 + 4 + cost_bytes + 8)
    return entries * entry_bytes + dense + sparse + sw * (4 + cost_bytes + 4)


def evaluate_bytes(prof: dict, entry_bytes: int, cost_bytes: int) -> float:
    """Evaluate: per recomputed vertex its parent, parent-edge cost, the
    parent's g and the g write; per candidate offer the CSR entry it comes
    from (offer updates themselves are not counted)."""
    return (prof["evaluate_vertices"] * (4 + cost_bytes + 8 + 8)
            + prof.get("evaluate_offers", 0) * entry_bytes)


def reduce_over_ranks(elapsed: float, units: float, world: int, device) -> tuple[float, float]:
    """Whole-job figures of a replicated run: the slowest rank's time (MAX)
    and the units every rank processed (SUM).  A no-op for one rank."""
    if world <= 1:
        return elapsed, units
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def run_ours(args) -> None:
    import torch
    import torch.distributed as dist

    import paper_2003_04920_gb300 as P

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    P.load_library()

    rm = load_roadmap(args.workload, args.n, args.block, args.trial)
    n_blocks = rm.n_blocks()
    stream = torch.cuda.current_stream()
    dev_u = torch.from_numpy(rm.u).cuda()
    dev_v = torch.from_numpy(rm.v).cuda()
    dev_c = torch.from_numpy(rm.cost).cuda()
    cost_bytes = rm.cost.dtype.itemsize
    entry_bytes = 8 if cost_bytes == 4 else 16
    G = P.Graph(rm.n, rm.m, 0, rm.cost.dtype, device=local, stream=stream.cuda_stream)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
    goal = None
    if args.goal == "far":
        # x_goal: the sample nearest to x_init reflected through the centre of
        # the sampled box; h = 0.99 x the Euclidean distance to it (admissible
        # and consistent: the edge costs are Euclidean lengths)
        lo, hi = rm.points.min(axis=0), rm.points.max(axis=0)
        target = (lo + hi) - rm.points[0]
        goal = int(np.argmin(np.linalg.norm(rm.points - target, axis=1)))
        h_goal = (0.99 * np.linalg.norm(rm.points - rm.points[goal], axis=1)).astype(np.float32)
        G.set_goal(goal, h_goal)

    extra = {"wave_levels": 0, "jump_evaluates": 0, "dense_sweeps": 0, "switches": 0,
             "improve_entries": 0, "offers": 0}
    block_ms = []  # per-block device time of the last step run with block_times=True
    traffic_block = -1 if args.traffic_block is None else \
        (args.traffic_block % n_blocks if n_blocks else -1)
    traffic_window = {}
    prof_on = [False]

    def step(device_inputs=True, block_times=False):
        G.reset()
        relax = 0
        iters = 0
        for k in extra:
            extra[k] = 0
        blocks = list(rm.blocks())
        ev = []
        for b, (v0, v1, e0, e1) in enumerate(blocks):
            if block_times:
                ev.append(torch.cuda.Event(enable_timing=True))
                ev[-1].record(stream)
            if device_inputs:
                G.insert_batch(v1 - v0, dev_u[e0:e1], dev_v[e0:e1], dev_c[e0:e1])
            else:
                G.insert_batch(v1 - v0, host_u[e0:e1], host_v[e0:e1], host_c[e0:e1])
                if b + 1 < len(blocks) and not args.no_prefetch:
                    # the next block's copy overlaps this exploit
                    _, _, f0, f1 = blocks[b + 1]
                    G.prefetch_batch(host_u[f0:f1], host_v[f0:f1], host_c[f0:f1])
            window = b == traffic_block and prof_on[0] and not traffic_window
            if window:
                # the exploit whose Evaluate launches a profiler captures by
                # this NVTX range (DRAM counters over a few launches)
                torch.cuda.nvtx.range_push("traffic_window")
                before = G.get_profile()
            st = G.exploit(group=args.group, tile=args.tile, dense_fraction=args.dense_fraction,
                           evaluate=args.evaluate, wave_levels=args.wave_levels,
                           host_loop=args.host_loop, wave_tail=args.wave_tail,
                           wave_ctas=args.wave_ctas, wave_local=args.wave_local,
                           wave_local_max=args.wave_local_max,
                           wave_local_step=args.wave_local_step)
            if window:
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_pop()
                after = G.get_profile()
                d = {k: after[k] - before[k] for k in ("evaluate_launches", "evaluate_vertices",
                                                       "evaluate_offers", "evaluate_ms")}
                traffic_window.update(block=b, evaluate_calls=int(d["evaluate_launches"]),
                                      evaluate_ms=round(float(d["evaluate_ms"]), 4),
                                      algorithmic_bytes=int(evaluate_bytes(
                                          {"evaluate_vertices": d["evaluate_vertices"],
                                           "evaluate_offers": d["evaluate_offers"]},
                                          entry_bytes, cost_bytes)))
            relax += st["relaxations"]
            iters += st["iterations"]
            for k in extra:
                extra[k] += st[k]
        if block_times:
            ev.append(torch.cuda.Event(enable_timing=True))
            ev[-1].record(stream)
            ev[-1].synchronize()
            block_ms[:] = [ev[i].elapsed_time(ev[i + 1]) for i in range(len(blocks))]
        return relax, iters

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()

    # device-resident inputs, one CUDA-event pair per step, L2 flushed between
    # steps outside the timed spans (the CSR is also ~8x larger than L2).
    # "graph": every exploit is one CUDA-graph launch (the product path), and
    # the per-kernel split comes from profiled steps run right after the
    # timed ones; "profiled": the timed steps themselves run the host loop
    # with an event pair around every kernel.
    timed_extra = []

    def timed_steps(k):
        ts, rs, its = [], [], []
        timed_extra.clear()
        for _ in range(k):
            flush.fill_(1)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r, it = step()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
            rs.append(r)
            its.append(it)
            timed_extra.append(dict(extra))
        return ts, rs, its

    with ClockSampler(local) as clk:
        G.set_profiling(args.timing == "profiled")
        prof_on[0] = args.timing == "profiled"
        times, relaxes, iters_all = timed_steps(args.steps)
        improve_only = float(sum(e["improve_entries"] for e in timed_extra))
        step_extra = dict(timed_extra[-1]) if timed_extra else dict(extra)
        # the library counts its kernel launches also while not profiling
        timed_launches = G.get_profile()["launches"]
        if args.timing == "graph":
            G.set_profiling(True)
            prof_on[0] = True
            prof_times, _, _ = timed_steps(args.profile_steps)
        else:
            prof_times = times
        prof = G.get_profile()
        if args.trace:
            np.save(args.trace, G.get_trace())
        # one more step with every exploit a single CUDA-graph launch and only
        # the device-side trace on: how long the wave launches run, and the
        # time between one launch's end and the next one's start
        G.set_profiling(2)
        graph_trace_ms, _, _ = timed_steps(1)
        gprof = G.get_profile()
        G.set_profiling(False)
        prof_on[0] = False
    barrier()
    clocks = clk.summary()
    prof_ms = float(sum(prof_times))

    total_ms = float(sum(times))
    total_relax = float(sum(relaxes))
    total_ms, total_relax = reduce_over_ranks(total_ms, total_relax, world, "cuda")
    value = total_relax / (total_ms / 1e3)
    improve_ms, improve_only = reduce_over_ranks(float(sum(times)), improve_only, world, "cuda")
    value_improve_only = improve_only / (improve_ms / 1e3)
    ms_per_step = total_ms / args.steps

    # end to end through the C ABI with pinned host buffers
    e2e_steps = 0 if args.no_e2e else args.steps
    pin_u = torch.from_numpy(rm.u).pin_memory()
    pin_v = torch.from_numpy(rm.v).pin_memory()
    pin_c = torch.from_numpy(rm.cost).pin_memory()
    host_u, host_v, host_c = pin_u.numpy(), pin_v.numpy(), pin_c.numpy()
    out_g = torch.empty(rm.n, dtype=torch.float64).pin_memory().numpy()
    out_p = torch.empty(rm.n, dtype=torch.int32).pin_memory().numpy()
    barrier()
    t0 = time.perf_counter()
    e2e_relax = 0
    for _ in range(e2e_steps):
        r, _ = step(device_inputs=False)
        G.get_costs(out_g)
        G.get_parents(out_p)
        e2e_relax += r
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s, e2e_relax = reduce_over_ranks(e2e_s, float(e2e_relax), world, "cuda")
    h2d = rm.m * (4 + 4 + cost_bytes)
    d2h = rm.n * (8 + 4)

    peak, peak_src = measured_peaks()
    offers = args.tile == 0
    kernels = {}
    kbytes = {"improve": improve_bytes(prof, entry_bytes, cost_bytes, offers),
              "evaluate": evaluate_bytes(prof, entry_bytes, cost_bytes),
              "mark_frontier": None,
              "insert": prof["insert_new_entries"] * entry_bytes}
    for name, ms_key, launches_key in (
            ("improve", "improve_ms", "improve_launches"),
            ("evaluate", "evaluate_ms", "evaluate_launches"),
            ("mark_frontier", "mark_ms", "mark_launches"),
            ("insert", "insert_ms", "insert_calls")):
        ms = prof[ms_key]
        nbytes = kbytes[name]
        k = {"ms": round(ms, 3), "launches": prof[launches_key],
             "share_of_step": round(ms / prof_ms, 4) if prof_ms else None}
        if nbytes is not None and ms > 0:
            k["algorithmic_gbs"] = round(nbytes / (ms / 1e3) / 1e9, 1)
            k["algorithmic_bytes"] = int(nbytes)
        kernels[name] = k
    # the dominant kernel: the largest share of the profiled step
    dom = max(("improve", "evaluate", "insert"), key=lambda k: kernels[k]["ms"])
    launches = max(1, kernels[dom]["launches"])
    dom_ms_avg = kernels[dom]["ms"] / launches
    dom_bytes = kbytes[dom]
    achieved = (dom_bytes / launches) / (dom_ms_avg / 1e3) / 1e9 if dom_ms_avg > 0 else 0.0
    traffic = None
    g_goal = None
    if goal is not None:
        g_goal = float(G.get_costs()[goal])
    tpath = os.path.join(ROOT, "profiles", f"{dom}_traffic_{args.workload}.json")
    if not os.path.exists(tpath):
        tpath = os.path.join(ROOT, "profiles", f"{dom}_traffic.json")
    if os.path.exists(tpath):
        with open(tpath) as f:
            tj = json.load(f)
        if (tj.get("workload") == args.workload and tj.get("kernel_hash") == kernel_hash(dom)
                and goal is None):
            traffic = tj.get("traffic_bytes_per_launch")

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 3),
        "ms_per_batch": round(ms_per_step / n_blocks, 4),
        "value_improve_only": round(value_improve_only, 1),
        "value_note": ("value counts every candidate g(u) + c(u, v) formed: the adjacency entries "
                       "Improve scans plus the candidates Evaluate offers to the next Improve; "
                       "value_improve_only counts the Improve scans alone"),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded roadmap generator)",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload][1]}",
                   "vertices": rm.n, "undirected_edges": rm.m, "csr_entries": 2 * rm.m,
                   "blocks_per_step": n_blocks, "block_size": rm.block,
                   "evaluate": args.evaluate, "wave_tail": args.wave_tail,
                   "goal": None if goal is None else {
                       "vertex": goal, "g_goal": g_goal,
                       "heuristic": "0.99 x Euclidean distance to x_goal (FP32)",
                       "pruned_form": "goal-directed Replan, promising g + h < g(x_goal)"},
                   "wave_ctas": args.wave_ctas, "wave_local": args.wave_local,
                   "wave_local_max": args.wave_local_max,
                   "wave_local_step": args.wave_local_step,
                   "iterations_per_step": iters_all[-1], "relaxations_per_step": relaxes[-1],
                   "per_step": step_extra,
                   "improve_kernel": {0: "candidate offers; dense sweeps by lane groups with "
                                         "FP32 screening",
                                      2: "lane groups, FP32 screening", 1: "staged bulk copies",
                                      3: "lane groups, exact FP64"}[args.tile],
                   "improve_lanes_per_vertex": args.group or (4 if args.tile == 0 else 8),
                   "timing": ("each exploit one CUDA-graph launch; per-kernel split and roofline "
                              f"from {args.profile_steps} profiled step(s) (host loop, CUDA events "
                              f"around every kernel, {round(prof_ms / max(1, len(prof_times)), 3)} "
                              "ms per step) run right after the timed steps")
                             if args.timing == "graph" else
                             "host loop with CUDA events around every kernel",
                   "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (CSR ~%.2f GB) and L2 flushed between steps"
                         % (2 * rm.m * entry_bytes / 1e9)},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_source": f"{peak_src} copy bandwidth",
                     "frac_of_nominal_8tbs": round(achieved / 8000.0, 4),
                     "traffic": traffic,
                     "bytes_per_launch": round(dom_bytes / launches, 1),
                     "avg_launch_ms": round(dom_ms_avg, 5)},
        "kernels": kernels,
        # the whole step against the same peak: every phase's algorithmic bytes
        # (scaled from the profiled step to the timed ones by their relaxations)
        # over the timed step time
        "step_roofline": step_roofline(kbytes, max(1, len(prof_times)), ms_per_step, peak),
        "wave_level_profile": level_profile(prof, clocks),
        "graph_launch_trace": {
            "step_ms": round(graph_trace_ms[0], 3), "wave_launches": gprof["wave_spans"],
            "wave_span_ms": round(gprof["wave_span_ns"] / 1e6, 3),
            "gaps": gprof["wave_gaps"], "gap_ms": round(gprof["wave_gap_ns"] / 1e6, 3),
            "note": "one step of captured loops: wave launches from CTA 0's start to the end of "
                    "their iteration, and the time from one launch's end to the next one's start "
                    "within an exploit (the dense-sweep kernel between them and the launch "
                    "latency), on the global timer"},
        "e2e": {"value": round(e2e_relax / e2e_s, 1) if e2e_steps else None, "unit": UNIT,
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "prefetch": not args.no_prefetch},
        "gpu_launches": int(timed_launches),
        "clocks": clocks,
    }
    if traffic_window:
        line["traffic_window"] = traffic_window
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # per-block device times of one more (untimed) step, for a GPU figure
        # over exactly the block prefix the oracle covers
        step(block_times=True)
        line["cpu_baseline"] = cpu_baseline(rm, args.cpu_seconds, goal,
                                            h_goal if goal is not None else None,
                                            gpu_block_ms=list(block_ms),
                                            dijkstra=not args.no_dijkstra)
    G.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


KERNEL_FILES = {"improve": ("improve_push.cuh", "improve_screen.cuh", "graph_kernels.cuh",
                            "replan_iteration.cuh", "device_common.cuh"),
                "evaluate": ("graph_kernels.cuh", "replan_iteration.cuh", "improve_push.cuh",
                             "evaluate_async.cuh", "device_common.cuh"),
                "insert": ("graph_kernels.cuh", "device_common.cuh")}


def kernel_hash(kernel: str) -> str:
    """Hash of the code a kernel is built from (its sources with comments and
    whitespace removed): a stored DRAM traffic figure is used only while it
    matches."""
    import hashlib
    import re
    h = hashlib.sha1()
    for f in KERNEL_FILES[kernel]:
        with open(os.path.join(ROOT, "paper_2003_04920_gb300", "csrc", f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("".join(text.split()).encode())
    return h.hexdigest()[:12]


def oracle_prefix(rm, seconds: float, goal=None, h=None, lib=None, max_blocks=None) -> dict:
    """Serial policy iteration (the oracle, Alg. 2) on a prefix of the same
    Batched-Extension schedule, block by block, until `seconds` have passed
    or `max_blocks` blocks are done (goal-directed, Sec. IV-C, when `goal` is
    given); `lib` picks another build of the oracle."""
    import oracle as O
    G = O.OracleGraph(rm.n, lib=lib)
    if goal is not None:
        G.set_goal(goal, np.asarray(h, dtype=np.float64))
    relax = 0
    blocks = 0
    t_exploit = 0.0
    t0 = time.perf_counter()
    for v0, v1, e0, e1 in rm.blocks():
        G.insert(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1].astype(np.float64))
        t = time.perf_counter()
        st = G.replan()
        t_exploit += time.perf_counter() - t
        relax += st["relaxations"]
        blocks += 1
        if time.perf_counter() - t0 > seconds or (max_blocks is not None and blocks >= max_blocks):
            break
    G.close()
    return dict(relax=relax, blocks=blocks, seconds=t_exploit, n_present=min(rm.n, blocks * rm.block))


def dijkstra_baseline(rm) -> dict:
    """O2, the oracle's FP64 binary-heap Dijkstra (1 core), on the final graph
    of the schedule: the shortest-path tree that every Replan converges to
    (Sec. V), computed once from scratch."""
    import oracle as O
    t0 = time.perf_counter()
    A = O.CSR(rm.n, rm.u, rm.v, rm.cost.astype(np.float64))
    t1 = time.perf_counter()
    A.dijkstra(0)
    t2 = time.perf_counter()
    entries = A.entries
    A.close()
    return {"kind": "oracle O2 (FP64 binary-heap Dijkstra)", "cores": 1,
            "ms": round(1e3 * (t2 - t1), 1), "csr_build_ms": round(1e3 * (t1 - t0), 1),
            "edges_scanned_per_s": round(entries / (t2 - t1), 1),
            "sample": f"final graph of the schedule: {rm.n} vertices, {entries} adjacency entries, "
                      "one shortest-path tree from x_init"}


def cpu_baseline(rm, seconds: float, goal=None, h=None, gpu_block_ms=None,
                 dijkstra: bool = False) -> dict:
    r = oracle_prefix(rm, seconds, goal, h)
    form = "" if goal is None else f"goal-directed toward vertex {goal} (Sec. IV-C), "
    out = {"value": round(r["relax"] / r["seconds"], 1), "unit": UNIT, "cores": 1,
           "kind": "oracle",
           "ms_per_batch": round(1e3 * r["seconds"] / r["blocks"], 3),
           "sample": f"serial policy iteration (Alg. 2), {form}on the first {r['blocks']} of "
                     f"{rm.n_blocks()} blocks of the same schedule ({r['n_present']} vertices), "
                     f"Improve sweeping every vertex each round; {r['relax']} relaxations "
                     f"in {r['seconds']:.2f} s (exploitation only)"}
    if gpu_block_ms:
        k = min(r["blocks"], len(gpu_block_ms))
        out["gpu_ms_per_batch_same_prefix"] = round(sum(gpu_block_ms[:k]) / k, 4)
        out["gpu_prefix_note"] = (f"GPU insertion plus exploitation per block over the same first "
                                  f"{k} blocks, CUDA events, one step")
    if dijkstra:
        out["dijkstra"] = dijkstra_baseline(rm)
    out["openmp"] = openmp_baseline(rm, r, goal, h)
    return out


def openmp_baseline(rm, serial: dict, goal=None, h=None) -> dict:
    """The oracle built with OpenMP (its Jacobi Improve sweep over the host's
    cores, results identical to the serial build) on the same block prefix as
    the serial run: an all-core CPU baseline beside the one-core one."""
    import oracle as O
    try:
        lib = O.load_parallel()
        if lib is None:
            return {"unavailable": "the compiler has no OpenMP"}
        r = oracle_prefix(rm, 10.0 * serial["seconds"] + 60.0, goal, h, lib=lib,
                          max_blocks=serial["blocks"])
    except Exception as e:  # a baseline beside the measurement, never a reason to fail it
        return {"unavailable": f"{type(e).__name__}: {e}"}
    return {"kind": "oracle built with OpenMP: the Jacobi Improve sweep shared over the host's "
                    "cores, Evaluate's walk serial; the serial build's results bit for bit",
            "cores": O.threads(lib), "value": round(r["relax"] / r["seconds"], 1), "unit": UNIT,
            "ms_per_batch": round(1e3 * r["seconds"] / r["blocks"], 3),
            "sample": f"the first {r['blocks']} blocks, as the one-core run; {r['relax']} "
                      f"relaxations in {r['seconds']:.2f} s (exploitation only)"}


def run_batch(args) -> None:
    """Batched form: every member roadmap inserted and exploited to a fixpoint
    in one CUDA-graph launch (options picked by the batch autotuner), next to
    the same members exploited one after another as separate graphs."""
    import torch

    import paper_2003_04920_gb300 as P

    torch.cuda.set_device(0)
    P.load_library()
    n_graphs = args.graphs
    rms = W.cached_batch(n_graphs, args.trial, 1_000, args.n or 200_000,
                         workers=max(1, (os.cpu_count() or 2) - 1))
    dev = [(torch.from_numpy(r.u).cuda(), torch.from_numpy(r.v).cuda(),
            torch.from_numpy(r.cost).cuda()) for r in rms]
    stream = torch.cuda.current_stream()
    B = P.Batch([r.n for r in rms], [r.m for r in rms], stream=stream.cuda_stream)

    def fill():
        B.reset()
        for i, (u, v, c) in enumerate(dev):
            B.insert(i, u, v, c)

    fill()
    # the library's searching autotuner: coordinate descent over the Improve
    # kernel and its lanes, the dense threshold, the Evaluate form and the
    # wave's shape, every trial from the same merged state
    t_tune = time.perf_counter()
    best, best_ms, trials = B.autotune_search(max_trials=args.tune_trials)
    tune_s = time.perf_counter() - t_tune

    def timed(fn, k):
        ts = []
        for _ in range(k):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return ts, r

    def batched():
        fill()
        return B.exploit(**best)

    for _ in range(args.warmup):
        batched()
    B.set_profiling(False)  # clears the launch count
    with ClockSampler(0) as clk:
        ts, st = timed(batched, args.steps)
    clocks = clk.summary()
    timed_launches = B.get_profile()["launches"]
    relax = st["relaxations"]
    ms = sum(ts) / len(ts)
    # the same members, one graph and one exploit each
    solos = [P.Graph(r.n, r.m, 0, r.cost.dtype, stream=stream.cuda_stream) for r in rms]

    def separate():
        tot = 0
        for G, (u, v, c), r in zip(solos, dev, rms):
            G.reset()
            G.insert_batch(r.n, u, v, c)
            tot += G.exploit(**best)["relaxations"]
        return tot

    separate()
    ts2, _ = timed(separate, max(1, args.steps))
    ms2 = sum(ts2) / len(ts2)
    # one profiled pass for the per-kernel split
    fill()
    B.set_profiling(True)
    B.exploit(**{**best, "host_loop": True})
    prof = B.get_profile()
    B.set_profiling(False)
    peak, peak_src = measured_peaks()
    launches = max(1, prof["improve_launches"])
    imp_bytes = improve_bytes(prof, 8, 4, best.get("tile", 0) == 0)
    imp_avg = prof["improve_ms"] / launches
    achieved = (imp_bytes / launches) / (imp_avg / 1e3) / 1e9 if imp_avg > 0 else 0.0
    line = {
        "metric": METRIC, "value": round(relax / (ms / 1e3), 1), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "ms_per_batch": round(ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded roadmap generator)",
        "config": {"workload": f"c4: {n_graphs} roadmaps, N log-uniform in [1e3, {args.n or 200000:.0e}], "
                               "dimension in {2,3,4,6,7}, k=ceil(2e ln N), FP32 costs; one exploit "
                               "of all members to a fixpoint per step",
                   "vertices": sum(r.n for r in rms), "undirected_edges": sum(r.m for r in rms),
                   "autotuned_options": best,
                   "autotune": {"kind": "coordinate descent (pirrt_batch_autotune_search)",
                                "trials": trials, "best_trial_ms": round(best_ms, 3),
                                "seconds": round(tune_s, 2)},
                   "separate_graphs_ms_per_step": round(ms2, 3),
                   "batched_speedup_vs_separate": round(ms2 / ms, 3),
                   "iterations": st["iterations"], "graph_launch": st["graph_launch"],
                   "l2": "inputs larger than L2"},
        "roofline": {"bound": "hbm", "kernel": "improve", "achieved": round(achieved, 1),
                     "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "peak_source": f"{peak_src} copy bandwidth (profiled host-loop pass)",
                     "traffic": None},
        "gpu_launches": int(timed_launches),
        "clocks": clocks,
    }
    for G in solos:
        G.close()
    B.close()
    print(json.dumps(line), flush=True)


SWEEP_S = (1, 3, 10, 30, 100, 300, 1000, 3000)


def sweep_case(n: int, trial: int, goal: bool):
    """The block-size sweep's query (Sec. VI: a 2-D query, N samples in
    batches of S).  The unit square with 200 circles r ~ U[0.01, 0.04] (an
    obstacle covering either end is redrawn); vertex 0 = x_init = (0.05, 0.05)
    and vertex 1 = x_goal = (0.95, 0.95), both in V from the start as in
    Alg. 1, then N - 2 uniform free samples; k = ceil(2e ln N), FP32 costs.
    Goal-directed Replan (Sec. IV-C) with h = 0.99 x the Euclidean distance to
    x_goal, or no goal."""
    scene = W.c5_scene(900 + trial)
    rng = np.random.default_rng(6 * 1000 + trial)
    ends = np.array([W.C5_X_INIT, W.C5_X_GOAL], dtype=np.float64)
    pts = np.vstack([ends, W.free_uniform(rng, scene, n - 2)])
    rm = W.roadmap_from_points("sweep", pts, scene)
    if not goal:
        return rm, None, None
    h = (0.99 * np.linalg.norm(rm.points - rm.points[1], axis=1)).astype(np.float32)
    return rm, 1, h


def sweep_gpu(rm, goal, h, s_list, reps: int) -> dict:
    """Insertion plus exploitation of the whole schedule for each S on the
    GPU: wall time from the first insertion to the last exploit's result
    (each exploit returns its statistics to the host), median of `reps` runs
    after one warm-up run; blocks resident in device memory."""
    import torch

    import paper_2003_04920_gb300 as P
    P.load_library()
    dev = [torch.from_numpy(a).cuda() for a in (rm.u, rm.v, rm.cost)]
    out = {}
    with P.Graph(rm.n, rm.m, 0, rm.cost.dtype,
                 stream=torch.cuda.current_stream().cuda_stream) as G:
        if goal is not None:
            G.set_goal(goal, h)
        for S in s_list:
            blocks = list(rm.blocks(S))
            times = []
            for r in range(reps + 1):
                G.reset()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                relax = iters = 0
                for v0, v1, e0, e1 in blocks:
                    G.insert_batch(v1 - v0, dev[0][e0:e1], dev[1][e0:e1], dev[2][e0:e1])
                    st = G.exploit()
                    relax += st["relaxations"]
                    iters += st["iterations"]
                torch.cuda.synchronize()
                if r:
                    times.append(time.perf_counter() - t0)
            g = G.get_costs()
            out[S] = {"ms": round(1e3 * statistics.median(times), 3), "blocks": len(blocks),
                      "iterations": iters, "relaxations": relax,
                      "g_goal": None if goal is None else float(g[goal])}
    return out


def sweep_oracle(rm, goal, h, s_list, seconds: float) -> dict:
    """The same schedules on the oracle (serial policy iteration, one core),
    insertion plus Replan timed block by block; a schedule that passes
    `seconds` stops there and reports the blocks it finished."""
    import oracle as O
    out = {}
    for S in s_list:
        blocks = list(rm.blocks(S))
        G = O.OracleGraph(rm.n)
        if goal is not None:
            G.set_goal(goal, np.asarray(h, dtype=np.float64))
        spent = 0.0
        done = relax = iters = 0
        for v0, v1, e0, e1 in blocks:
            t0 = time.perf_counter()
            G.insert(v1 - v0, rm.u[e0:e1], rm.v[e0:e1], rm.cost[e0:e1].astype(np.float64))
            st = G.replan()
            spent += time.perf_counter() - t0
            relax += st["relaxations"]
            iters += st["iterations"]
            done += 1
            if spent > seconds:
                break
        g, _ = G.get()
        G.close()
        full = done == len(blocks)
        out[S] = {"ms": round(1e3 * spent, 3), "blocks": len(blocks), "blocks_done": done,
                  "complete": full, "iterations": iters, "relaxations": relax,
                  "g_goal": float(g[goal]) if (goal is not None and full) else None}
    return out


def run_sweep(args) -> None:
    """Planning time against the block size S (Sec. VI's Batched-Extension
    experiment) at each N of --sweep-n, on the GPU and on the oracle, as one
    JSON line.  Not the benchmark's headline: every run here fits in L2."""
    ns = [int(x) for x in args.sweep_n.split(",")]
    s_list = [int(x) for x in args.sweep_s.split(",")]
    legs = set(args.sweep_legs.split(","))
    rows = []
    clocks = None
    for n in ns:
        rm, goal, h = sweep_case(n, args.trial, args.goal != "none")
        ss = [S for S in s_list if S <= n]
        gpu = {}
        if "gpu" in legs:
            with ClockSampler(0) as clk:
                gpu = sweep_gpu(rm, goal, h, ss, max(1, args.steps))
            c = clk.summary()
            clocks = c if clocks is None else {
                "sm_mhz": c["sm_mhz"], "sm_max_mhz": c["sm_max_mhz"],
                "reasons": sorted(set(clocks["reasons"]) | set(c["reasons"])),
                "samples": clocks["samples"] + c["samples"]}
        cpu = sweep_oracle(rm, goal, h, ss, args.cpu_seconds) if "oracle" in legs else {}
        for S in ss:
            rows.append({"n": n, "S": S, "gpu": gpu.get(S), "oracle": cpu.get(S)})
    line = {"experiment": "block-size sweep (Sec. VI, Batched-Extension)",
            "unit": "ms of insertion plus exploitation for the whole schedule",
            "workload": "2-D unit square, 200 circles r~U[0.01,0.04], x_init=(0.05,0.05) "
                        "vertex 0, x_goal=(0.95,0.95) vertex 1, k=ceil(2e ln N), FP32 costs, "
                        "FP64 g",
            "goal": "x_goal = vertex 1, h = 0.99 x Euclidean distance"
                    if args.goal != "none" else None,
            "oracle": {"kind": "oracle", "cores": 1, "budget_s": args.cpu_seconds,
                       "host": os.uname().machine, "host_cores": os.cpu_count()},
            "gpu_repeats": max(1, args.steps) if "gpu" in legs else 0,
            "gpu_timing": "median of the repeats after one warm-up run, wall time from the "
                          "first insertion to the last exploit's statistics",
            "clocks": clocks,
            "rows": rows}
    print(json.dumps(line), flush=True)


def run_explore(args) -> None:
    """Exploration overlapped with exploitation (the asynchronous form the
    paper leaves to future work, Sec. VII) on the 6-D workload's scene law:
    every block's Extend step -- its samples' nearest predecessors, collision
    checks, edge costs -- built on the GPU (workloads.gpu.Explorer), then
    inserted and exploited to a stable policy.  Two passes over the same
    roadmap: one stream doing exploration then exploitation block after block,
    and two streams, the exploration of block b + 1 running while block b is
    exploited (double-buffered edge blocks, events between the streams)."""
    import torch

    import paper_2003_04920_gb300 as P
    from paper_2003_04920_gb300.workloads import gpu as GG

    torch.cuda.set_device(0)
    P.load_library()
    GG.load()
    n = args.n or 4_000_000
    S = args.block or 50_000
    k = 30
    seed = 3 * 1000 + args.trial
    scene = W._draw_scene(np.random.default_rng(seed), 6, -math.pi, math.pi, 64, 0.3, 0.8, [])
    lo_pri, hi_pri = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream, "priority_range") \
        else (0, -1)
    sx = torch.cuda.Stream(priority=hi_pri)   # exploitation
    se = torch.cuda.Stream(priority=lo_pri)   # exploration
    X = GG.Explorer(scene, n, k, seed, S, stream=se.cuda_stream)
    G = P.Graph(n, n * k, 0, np.float32, stream=sx.cuda_stream)
    blocks = [(v0, min(n, v0 + S)) for v0 in range(0, n, S)]

    def sequential():
        G.reset()
        it = 0
        for b, (v0, v1) in enumerate(blocks):
            u, v, c, cnt = X.extend(v0, v1, b & 1, stream=sx.cuda_stream)
            sx.synchronize()
            m = int(cnt.item())
            G.insert_batch(v1 - v0, u[:m], v[:m], c[:m])
            it += G.exploit()["iterations"]
        return it

    def overlapped():
        G.reset()
        it = 0
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        freed = [torch.cuda.Event(), torch.cuda.Event()]
        nxt = X.extend(blocks[0][0], blocks[0][1], 0, stream=se.cuda_stream)
        ready[0].record(se)
        for b, (v0, v1) in enumerate(blocks):
            u, v, c, cnt = nxt
            ready[b & 1].synchronize()  # the block's edge count is on the host
            m = int(cnt.item())
            sx.wait_event(ready[b & 1])
            G.insert_batch(v1 - v0, u[:m], v[:m], c[:m])
            freed[b & 1].record(sx)
            if b + 1 < len(blocks):
                # the next block's Extend on its own stream, into the other buffer
                # (free once the insertion of block b - 1 has read it)
                if b >= 1:
                    se.wait_event(freed[(b + 1) & 1])
                nxt = X.extend(blocks[b + 1][0], blocks[b + 1][1], (b + 1) & 1,
                               stream=se.cuda_stream)
                ready[(b + 1) & 1].record(se)
            it += G.exploit()["iterations"]
        return it

    def explore_only():
        for b, (v0, v1) in enumerate(blocks):
            X.extend(v0, v1, b & 1, stream=se.cuda_stream)
        se.synchronize()

    def timed(fn, reps):
        ts, out = [], None
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            ts.append(1e3 * (time.perf_counter() - t0))
        return statistics.median(ts), out

    for _ in range(max(1, args.warmup)):
        sequential()
        overlapped()
    reps = max(1, args.steps)
    with ClockSampler(0) as clk:
        t_exp, _ = timed(explore_only, reps)
        t_seq, it_seq = timed(sequential, reps)
        t_ovl, it_ovl = timed(overlapped, reps)
    g_ovl = G.get_costs()
    sequential()
    same = bool(np.array_equal(G.get_costs(), g_ovl))
    G.close()
    X.close()
    line = {"experiment": "exploration overlapped with exploitation (Sec. VII)",
            "workload": f"6-D [-pi,pi]^6, 64 hyperspheres r~U[0.3,0.8], N={n}, each vertex joined "
                        f"to its {k} nearest predecessors, 16-point edge check, FP32 costs, "
                        f"blocks of {S}, Extend on the GPU",
            "unit": "ms per step (all blocks: Extend, insertion, exploitation to a stable policy)",
            "repeats": reps, "timing": "median wall time, host clock, device synchronised",
            "explore_only_ms": round(t_exp, 2), "sequential_ms": round(t_seq, 2),
            "overlapped_ms": round(t_ovl, 2), "saved_ms": round(t_seq - t_ovl, 2),
            "iterations": {"sequential": it_seq, "overlapped": it_ovl},
            "same_costs": same, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def run_reference(args) -> None:
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    rm = load_roadmap(args.workload, args.n, args.block, args.trial)
    per_step = args.cpu_seconds
    for _ in range(args.warmup):
        oracle_prefix(rm, per_step / 4)
    relax, secs, blocks = 0, 0.0, 0
    for _ in range(args.steps):
        r = oracle_prefix(rm, per_step)
        relax += r["relax"]
        secs += r["seconds"]
        blocks += r["blocks"]
    value = relax / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * secs / args.steps, 3),
        "ms_per_batch": round(1e3 * secs / blocks, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded roadmap generator)",
        "config": {"workload": f"{args.workload}: {WORKLOADS[args.workload][1]}",
                   "vertices": rm.n, "undirected_edges": rm.m},
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: serial policy iteration (Alg. 2) on the first "
                                   f"blocks of the schedule for ~{per_step:.0f} s "
                                   f"({blocks / args.steps:.1f} blocks per step)"},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def step_roofline(kbytes: dict, prof_steps: int, ms_per_step: float, peak: float) -> dict:
    """Algorithmic bytes of one step (Improve, Evaluate and insertion, counted
    over the profiled steps, which run the same schedule to the same trees)
    divided by the timed step time."""
    total = float(sum(v for v in kbytes.values() if v is not None)) / prof_steps
    gbs = total / (ms_per_step / 1e3) / 1e9 if ms_per_step > 0 else 0.0
    return {"algorithmic_bytes": int(total), "achieved": round(gbs, 1), "peak": peak,
            "unit": "GB/s", "frac": round(gbs / peak, 4),
            "note": "every phase's algorithmic bytes of one step over ms_per_step"}


def level_profile(prof: dict, clocks: dict) -> dict:
    """The top-down Evaluate's levels by size (from the profiled step): how
    many levels of each size bucket, the vertices they held, and the time of
    one level (CTA 0's clock from a level's start to the next one's, the grid
    barrier included), converted with the SM clock sampled under load."""
    mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    to_us = lambda cyc: cyc / mhz
    rows = []
    for b, (n, items, cyc) in enumerate(zip(prof["level_count"], prof["level_vertices"],
                                            prof["level_cycles"])):
        if n:
            lo = 1 << (b - 1) if b > 0 else 0
            rows.append({"vertices_lo": lo, "vertices_hi": (1 << b) - 1, "levels": n,
                         "vertices": items, "us_total": round(to_us(cyc), 1),
                         "us_per_level": round(to_us(cyc) / n, 2)})
    calls = prof["wave_calls"]

    def tiles(kind):
        out = []
        for b, (n, items, cyc) in enumerate(zip(prof[f"{kind}_tiles"], prof[f"{kind}_vertices"],
                                                prof[f"{kind}_cycles"])):
            if n:
                out.append({"vertices_lo": 1 << (b - 1) if b > 0 else 0, "tiles": n,
                            "vertices": items, "us_per_tile": round(to_us(cyc) / n, 2)})
        return out
    return {"sm_mhz": mhz, "wave_launches": calls, "buckets": rows,
            "cta0_share_tiles": tiles("share"), "cta0_local_tiles": tiles("local"),
            "levels_us_total": round(to_us(sum(prof["level_cycles"])), 1),
            "pre_us_total": round(to_us(prof["wave_pre_cycles"]), 1),
            "post_us_total": round(to_us(prof["wave_post_cycles"]), 1),
            "jump_finish_us_total": round(to_us(prof["wave_jump_cycles"]), 1),
            "note": "pre: Improve from offers and its grid barrier inside the wave launch; "
                    "post: after the last level; jump_finish: pointer jumping after a level cap"}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["c4", "sweep", "explore"],
                    default="c3")
    ap.add_argument("--graphs", type=int, default=512, help="members of the batched workload")
    ap.add_argument("--tune-trials", type=int, default=40,
                    help="batched workload: exploits the searching autotuner may run")
    ap.add_argument("--n", type=int, default=None, help="override the vertex count")
    ap.add_argument("--block", type=int, default=None, help="override the block size S")
    ap.add_argument("--trial", type=int, default=0)
    ap.add_argument("--group", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--dense-fraction", type=float, default=0.0)
    ap.add_argument("--evaluate", choices=("auto", "wave", "jump", "async"), default="auto")
    ap.add_argument("--wave-levels", type=int, default=0)
    ap.add_argument("--wave-ctas", type=int, default=0, help="wave CTAs per SM (0 tuned)")
    ap.add_argument("--wave-tail", type=int, default=0,
                    help="levels of at most this many vertices walked by one CTA (0 tuned, <0 off)")
    ap.add_argument("--wave-local", type=int, default=0,
                    help="tree levels a CTA walks on its own per grid step (0 tuned, <0 none)")
    ap.add_argument("--wave-local-max", type=int, default=0,
                    help="local walks go on while the local list holds at most this many (0 tuned)")
    ap.add_argument("--wave-local-step", type=int, default=0,
                    help="local walks only in grid steps of at most this many vertices (0 tuned)")
    ap.add_argument("--timing", choices=("graph", "profiled"), default="graph")
    ap.add_argument("--profile-steps", type=int, default=1)
    ap.add_argument("--host-loop", action="store_true",
                    help="run every exploit from the host loop (no CUDA graphs), e.g. under ncu")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-dijkstra", action="store_true",
                    help="skip the oracle Dijkstra (O2) baseline on the final graph")
    ap.add_argument("--goal", choices=("none", "far"), default=None,
                    help="goal-directed Replan toward the sample opposite x_init (default: "
                         "none, except for the sweep's query)")
    ap.add_argument("--sweep-n", default="10000,30000", help="sweep: vertex counts")
    ap.add_argument("--sweep-s", default=",".join(str(x) for x in SWEEP_S),
                    help="sweep: block sizes")
    ap.add_argument("--sweep-legs", default="gpu,oracle", help="sweep: gpu, oracle or both")
    ap.add_argument("--no-prefetch", action="store_true",
                    help="end-to-end pass: copy each block when it is inserted, not during the "
                         "previous exploit")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the end-to-end pass (e.g. for a profiler's launch list)")
    ap.add_argument("--trace", default=None, help="save the per-iteration trace (.npy)")
    ap.add_argument("--traffic-block", type=int, default=None,
                    help="mark this block's exploit with the NVTX range 'traffic_window' while "
                         "profiling and report its Evaluate calls and algorithmic bytes "
                         "(negative: from the end)")
    args = ap.parse_args()
    if args.workload == "sweep":
        if args.impl == "reference":
            args.sweep_legs = "oracle"
        run_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    elif args.workload == "c4":
        run_batch(args)
    elif args.workload == "explore":
        run_explore(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
