#!/usr/bin/env python
"""Benchmark: exact per-pattern hyper-triangle counting on one synthetic workload.

A step is one pass of the whole path over one hypergraph already resident in
HBM: load/validate/transpose (hg_load_csr from device pointers), hyperwedge
construction and orientation (hg_build_wedges), closure + classification +
reduction (hg_count_patterns) and the clustering coefficient
(hg_clustering_coeff).  `value` is hyper-triangles classified per second over
K timed steps (CUDA events on the library's stream, L2 flushed between steps
outside the events).  `e2e` is the same through the C ABI from pinned HOST
buffers, the host->device copy of the CSR and the device->host read of the
counts inside the timed region.

--impl reference times the CPU oracle (the plain Exact-bs-shaped enumeration)
on the host cores, on a bounded sample of the same workload per step.

Multi-GPU: the path has no exchange step across hypergraphs, so N GPUs run N
independent replicas (one process each, launched by torchrun); `value` is the
sum of their work divided by the slowest rank's time.
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

METRIC = "hyper-triangles classified/s (exact per-pattern counts); HBM GB/s vs peak"
UNIT = "hyper-triangles/s"
L2_FLUSH_BYTES = 256 << 20


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="coauthor")
    ap.add_argument("--skip-cpu-baseline", action="store_true")
    ap.add_argument("--close-mode", type=int, default=0,
                    help="hg_tuning.close_mode (1: every closing team on the global-table kernel)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="build with the default tuning instead of hg_autotune's choice")
    ap.add_argument("--cpu-sample-edges", type=int, default=8000,
                    help="hyperedges whose owned triangles the CPU baseline counts")
    ap.add_argument("--e2e-steps", type=int, default=-1,
                    help="end-to-end steps from host buffers (-1: as many as --steps on the "
                         "default workload, 3 on the others)")
    ap.add_argument("--dense-min-size", type=int, default=0,
                    help="hyperedges at least this large use the tensor-core tiles (0 auto, -1 off)")
    ap.add_argument("--dense-max-count", type=int, default=0,
                    help="cap on the tensor-core set (0 = 1%% of |E|)")
    ap.add_argument("--batch-members", type=int, default=4096,
                    help="--workload batched: members (seeds 100 ..) in the batch")
    ap.add_argument("--per-graph-steps", type=int, default=2,
                    help="--workload batched: timed steps of the one-handle-per-hypergraph form")
    ap.add_argument("--queries", type=int, default=10_000, help="--workload served: stream length")
    ap.add_argument("--rate", type=float, default=2000.0,
                    help="--workload served: Poisson arrival rate (queries/s)")
    ap.add_argument("--plain-queries", type=int, default=1000,
                    help="--workload served: queries replayed with batching off")
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--samples", type=int, default=10_000_000,
                    help="--workload sample: draws per step")
    return ap.parse_args()


# ------------------------------------------------------------------ workload

def workload(name):
    import hgen

    if name in hgen.WORKLOADS:
        spec = hgen.WORKLOADS[name]
        e_ptr, e_idx = hgen.generate(spec)
        return spec, e_ptr, e_idx, None
    base, _, pre = name.partition("_prefix")
    spec = hgen.WORKLOADS[base]
    e_ptr, e_idx = hgen.generate(spec)
    e_ptr, e_idx = hgen.prefix(e_ptr, e_idx, int(pre))
    return spec, e_ptr, e_idx, int(pre)


def workload_config(spec, e_ptr, prefix):
    dist = {0: f"uniform on [{spec.size_lo},{spec.size_hi}]",
            1: f"truncated power law {spec.size_p1} on [{spec.size_lo},{spec.size_hi}]",
            2: f"log-normal({spec.size_p1},{spec.size_p2}) clipped to [{spec.size_lo},{spec.size_hi}]"}
    return {"workload": spec.name + (f"_prefix{prefix}" if prefix else ""),
            "num_vertices": spec.num_vertices, "num_edges": len(e_ptr) - 1,
            "nnz": int(e_ptr[-1]), "hyperedge_sizes": dist[spec.size_dist],
            "vertex_popularity": f"Zipf({spec.zipf_s})", "degree_cap": spec.degree_cap,
            "seed": spec.seed}


def golden_counts(cfg_name):
    path = os.path.join(ROOT, "tests", "golden", "workloads.json")
    try:
        with open(path) as f:
            return json.load(f).get(cfg_name)
    except OSError:
        return None


# ------------------------------------------------------------------ clocks

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={CLOCK_QUERY}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu), "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
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
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ roofline inputs

def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def measured_tensor_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        return 1900.0


def source_sha(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def profiled_traffic(kernel, workload_name, units=None):
    """DRAM bytes per launch from the committed ncu summary, if the kernel source is unchanged.

    Entries captured on a smaller launch store bytes per unit (`dram_bytes_per_sample`);
    they are scaled by the `units` of the measured launch."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    e = d.get(f"{kernel}/{workload_name}")
    if not e:
        return None
    src = os.path.join(ROOT, "paper_2504_02271_gb300", "csrc", e["source"])
    if not os.path.exists(src) or source_sha(src) != e["source_sha"]:
        return None
    if "dram_bytes_per_sample" in e:
        return None if units is None else round(float(e["dram_bytes_per_sample"]) * units)
    return float(e["dram_bytes_per_launch"])


# team shape of each closure kernel group -> index of its work counters
CLOSE_GROUPS = {"close_warp256": 0, "close_warp512": 1, "close_warp1024": 2, "close_block2048": 3,
                "close_block4096": 4, "close_block8192": 5, "close_wide": 6, "close_cluster": 7}
ISSUE_LANE_OPS_PER_CYCLE_PER_SM = 4 * 32   # 4 schedulers, one 32-lane instruction per cycle


def dram_rate(traffic, launch_ms, peak_gbs):
    """DRAM GB/s of a launch from captured traffic (bytes per launch) and its live duration."""
    if not traffic or not launch_ms or launch_ms <= 0:
        return {}
    gbs = float(traffic) / (launch_ms / 1000.0) / 1e9
    return {"dram_achieved": round(gbs, 1), "dram_frac": round(gbs / peak_gbs, 4),
            "dram_source": "ncu dram__bytes_read + dram__bytes_write of the committed capture"
                           " / live launch time"}


def close_algorithmic(cs, b, T):
    """Algorithmic work of the closure kernels of team shape b in one launch.

    Per probe (an entry of out(v) looked up in u's table): 4 bytes read, 8 integer
    operations (decode 2, two hashes 2, two slot compares 4).  Per out-entry of u:
    20 bytes (entry, row start, out-degree, |e_x|) and 10 operations (table insert).
    Per E_y entry read for the vertex masks: 4 bytes and 8 operations.  Per
    hyper-triangle: 27 operations (index and mask loads 5, seven region tests 20,
    histogram 2); the triangles of shape b are taken in proportion to its probes.
    """
    probes, gathers, outs = cs["bucket_probes"][b], cs["bucket_gathers"][b], cs["bucket_out_entries"][b]
    hits = T * probes / max(cs["probes"], 1)
    nbytes = 4 * probes + 20 * outs + 4 * gathers
    ops = 8 * probes + 10 * outs + 8 * gathers + 27 * hits
    return nbytes, ops


# ------------------------------------------------------------------ multi-rank aggregation

def aggregate(units: float, seconds: float, dist=None, device=None):
    """Whole-job (units, seconds): units summed over ranks, time = slowest rank.

    The ranks are independent replicas (no exchange step in the counting path), so
    the job's throughput is all ranks' work over the time of the last one to finish.
    """
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(units), float(seconds)
    import torch

    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()), float(t.item())


# ------------------------------------------------------------------ our arm

def run_ours(args):
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    import paper_2504_02271_gb300 as hg

    hg.use_torch_allocator()
    spec, e_ptr, e_idx, prefix = workload(args.workload)
    cfg = workload_config(spec, e_ptr, prefix)
    nv, ne = spec.num_vertices, len(e_ptr) - 1
    gold = golden_counts(cfg["workload"])

    stream = torch.cuda.Stream()
    d_ptr = torch.from_numpy(e_ptr).to(dev)
    d_idx = torch.from_numpy(e_idx).to(dev)
    h_ptr = torch.from_numpy(e_ptr).pin_memory()
    h_idx = torch.from_numpy(e_idx).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ones = [1.0] * 20
    torch.cuda.synchronize()

    tuning = {"dense_min_size": args.dense_min_size, "dense_max_count": args.dense_max_count,
              "close_mode": args.close_mode}

    def one_step(p, i, timing=False):
        g = hg.hg_load_csr(nv, ne, p, i, stream=stream.cuda_stream)
        try:
            if timing:
                hg.hg_set_timing(g, True)
            st = hg.hg_build_wedges(g, **tuning)
            counts = hg.hg_count_patterns(g)
            cc = hg.hg_clustering_coeff(g, ones)
            kt = hg.hg_kernel_times(g) if timing else {}
            cs = hg.hg_close_stats_get(g)
        finally:
            hg.hg_free(g)
        return counts, st, cc, kt, cs

    def do_flush(k):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)

    # warm-up (also the parity check against the stored oracle values)
    counts = st = cs = None
    for k in range(args.warmup):
        do_flush(k)
        counts, st, _, _, cs = one_step(d_ptr, d_idx)
    parity = None
    if gold is not None and counts is not None:
        parity = counts.tolist() == gold["counts"] and st["W"] == gold["W"]
        if not parity:
            raise SystemExit(f"bench: counts differ from the stored oracle values: {counts.tolist()}")
    # autotune once (warm-up): the timed steps build with its choice
    tune = None
    if not args.no_autotune and not (args.dense_min_size or args.dense_max_count or args.close_mode):
        g = hg.hg_load_csr(nv, ne, d_ptr, d_idx, stream=stream.cuda_stream)
        try:
            tune = hg.hg_autotune(g)
        finally:
            hg.hg_free(g)
        tuning = tune["best"]
        one_step(d_ptr, d_idx)

    def barrier():
        if dist is not None:
            dist.barrier()

    # timed region: device-resident inputs, K steps with no per-kernel events (value),
    # then K more steps with CUDA events around every launch (per-kernel durations for
    # the roofline), both under the clock sampler
    clocks = ClockSampler(dev)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    launches0 = hg.hg_kernel_launches()
    step_ms, kernel_ms = [], {}
    tri = 0
    for k in range(args.steps):
        do_flush(k + 17)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        counts, st, cc, kt, cs = one_step(d_ptr, d_idx)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        tri += int(counts[0])
    torch.cuda.synchronize()
    launches = hg.hg_kernel_launches() - launches0
    barrier()
    for k in range(args.steps):
        do_flush(k + 57)
        c3, _, _, kt, _ = one_step(d_ptr, d_idx, timing=True)
        assert c3.tolist() == counts.tolist()
        for name, (ms, n) in kt.items():
            a = kernel_ms.setdefault(name, [0.0, 0])
            a[0] += ms
            a[1] += n
    torch.cuda.synchronize()
    clk = clocks.stop()

    tri_all, total_s = aggregate(float(tri), sum(step_ms) / 1000.0, dist, dev)
    value = tri_all / total_s

    # end to end through the C ABI from pinned host buffers (--e2e-steps 0 skips it)
    e2e_ms = []
    for k in range(args.steps if args.e2e_steps < 0 else args.e2e_steps):
        do_flush(k + 99)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        c2, _, _, _, _ = one_step(h_ptr, h_idx)
        e1.record(stream)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        assert c2.tolist() == counts.tolist()
    e2e_value = None
    if e2e_ms:
        e2e_units, e2e_s = aggregate(float(int(counts[0]) * len(e2e_ms)), sum(e2e_ms) / 1000.0,
                                     dist, dev)
        e2e_value = e2e_units / e2e_s

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel (the closure kernel with the largest share)
    peak_hbm, peak_kind = measured_peaks()
    groups = {n: v for n, v in kernel_ms.items() if n in CLOSE_GROUPS}
    dom = max(groups, key=lambda n: groups[n][0])
    dom_ms = groups[dom][0] / groups[dom][1]            # average launch duration
    nbytes, ops = close_algorithmic(cs, CLOSE_GROUPS[dom], int(counts[0]))
    sm_mhz = ((clk or {}).get("sm_mhz") or 2070.0)
    peak_ops = 152 * ISSUE_LANE_OPS_PER_CYCLE_PER_SM * sm_mhz * 1e6 / 1e12   # Tops/s
    achieved_ops = ops / (dom_ms / 1000.0) / 1e12
    achieved_gbs = nbytes / (dom_ms / 1000.0) / 1e9
    traffic = profiled_traffic(dom, cfg["workload"])
    roof = {"bound": "alu", "kernel": f"{dom} (k_close_warp / k_close_block / k_close_wide / k_close_cluster)",
            "achieved": round(achieved_ops, 3), "peak": round(peak_ops, 2), "unit": "Tops/s",
            "frac": round(achieved_ops / peak_ops, 4),
            "peak_source": f"derived: 152 SMs x 128 lane-ops/cycle x {sm_mhz:.0f} MHz (median SM clock under load)",
            "algorithmic_ops_per_launch": int(ops), "algorithmic_bytes_per_launch": int(nbytes),
            "launch_ms": round(dom_ms, 4), "traffic": traffic,
            "hbm": {"achieved": round(achieved_gbs, 1), "peak": peak_hbm, "unit": "GB/s",
                    "frac": round(achieved_gbs / peak_hbm, 4), "peak_source": peak_kind}}
    roof["hbm"].update(dram_rate(traffic, dom_ms, peak_hbm))

    dense = None
    if "dense_omega" in kernel_ms and st["dense_edges"]:
        # algorithmic work of the tile product: 2 * nh * nh * |V| (multiply-adds of A A^T)
        nh = st["dense_edges"]
        flops = 2.0 * nh * nh * nv
        d_ms = kernel_ms["dense_omega"][0] / kernel_ms["dense_omega"][1]
        bf16 = measured_tensor_peak()
        peak = bf16 * 2.0   # e4m3 dense rate = 2x bf16 (4.5 vs 2.25 PFLOP/s nominal)
        ach = flops / (d_ms / 1000.0) / 1e12
        dense = {"bound": "tensor", "kernel": "dense_omega (k_dense_omega, tcgen05 kind::f8f6f4)",
                 "achieved": round(ach, 1), "peak": round(peak, 1), "unit": "TFLOP/s",
                 "frac": round(ach / peak, 4),
                 "peak_source": "measured bf16 burst x 2 (nominal e4m3/bf16 ratio)",
                 "rows": nh, "k": nv, "launch_ms": round(d_ms, 4),
                 "traffic": profiled_traffic("dense_omega", cfg["workload"])}

    cpu = None
    if world == 1 and not args.skip_cpu_baseline:
        cpu = cpu_baseline(e_ptr, e_idx, nv, args.cpu_sample_edges)

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(statistics.mean(step_ms), 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": dict(cfg, triangles_per_step=int(counts[0]), wedges=st["W"],
                       l2="256 MiB buffer written between steps, outside the per-step events",
                       kernel_timing="per-launch CUDA events in K further steps after the K "
                                     "steps that give value (those run without them)",
                       inputs="int64/int32 CSR resident in HBM", parallelism=f"replicas x{world}",
                       parity="counts equal stored oracle values" if parity else (
                           "no stored oracle values at this size; sampled owners of every team "
                           "shape are compared with the oracle in tests/test_gpu_owned.py"
                           if cfg["workload"] == "tag_heavy" else "not checked"),
                       dense_tiles={"min_size": tuning["dense_min_size"],
                                    "max_count": tuning["dense_max_count"],
                                    "hyperedges": st["dense_edges"]},
                       tuning=tuning,
                       autotune=None if tune is None else {
                           "candidates": len(tune["tried"]),
                           "ms": [round(x, 3) for x in tune["ms"]],
                           "default_ms": round(tune["ms"][0], 3),
                           "chosen_ms": round(tune["best_ms"], 3),
                           "all_candidates_equal_counts": bool(all(
                               c.tolist() == tune["counts"][0].tolist() for c in tune["counts"]))}),
        "e2e": None if e2e_value is None else {
            "value": round(e2e_value, 1), "unit": UNIT,
            "h2d_bytes_per_step": int(e_ptr.nbytes + e_idx.nbytes),
            "d2h_bytes_per_step": 21 * 8 + 8 * 8,
            "ms_per_step": round(statistics.mean(e2e_ms), 4)},
        "roofline": roof,
        "dense_roofline": dense,
        "kernel_ms_per_step": {n: round(v[0] / args.steps, 4) for n, v in sorted(kernel_ms.items())},
        "gpu_launches": int(launches),
        "clocks": clk,
        "cpu_baseline": cpu,
        "counts": [int(x) for x in counts],
        "close_stats": cs,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# ------------------------------------------------------------------ batches of hypergraphs

def roofline_from_times(kernel_ms, cs, T, clk, steps):
    """ALU roofline of the closure kernel with the largest share (see close_algorithmic).

    kernel_ms holds (summed ms, launches) over `steps` steps; cs and T are one step's
    work, which that kernel does in launches / steps launches (one per wave)."""
    peak_hbm, peak_kind = measured_peaks()
    groups = {n: v for n, v in kernel_ms.items() if n in CLOSE_GROUPS}
    dom = max(groups, key=lambda n: groups[n][0])
    dom_ms = groups[dom][0] / groups[dom][1]            # average launch duration
    per_step = groups[dom][1] / steps                   # launches of it in one step
    nbytes, ops = close_algorithmic(cs, CLOSE_GROUPS[dom], T)
    nbytes, ops = nbytes / per_step, ops / per_step     # per launch
    sm_mhz = ((clk or {}).get("sm_mhz") or 2070.0)
    peak_ops = 152 * ISSUE_LANE_OPS_PER_CYCLE_PER_SM * sm_mhz * 1e6 / 1e12
    achieved_ops = ops / (dom_ms / 1000.0) / 1e12
    achieved_gbs = nbytes / (dom_ms / 1000.0) / 1e9
    return {"bound": "alu", "kernel": f"{dom} (k_close_warp / k_close_block / k_close_wide)",
            "achieved": round(achieved_ops, 3), "peak": round(peak_ops, 2), "unit": "Tops/s",
            "frac": round(achieved_ops / peak_ops, 4),
            "peak_source": f"derived: 152 SMs x 128 lane-ops/cycle x {sm_mhz:.0f} MHz (median SM clock under load)",
            "algorithmic_ops_per_launch": int(ops), "algorithmic_bytes_per_launch": int(nbytes),
            "launch_ms": round(dom_ms, 4), "traffic": None,
            "hbm": {"achieved": round(achieved_gbs, 1), "peak": peak_hbm, "unit": "GB/s",
                    "frac": round(achieved_gbs / peak_hbm, 4), "peak_source": peak_kind}}


def run_batched(args):
    """4,096 independent hypergraphs (|E| log-uniform in [100, 200000], |V| = |E|/4,
    sizes power law 2.2 on [2, 50], Zipf(1.0), degree cap 100, seeds 100 ..): one
    batch (hg_load_batch / hg_batch_*) against one handle per hypergraph."""
    import numpy as np
    import torch

    import hgen

    if int(os.environ.get("WORLD_SIZE", "1")) > 1:
        raise SystemExit("bench: --workload batched runs on one GPU (replicas: run one per GPU)")
    torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    import paper_2504_02271_gb300 as hg

    hg.use_torch_allocator()
    G = args.batch_members
    specs = [hgen.batched(s) for s in range(100, 100 + G)]
    nv, eoff, eptr, evtx, used = hgen.generate_batch(specs, redraw=hgen.batched_redraw)
    redrawn = [u.name for u in used if u.seed >= 2**32]
    stream = torch.cuda.Stream()
    d_ptr = torch.from_numpy(eptr).to(dev)
    d_idx = torch.from_numpy(evtx).to(dev)
    h_ptr = torch.from_numpy(eptr).pin_memory()
    h_idx = torch.from_numpy(evtx).pin_memory()
    # per-member device CSRs for the one-handle-per-hypergraph form (offsets from 0)
    m_ptr = [torch.from_numpy(np.ascontiguousarray(eptr[eoff[m]:eoff[m + 1] + 1] - eptr[eoff[m]])).to(dev)
             for m in range(G)]
    m_idx = [d_idx[int(eptr[eoff[m]]):int(eptr[eoff[m + 1]])] for m in range(G)]
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ones = [1.0] * 20
    torch.cuda.synchronize()

    def do_flush(k):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)

    tuning = {}

    def batch_step(p, i, timing=False):
        b = hg.hg_load_batch(nv, eoff, p, i, stream=stream.cuda_stream)
        try:
            waves = hg.hg_batch_waves(b)
            if timing:
                for w in waves:
                    hg.hg_set_timing(w[0], True)
            hg.hg_batch_build_wedges(b, **tuning)
            counts, stats = hg.hg_batch_count_patterns(b)
            cc = hg.hg_batch_clustering_coeff(b, ones)
            kt, cs = {}, None
            for w in waves:
                if timing:
                    for n, (ms, c) in hg.hg_kernel_times(w[0]).items():
                        a = kt.setdefault(n, [0.0, 0])
                        a[0] += ms
                        a[1] += c
                one = hg.hg_close_stats_get(w[0])
                if cs is None:
                    cs = one
                else:
                    for k, v in one.items():
                        cs[k] = [x + y for x, y in zip(cs[k], v)] if isinstance(v, list) else cs[k] + v
        finally:
            hg.hg_batch_free(b)
        return counts, stats, cc, kt, cs, len(waves)

    def per_graph_step():
        out = np.zeros((G, 21), dtype=np.uint64)
        for m in range(G):
            g = hg.hg_load_csr(int(nv[m]), int(eoff[m + 1] - eoff[m]), m_ptr[m], m_idx[m],
                               stream=stream.cuda_stream)
            try:
                hg.hg_build_wedges(g, **tuning)
                out[m] = hg.hg_count_patterns(g)
                hg.hg_clustering_coeff(g, ones)
            finally:
                hg.hg_free(g)
        return out

    def timed(fn, k):
        do_flush(k)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1)

    counts = None
    tune = None
    for k in range(args.warmup):
        do_flush(k)
        counts, stats, _, _, _, nwaves = batch_step(d_ptr, d_idx)
        if k == 0 and not args.no_autotune:   # autotune on the largest wave, then use it
            b = hg.hg_load_batch(nv, eoff, d_ptr, d_idx, stream=stream.cuda_stream)
            try:
                tune = hg.hg_batch_autotune(b)
            finally:
                hg.hg_batch_free(b)
            tuning = tune["best"]
    T = int(counts[:, 0].sum())

    # timed region: K steps without per-kernel events (value), then K with them (roofline)
    clocks = ClockSampler(dev)
    torch.cuda.synchronize()
    clocks.start()
    launches0 = hg.hg_kernel_launches()
    step_ms, kernel_ms, cs = [], {}, None
    for k in range(args.steps):
        (c2, _, _, _, cs, _), ms = timed(lambda: batch_step(d_ptr, d_idx), k + 17)
        assert np.array_equal(c2, counts)
        step_ms.append(ms)
    torch.cuda.synchronize()
    launches = hg.hg_kernel_launches() - launches0
    for k in range(args.steps):
        (c2, _, _, kt, _, _), _ = timed(lambda: batch_step(d_ptr, d_idx, timing=True), k + 47)
        assert np.array_equal(c2, counts)
        for n, (t, c) in kt.items():
            a = kernel_ms.setdefault(n, [0.0, 0])
            a[0] += t
            a[1] += c
    torch.cuda.synchronize()
    clk = clocks.stop()
    value = T * len(step_ms) / (sum(step_ms) / 1000.0)

    # the same members one handle at a time: identical counts, and its throughput
    pg_counts, _ = timed(per_graph_step, 5)   # warm-up
    if not np.array_equal(pg_counts, counts):
        raise SystemExit("bench: batch counts differ from one-handle-per-hypergraph counts")
    launches_pg0 = hg.hg_kernel_launches()
    pg_ms = [timed(per_graph_step, 40 + k)[1] for k in range(max(1, args.per_graph_steps))]
    launches_pg = (hg.hg_kernel_launches() - launches_pg0) // len(pg_ms)
    pg_value = T * len(pg_ms) / (sum(pg_ms) / 1000.0)

    # end to end from pinned host buffers (upload inside the timed region)
    e2e_ms = []
    for k in range(max(1, args.e2e_steps if args.e2e_steps >= 0 else 3)):
        (c3, _, _, _, _, _), ms = timed(lambda: batch_step(h_ptr, h_idx), 99 + k)
        assert np.array_equal(c3, counts)
        e2e_ms.append(ms)
    e2e_value = T * len(e2e_ms) / (sum(e2e_ms) / 1000.0)

    roof = roofline_from_times(kernel_ms, cs, T, clk, args.steps)
    cpu = None
    if not args.skip_cpu_baseline:
        import oracle

        # bounded sample: whole members in seed order until about 15 s of oracle time
        tri, secs, threads, done = 0, 0.0, 1, 0
        for m in range(G):
            if secs > 15.0:
                break
            p = eptr[eoff[m]:eoff[m + 1] + 1] - eptr[eoff[m]]
            r = oracle.count(p, evtx[eptr[eoff[m]]:eptr[eoff[m + 1]]], int(nv[m]))
            if r.counts.tolist() != counts[m].tolist():
                raise SystemExit(f"bench: member {m} differs from the oracle")
            tri, secs, threads, done = tri + r.T, secs + r.seconds, r.threads, m + 1
        cpu = {"value": round(tri / secs, 1), "unit": UNIT, "cores": threads, "kind": "oracle",
               "seconds": round(secs, 2), "triangles": tri,
               "sample": f"members 0..{done - 1} of the batch, each counted whole (counts equal the GPU's)"}

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(statistics.mean(step_ms), 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"batched_{G}", "members": G, "seeds": f"100..{99 + G}",
                   "member_edges": "log-uniform in [100, 200000]", "member_vertices": "|E|/4",
                   "hyperedge_sizes": "truncated power law 2.2 on [2,50]",
                   "vertex_popularity": "Zipf(1.0)", "degree_cap": 100,
                   "redrawn_members": redrawn, "sum_edges": int(eoff[-1]), "sum_nnz": int(eptr[-1]),
                   "waves": nwaves, "triangles_per_step": T,
                   "wedges": int(stats["W"].sum()),
                   "l2": "inputs (%.1f GB) larger than L2; 256 MiB buffer also written between steps"
                         % ((eptr.nbytes + evtx.nbytes) / 1e9),
                   "inputs": "concatenated int64/int32 CSRs resident in HBM",
                   "parallelism": "replicas x1",
                   "parity": "per-member counts equal one-handle-per-hypergraph counts",
                   "tuning": tuning or "defaults",
                   "autotune": None if tune is None else {
                       "wave": "the wave with the most hyperedges",
                       "candidates": len(tune["tried"]), "ms": [round(x, 2) for x in tune["ms"]],
                       "chosen": tune["best"],
                       "all_candidates_equal_counts": bool(all(
                           c.tolist() == tune["counts"][0].tolist() for c in tune["counts"]))}},
        "per_graph": {"value": round(pg_value, 1), "unit": UNIT, "ms_per_step": round(statistics.mean(pg_ms), 3),
                      "steps": len(pg_ms), "gpu_launches_per_step": int(launches_pg),
                      "form": "hg_load_csr / hg_build_wedges / hg_count_patterns / hg_clustering_coeff per member"},
        "e2e": {"value": round(e2e_value, 1), "unit": UNIT,
                "h2d_bytes_per_step": int(eptr.nbytes + evtx.nbytes),
                "d2h_bytes_per_step": int(G * 21 * 8 + G * 64),
                "ms_per_step": round(statistics.mean(e2e_ms), 3)},
        "roofline": roof,
        "kernel_ms_per_step": {n: round(v[0] / args.steps, 3) for n, v in sorted(kernel_ms.items())},
        "gpu_launches": int(launches),
        "clocks": clk,
        "cpu_baseline": cpu,
        "close_stats": cs,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ sampling (Algorithms 6-7)

def run_sample(args):
    """Hyperwedge sampling on the co-authorship workload: a step is one
    hg_sample_estimate call of --samples draws (Algorithm 6) on a handle whose step one
    is built; Appro-adv (Algorithm 7) is timed the same way beside it."""
    import numpy as np
    import torch

    import oracle

    torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    import paper_2504_02271_gb300 as hg

    hg.use_torch_allocator()
    spec, e_ptr, e_idx, prefix = workload("coauthor")
    cfg = workload_config(spec, e_ptr, prefix)
    nv, ne, N = spec.num_vertices, len(e_ptr) - 1, args.samples
    stream = torch.cuda.Stream()
    d_ptr, d_idx = torch.from_numpy(e_ptr).to(dev), torch.from_numpy(e_idx).to(dev)
    h_ptr, h_idx = torch.from_numpy(e_ptr).pin_memory(), torch.from_numpy(e_idx).pin_memory()
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    g = hg.hg_load_csr(nv, ne, d_ptr, d_idx, stream=stream.cuda_stream)
    st = hg.hg_build_wedges(g)

    def timed(fn, k):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xFF)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        e1.synchronize()
        return r, e0.elapsed_time(e1)

    seed = 2024
    for k in range(args.warmup):   # the first call also builds the sorted upper rows
        hg.hg_sample_estimate(g, seed, k * N, N)
        hg.hg_sample_estimate_adv(g, seed, k * N, N)
    # parity: a sub-range of draws against the oracle, bit for bit
    check_n = 200_000
    raw, est = hg.hg_sample_estimate(g, seed, 0, check_n)
    ref = oracle.sample_estimate(e_ptr, e_idx, nv, seed=seed, first=0, num=check_n)
    araw, aest, _ = hg.hg_sample_estimate_adv(g, seed, 0, check_n)
    aref = oracle.sample_estimate_adv(e_ptr, e_idx, nv, seed=seed, first=0, num=check_n)
    if raw.tolist() != ref.raw.tolist() or est.tolist() != ref.est.tolist() or \
            araw.tolist() != aref.raw.tolist() or aest.tolist() != aref.est.tolist():
        raise SystemExit("bench: sampled estimates differ from the oracle")

    clocks = ClockSampler(dev)
    torch.cuda.synchronize()
    clocks.start()
    launches0 = hg.hg_kernel_launches()
    hg.hg_set_timing(g, True)
    bs_ms, adv_ms, kernel_ms, work, tri = [], [], {}, np.zeros(3), 0
    for k in range(args.steps):
        (r, _), ms = timed(lambda: hg.hg_sample_estimate(g, seed, (100 + k) * N, N), 17 + k)
        bs_ms.append(ms)
        tri += int(r[0])
        w = hg.hg_sample_work_get(g)
        work += [w["ptr_reads"], w["entry_reads"], w["vertex_reads"]]
        for n, (t, c) in hg.hg_kernel_times(g).items():
            a = kernel_ms.setdefault(n, [0.0, 0])
            a[0] += t
            a[1] += c
    for k in range(args.steps):
        _, ms = timed(lambda: hg.hg_sample_estimate_adv(g, seed, (200 + k) * N, N), 40 + k)
        adv_ms.append(ms)
        for n, (t, c) in hg.hg_kernel_times(g).items():
            a = kernel_ms.setdefault(n, [0.0, 0])
            a[0] += t
            a[1] += c
    torch.cuda.synchronize()
    launches = hg.hg_kernel_launches() - launches0
    clk = clocks.stop()
    hg.hg_free(g)
    value = N * len(bs_ms) / (sum(bs_ms) / 1000.0)
    adv_value = N * len(adv_ms) / (sum(adv_ms) / 1000.0)

    # end to end from pinned host buffers: load, step one, sorted rows, N draws
    def e2e_step():
        h = hg.hg_load_csr(nv, ne, h_ptr, h_idx, stream=stream.cuda_stream)
        try:
            hg.hg_build_wedges(h)
            return hg.hg_sample_estimate(h, seed, 0, N)
        finally:
            hg.hg_free(h)
    e2e_ms = [timed(e2e_step, 90 + k)[1]
              for k in range(max(1, args.e2e_steps if args.e2e_steps >= 0 else 3))]

    # HBM view of the sampling kernel: the reads it made (row pointers 8 B, packed
    # entries 4 B, vertex ids 4 B) over its event-timed duration
    peak_hbm, peak_kind = measured_peaks()
    s_ms = kernel_ms["sample"][0] / kernel_ms["sample"][1]
    nbytes = (8 * work[0] + 4 * work[1] + 4 * work[2]) / args.steps
    roof = {"bound": "hbm", "kernel": "sample (k_sample)", "achieved": round(nbytes / s_ms / 1e6, 1),
            "peak": peak_hbm, "unit": "GB/s", "frac": round(nbytes / s_ms / 1e6 / peak_hbm, 4),
            "peak_source": peak_kind, "algorithmic_bytes_per_launch": int(nbytes),
            "launch_ms": round(s_ms, 4), "traffic": profiled_traffic("sample", "coauthor", N),
            "reads_per_sample": {"row_pointer": round(work[0] / args.steps / N, 2),
                                 "entries": round(work[1] / args.steps / N, 2),
                                 "vertex_ids": round(work[2] / args.steps / N, 2)},
            "note": "dependent random 4- and 8-byte reads (binary searches, row walks): "
                    "latency-bound gathers, mostly L2-resident"}
    cpu = None
    if not args.skip_cpu_baseline:
        n_cpu = 2_000_000
        t0 = time.perf_counter()
        oracle.sample_estimate(e_ptr, e_idx, nv, seed=seed, first=0, num=n_cpu)
        secs = time.perf_counter() - t0
        cpu = {"value": round(n_cpu / secs, 1), "unit": "samples/s", "cores": oracle._load().oracle_max_threads(),
               "kind": "oracle", "seconds": round(secs, 2),
               "sample": f"{n_cpu} draws of Algorithm 6 on the same hypergraph (including the "
                         f"oracle's own set-up of its wedge lists)"}
    line = {
        "metric": "hyperwedge samples/s (Algorithm 6, bit-exact with the oracle for the same sample indices)",
        "value": round(value, 1), "unit": "samples/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(statistics.mean(bs_ms), 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": dict(cfg, samples_per_step=N, wedges=st["W"], seed=seed,
                       l2="256 MiB buffer written between steps, outside the per-step events",
                       parity=f"draws 0..{check_n - 1} equal the oracle's (Algorithms 6 and 7)",
                       triangles_per_step=tri // args.steps),
        "appro_adv": {"value": round(adv_value, 1), "unit": "samples/s",
                      "ms_per_step": round(statistics.mean(adv_ms), 3)},
        "e2e": {"value": round(N * len(e2e_ms) / (sum(e2e_ms) / 1000.0), 1), "unit": "samples/s",
                "h2d_bytes_per_step": int(e_ptr.nbytes + e_idx.nbytes), "d2h_bytes_per_step": 21 * 16,
                "ms_per_step": round(statistics.mean(e2e_ms), 3),
                "note": "includes load, step one and the sorted upper rows"},
        "roofline": roof,
        "kernel_ms_per_step": {n: round(v[0] / args.steps, 4) for n, v in sorted(kernel_ms.items())},
        "gpu_launches": int(launches), "clocks": clk, "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving

def served_stream(n, n_graphs, rate, seed=5):
    """The query stream: Poisson arrivals at `rate`/s; kind and hypergraph uniform;
    estimates draw samples k*1e6 .. k*1e6 + 1e6 - 1 under seed 2024 (query k)."""
    import numpy as np

    rng = np.random.default_rng(seed)
    kinds = rng.integers(0, 3, n)
    gids = rng.integers(0, n_graphs, n)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n))
    qs = [{"kind": int(kinds[k]), "graph": int(gids[k]), "seed": 2024,
           "first_sample": k * 1_000_000, "num_samples": 1_000_000} for k in range(n)]
    return qs, arrivals


def serve_stream(hg, srv, ids, qs, arrivals, eps):
    """Submit at the arrival times from a producer thread; collect every answer."""
    import threading

    tickets = [None] * len(qs)

    def producer():
        t0 = time.perf_counter()
        for k, q in enumerate(qs):
            delay = arrivals[k] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            tickets[k] = srv.submit(q["kind"], ids[q["graph"]], q["seed"], q["first_sample"],
                                    q["num_samples"], eps)

    th = threading.Thread(target=producer)
    th.start()
    th.join()
    return [srv.wait(t) for t in tickets]


def latency_summary(res):
    import numpy as np

    lat = np.array([r["t_done"] - r["t_submit"] for r in res]) * 1000.0
    span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
    return {"queries": len(res), "seconds": round(span, 3), "queries_per_s": round(len(res) / span, 1),
            "p50_ms": round(float(np.percentile(lat, 50)), 2),
            "p99_ms": round(float(np.percentile(lat, 99)), 2),
            "max_ms": round(float(lat.max()), 2)}


def run_served(args):
    """64 resident hypergraphs (|E| log-uniform in [1000, 1000000], |V| = |E|/5, otherwise
    the co-authorship shape), a Poisson stream of queries answered by hg_server."""
    import numpy as np
    import torch

    import hgen
    import oracle

    torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    import paper_2504_02271_gb300 as hg

    n_graphs, n_queries, rate = 64, args.queries, float(args.rate)
    specs = [hgen.served(m) for m in range(n_graphs)]
    nv, eoff, eptr, evtx, _ = hgen.generate_batch(specs)
    gs = []
    for m in range(n_graphs):
        p = np.ascontiguousarray(eptr[eoff[m]:eoff[m + 1] + 1] - eptr[eoff[m]])
        gs.append((int(nv[m]), p, np.ascontiguousarray(evtx[eptr[eoff[m]]:eptr[eoff[m + 1]]])))
    qs, arrivals = served_stream(n_queries, n_graphs, rate)
    eps = [1.0] * 20

    # answers of the plain calls alone: exact ones per hypergraph (and the oracle's on
    # the small ones); estimates for a sample of the queries
    stream = torch.cuda.Stream()
    alone = {}
    for m, (n_v, p, i) in enumerate(gs):
        g = hg.hg_load_csr(n_v, len(p) - 1, p, i, stream=stream.cuda_stream)
        try:
            hg.hg_build_wedges(g)
            alone[m] = (hg.hg_count_patterns(g), hg.hg_clustering_coeff(g, eps))
        finally:
            hg.hg_free(g)
    small = [m for m in range(n_graphs) if len(gs[m][1]) - 1 <= 3000]
    for m in small:
        r = oracle.count(gs[m][1], gs[m][2], gs[m][0])
        if r.counts.tolist() != alone[m][0].tolist():
            raise SystemExit(f"bench: hypergraph {m} differs from the oracle")

    clocks = ClockSampler(dev)
    clocks.start()
    launches0 = hg.hg_kernel_launches()
    t_reg = time.perf_counter()
    srv = hg.Server(workers=args.serve_workers)
    ids = [srv.add_graph(n_v, p, i) for n_v, p, i in gs]      # host buffers -> device
    reg_s = time.perf_counter() - t_reg
    res = serve_stream(hg, srv, ids, qs, arrivals, eps)
    stats = srv.stats()
    srv.close()
    wall = time.perf_counter() - t_reg
    launches = hg.hg_kernel_launches() - launches0
    clk = clocks.stop()

    # every exact answer equals the plain calls'; a sample of estimates too, some the oracle's
    for q, r in zip(qs, res):
        if r["status"] != 0:
            raise SystemExit(f"bench: query failed with status {r['status']}")
        if q["kind"] != 2:
            c, (cc, op, co) = alone[q["graph"]]
            if r["counts"].tolist() != c.tolist() or (q["kind"] == 1 and not (
                    (np.isnan(cc) and np.isnan(r["cc"])) or cc == r["cc"])):
                raise SystemExit("bench: a served exact answer differs from the plain calls")
    est_idx = [k for k, q in enumerate(qs) if q["kind"] == 2]
    rng = np.random.default_rng(11)
    for k in rng.choice(est_idx, min(40, len(est_idx)), replace=False):
        q, r = qs[k], res[k]
        n_v, p, i = gs[q["graph"]]
        g = hg.hg_load_csr(n_v, len(p) - 1, p, i, stream=stream.cuda_stream)
        try:
            hg.hg_build_wedges(g)
            raw, est = hg.hg_sample_estimate(g, q["seed"], q["first_sample"], q["num_samples"])
        finally:
            hg.hg_free(g)
        if raw.tolist() != r["counts"].tolist() or est.tolist() != r["est"].tolist():
            raise SystemExit("bench: a served estimate differs from the plain call")
    checked_oracle = 0
    for k in est_idx:
        q = qs[k]
        if q["graph"] in small and checked_oracle < 3:
            n_v, p, i = gs[q["graph"]]
            ref = oracle.sample_estimate(p, i, n_v, seed=q["seed"], first=q["first_sample"],
                                         num=q["num_samples"])
            if ref.raw.tolist() != res[k]["counts"].tolist() or ref.est.tolist() != res[k]["est"].tolist():
                raise SystemExit("bench: a served estimate differs from the oracle")
            checked_oracle += 1

    summary = latency_summary(res)
    exact_batches = {}   # (worker, start time) of an exact batch -> its distinct hypergraphs
    for r in res:
        if r["kind"] != 2:
            exact_batches.setdefault((r["worker"], r["t_start"]), set()).add(r["graph"])
    computed_T = sum(int(alone[g][0][0]) for gset in exact_batches.values() for g in gset)
    answered_T = sum(int(r["counts"][0]) for q, r in zip(qs, res) if q["kind"] != 2)

    # the same stream's first queries with batching off (one worker, one query per batch)
    n_plain = min(args.plain_queries, n_queries)
    srv1 = hg.Server(workers=1, max_batch_queries=1)
    ids1 = [srv1.add_graph(n_v, p, i) for n_v, p, i in gs]
    res1 = serve_stream(hg, srv1, ids1, qs[:n_plain], arrivals[:n_plain], eps)
    srv1.close()
    for a, b in zip(res[:n_plain], res1):
        if a["counts"].tolist() != b["counts"].tolist() or a["est"].tolist() != b["est"].tolist():
            raise SystemExit("bench: answers differ between batched and unbatched serving")
    plain = latency_summary(res1)

    cpu = None
    if not args.skip_cpu_baseline:
        # the oracle answering the stream's queries in order, one at a time, for ~15 s;
        # exact queries on hypergraphs above 200,000 hyperedges are skipped (one of them
        # alone runs for minutes on the host)
        secs, done, skipped, threads = 0.0, 0, 0, 1
        t0 = time.perf_counter()
        for q in qs:
            if time.perf_counter() - t0 > 15.0:
                break
            n_v, p, i = gs[q["graph"]]
            if q["kind"] != 2 and len(p) - 1 > 200_000:
                skipped += 1
                continue
            if q["kind"] == 2:
                r = oracle.sample_estimate(p, i, n_v, seed=q["seed"], first=q["first_sample"],
                                           num=q["num_samples"])
            else:
                r = oracle.count(p, i, n_v)
                threads = r.threads
            done += 1
        secs = time.perf_counter() - t0
        cpu = {"value": round(done / secs, 3), "unit": "queries/s", "cores": threads,
               "kind": "oracle", "seconds": round(secs, 2),
               "sample": f"the stream's first {done} queries answered one at a time (skipping "
                         f"{skipped} exact queries on hypergraphs above 200,000 hyperedges)"}

    line = {
        "metric": "queries answered/s (exact counts, clustering coefficients, 1e6-sample estimates) with p50/p99 latency",
        "value": summary["queries_per_s"], "unit": "queries/s", "n_gpus": 1, "steps": 1, "warmup": 0,
        "ms_per_step": round(summary["seconds"] * 1000, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": "served", "graphs": n_graphs, "sum_edges": int(eoff[-1]),
                   "sum_nnz": int(eptr[-1]), "graph_edges": "log-uniform in [1000, 1000000]",
                   "graph_vertices": "|E|/5, co-authorship shape, degree cap 100",
                   "queries": n_queries, "arrivals": f"Poisson {rate:.0f}/s",
                   "mix": "1/3 counts, 1/3 clustering coefficient, 1/3 estimate (1e6 Philox samples)",
                   "workers": args.serve_workers,
                   "parity": "exact answers equal the plain calls (and the oracle on hypergraphs "
                             "with <= 3000 hyperedges); 40 estimates equal the plain call, 3 the oracle"},
        "latency": summary,
        "triangles": {"answered": answered_T, "computed": computed_T,
                      "computed_per_s": round(computed_T / summary["seconds"], 1)},
        "server": stats,
        "unbatched": dict(plain, note="same server, workers=1, max_batch_queries=1, the stream's first "
                                      f"{n_plain} queries at the same arrival times"),
        "e2e": {"value": round(n_queries / wall, 1), "unit": "queries/s",
                "h2d_bytes_per_step": int(eptr.nbytes + evtx.nbytes),
                "d2h_bytes_per_step": int(n_queries * 416), "registration_s": round(reg_s, 3),
                "seconds": round(wall, 3)},
        "roofline": None,
        "gpu_launches": int(launches),
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(e_ptr, e_idx, nv, sample_edges):
    import oracle

    lo, hi = 0, min(sample_edges, len(e_ptr) - 1)
    r = oracle.count(e_ptr, e_idx, nv, i_range=(lo, hi))
    return {"value": round(r.T / r.seconds, 1), "unit": UNIT, "cores": r.threads, "kind": "oracle",
            "seconds": round(r.seconds, 2), "triangles": r.T,
            "sample": f"triangles whose smallest hyperedge id is in [{lo},{hi}) of the same "
                      f"hypergraph (Exact-bs enumeration, std::set classification)"}


# ------------------------------------------------------------------ reference arm (the oracle)

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    if args.workload == "batched":
        import hgen

        # per step: the next whole member of the batch (seeds 100 ..), in seed order
        G = args.batch_members
        cfg = {"workload": f"batched_{G}", "members": G, "seeds": f"100..{99 + G}"}
        members = [hgen.batched(s) for s in range(100, 100 + G)]
        per_step_desc = "one whole member of the batch (seed order, cycling)"

        def step(k):
            sp = members[k % G]
            r = 0
            while True:
                try:
                    p, i = hgen.generate(sp if r == 0 else hgen.batched_redraw(sp, r))
                    break
                except hgen.DedupExhausted:
                    r += 1
            return oracle.count(p, i, sp.num_vertices)
    else:
        spec, e_ptr, e_idx, prefix = workload(args.workload)
        cfg = workload_config(spec, e_ptr, prefix)
        nv = spec.num_vertices
        per_step = 2000
        ne = len(e_ptr) - 1
        per_step_desc = f"triangles owned by {per_step} consecutive hyperedges"

        def step(k):
            lo = (k * per_step) % max(ne - per_step, 1)
            return oracle.count(e_ptr, e_idx, nv, i_range=(lo, min(lo + per_step, ne)))

    for k in range(args.warmup):
        step(k)
    tri, secs, threads = 0, 0.0, 1
    t0 = time.perf_counter()
    for k in range(args.steps):
        r = step(args.warmup + k)
        tri += r.T
        secs += r.seconds
        threads = r.threads
    wall = time.perf_counter() - t0
    value = tri / secs
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1000 * wall / args.steps, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic", "impl": "reference", "config": cfg,
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"per step: {per_step_desc}"},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "served":
        run_served(args)
    elif args.workload == "sample":
        run_sample(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
