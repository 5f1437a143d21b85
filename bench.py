#!/usr/bin/env python
"""Benchmark of the Phase (A) level loop (arXiv 1812.08942, Sec. 3.2):
smoothing -> affinity -> aggregation -> Galerkin coarsening, level by level,
on a synthetic graph shaped like the paper's workloads.

One step = graph_reduce_create (CSR of the input edge list already resident
in HBM) + graph_reduce_multilevel (all levels down to the final target).
Metric: input edges per second summed over levels, i.e. sum_l m_l / t_step,
aggregated over all ranks (replicas; the path does not shard here).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload chunglu_434k|mesh3d_128|knn_200k|grid2d_64|knn_1m]

Under torchrun (N > 1) every rank runs an independent replica.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "input edges/s per aggregation level (sum over levels of m_l / step time)"
UNIT = "edges/s"
DEFAULT_WORKLOAD = "mesh3d_128"
# dense FP64 arithmetic of one GB300, nominal (TFLOP/s, a multiply-add = 2)
FP64_NOMINAL_TFLOPS = 1.25
# bounded oracle sample (reference arm): the same recipe at 1/8 scale
SAMPLE_DIV = 8


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 pipeline comparison")
    ap.add_argument("--no-eigen", action="store_true", help="skip the multilevel eigensolver measurement")
    return ap.parse_args()


def max_over_ranks(x, world, device=None):
    """Max of a host float over all ranks (the slowest rank sets the time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(edges_per_step, steps, world, t_max_ms):
    """Input edges/s of the whole job: every rank reduces its own replica."""
    return edges_per_step * steps * world / (t_max_ms / 1000.0)


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")), int(
        os.environ.get("WORLD_SIZE", "1"))


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# Algorithmic bytes of one Jacobi sweep (the dominant kernel): every CSR slot
# read once (column index + row-scaled weight), the row pointers, the vector
# block read once and written once.
# ---------------------------------------------------------------------------
def sweep_bytes(n, m, K, xbytes, wbytes):
    return 2 * m * (4 + wbytes) + 8 * (n + 1) + 2 * n * K * xbytes


def affinity_bytes(n, m, K, xbytes, dbytes):
    """Per-edge distance: the upper-triangle columns, the block read once, d written."""
    return m * 4 + n * K * xbytes + m * dbytes


def aggregate_bytes(n, m, dbytes, passes=2):
    """Suitor matching, every pass scanning every CSR slot once (column +
    key) and updating per-node state (8 bytes)."""
    return passes * (2 * m * (4 + dbytes) + 8 * n)


def galerkin_bytes(n, m, mc):
    """Galerkin product: the fine edge list (u, v, w) and the map read, the
    coarse edge list (u, v, w + its CSR slot pair) written."""
    return m * (4 + 4 + 8) + n * 4 + mc * 16


def loss_bytes(n, m, nc, mc, K, S):
    """Spectral-mismatch loss (forward) and its adjoint (the extra of the
    backward pass), algorithmic bytes: fine Rayleigh quotients (edge list and
    block), aggregate means, S coarse sweeps over the parameter weights (CSR
    slots: column, edge id, weight; row pointers, degrees; block read and
    written), the coarse quotients; backward: the sweeps recomputed with their
    iterates saved, S adjoint sweeps, and the per-edge gradient reading each
    saved iterate once."""
    sweep = 2 * mc * 12 + 8 * (nc + 1) + 4 * nc + 2 * nc * K * 4
    fwd = (m * 16 + 2 * n * K * 4) + (n * K * 4 + n * 4 + nc * K * 4) + S * sweep + (mc * 12 + nc * K * 4)
    bwd = S * (sweep + 2 * nc * K * 4) + S * sweep + (mc * 12 + 3 * S * nc * K * 4)
    return fwd, bwd


SWEEP_KERNEL_NAMES = {1: "k_sweep_row", 2: "k_sweep_stream", 3: "k_sweep_band"}
SWEEP_KERNEL_SOURCES = {"k_sweep_row": "gr_smooth.cu", "k_sweep_stream": "gr_smooth.cu", "k_sweep_band": "gr_band.cu"}


def kernel_source_sha(path):
    import hashlib
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def traffic_from_profile(workload, src_sha):
    """dram bytes per sweep launch from the committed ncu summary, if it was
    taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "k_sweep_%s.md" % workload)
    if not os.path.exists(p):
        return None
    txt = open(p).read()
    m_sha = re.search(r"source_sha256_16:\s*([0-9a-f]+)", txt)
    m_tr = re.search(r"traffic_bytes_per_launch_level0:\s*([0-9.eE+]+)", txt)
    if not m_sha or not m_tr or m_sha.group(1) != src_sha:
        return None
    return float(m_tr.group(1))


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, window=None):
        """Clock summary of the samples that arrived inside `window` (host
        perf_counter times around the timed region; all samples if none did)."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        inside = [x for x in lines if window[0] <= x[0] <= window[1]] if window is not None else []
        if inside:
            lines = inside
        for _, ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "samples_in_timed_region": len(inside)}


# ---------------------------------------------------------------------------
# Oracle timing (CPU baseline / reference arm)
# ---------------------------------------------------------------------------
def cpu_info():
    """Host CPU model and logical CPU count (the oracle runs on one of them)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for ln in f:
                    if ln.lower().startswith(("model name", "cpu part")):
                        model = ln.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"cpu_model": model or platform.processor() or platform.machine(), "cpu_count": os.cpu_count(),
            "machine": platform.machine()}


def oracle_sample_graph(workload):
    import workloads as W
    if workload == "knn_200k":
        g = W.knn_gmm(200_000 // SAMPLE_DIV, 10, 10, 10, 12347)
        desc = "kNN recipe at 1/%d of the points (%d points in 10-D, 10-component GMM, k=10, Gaussian weights)" % (
            SAMPLE_DIV, g.n)
    elif workload == "knn_1m":
        g = W.knn_gmm(1_000_000 // SAMPLE_DIV, 16, 20, 15, 12350)
        desc = "kNN recipe at 1/%d of the points (%d points in 16-D, 20-component GMM, k=15, Gaussian weights)" % (
            SAMPLE_DIV, g.n)
    elif workload == "chunglu_434k":
        g = W.chung_lu(434_000 // SAMPLE_DIV, 16_000_000 // SAMPLE_DIV)
        desc = "Chung-Lu recipe at 1/%d scale (%d nodes, %d edges, same mean degree and exponent)" % (
            SAMPLE_DIV, g.n, g.m)
    elif workload == "mesh3d_128":
        g = W.mesh3d(64, 64, 64)
        desc = "64^3 7-point mesh, log-normal weights (the same recipe at 1/8 of the nodes)"
    elif workload == "grid2d_64":
        g = W.grid2d(64, 64)
        desc = "the full 64x64 grid"
    else:
        raise ValueError("no oracle sample for workload %r" % workload)
    return g, desc


def time_oracle_multilevel(g, wl):
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    levels = oracle.reduce_multilevel(g.n, g.u, g.v, g.w, wl.K, wl.sweeps, wl.omega,
                                      final_target=max(1, int(wl.final_target * g.n / wl_full_n(wl))))
    dt = time.perf_counter() - t0
    edges = sum(lv.m for lv in levels)
    return edges, dt, len(levels)


def wl_full_n(wl):
    return {"chunglu_434k": 434_000, "mesh3d_128": 2_097_152, "knn_200k": 200_000, "grid2d_64": 4096,
            "knn_1m": 1_000_000}.get(wl.name, 434_000)


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    import workloads as W
    wl = W.WORKLOADS[args.workload]
    g, desc = oracle_sample_graph(args.workload)
    times = []
    edges = 0
    for i in range(args.warmup + args.steps):
        e, dt, nl = time_oracle_multilevel(g, wl)
        if i >= args.warmup:
            times.append(dt)
            edges = e
    total = sum(times)
    value = edges * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample": desc, "K": wl.K, "sweeps": wl.sweeps, "omega": wl.omega},
        "cpu_baseline": dict({"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                              "sample": "FP64 C oracle, single thread, full level loop on " + desc,
                              "same_config": False}, **cpu_info()),
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    rank, local_rank, world = dist_env()
    import torch
    import torch.distributed as dist

    if world > 1:
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    import __graft_entry__
    __graft_entry__.build()
    import numpy as np

    import paper_1812_08942_gb300 as gr
    import workloads as W

    wl = W.WORKLOADS[args.workload]
    g = wl.make(device=dev)
    prec = {"f64": gr.GR_F64, "f32": gr.GR_F32, "bf16": gr.GR_BF16}[wl.precision]
    xbytes = {"f64": 8, "f32": 4, "bf16": 2}[wl.precision]
    xdtype = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[wl.precision]
    wbytes = 8 if wl.precision == "f64" else 4
    params = gr.ReduceParams(K=wl.K, sweeps=wl.sweeps, omega=wl.omega, seed=0, prec=prec, passes=2,
                             level_ratio=4, final_target=wl.final_target, max_levels=32)
    # inputs resident in HBM before the timed region
    u_d = torch.from_numpy(g.u).to(dev)
    v_d = torch.from_numpy(g.v).to(dev)
    w_d = torch.from_numpy(g.w).to(dev)
    torch.cuda.synchronize()

    def step():
        G = gr.graph_reduce_create(g.n, u_d, v_d, w_d)
        levels, stats = gr.graph_reduce_multilevel(G, params, want_stats=True)
        return G, levels, stats

    for _ in range(args.warmup):
        G, levels, stats = step()
        del G, levels
    torch.cuda.synchronize()

    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local_rank)).split(",")[0]) if world == 1 else local_rank
    sampler = ClockSampler(gpu_index if world == 1 else local_rank)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = gr.graph_reduce_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t_begin = time.perf_counter()
    ev0.record()
    all_stats = []
    last = None
    for _ in range(args.steps):
        G, levels, stats = step()
        all_stats.append(stats)
        last = (G, levels)
        del G, levels
    ev1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = gr.graph_reduce_launch_count() - launches0
    t_end = time.perf_counter()
    clocks = sampler.stop((t_begin, t_end))
    t_ms = ev0.elapsed_time(ev1)
    t_max = max_over_ranks(t_ms, world, dev)
    edges_per_step = sum(s["m"] for s in all_stats[-1])
    value = whole_job_value(edges_per_step, args.steps, world, t_max)

    # the sweep kernel each level ran (the automatic choice, kept per context)
    sweep_kernels = []
    for ctx in [last[0]] + list(last[1][:-1]):
        sweep_kernels.append(SWEEP_KERNEL_NAMES[gr.graph_reduce_sweep_plan(ctx, wl.K, xdtype)])
    del last

    # roofline of the dominant kernel: the level-0 Jacobi sweep (algorithmic
    # bytes of one sweep x launches / event time of the level's sweeps); the
    # same over every level (coarser levels may run another sweep kernel)
    peak, peak_kind = load_peaks()
    lv0 = all_stats[-1][0]
    b0 = sweep_bytes(lv0["n"], lv0["m"], wl.K, xbytes, wbytes)
    l0_ms = sum(stats[0]["t_sweeps"] for stats in all_stats)
    l0_launches = sum(stats[0]["sweeps"] for stats in all_stats)
    achieved = b0 * l0_launches / (l0_ms / 1000.0) / 1e9 if l0_ms > 0 else 0.0
    sw_bytes = 0.0
    sw_ms = 0.0
    sw_launches = 0
    for stats in all_stats:
        for s in stats:
            sw_bytes += s["sweeps"] * sweep_bytes(s["n"], s["m"], wl.K, xbytes, wbytes)
            sw_ms += s["t_sweeps"]
            sw_launches += s["sweeps"]
    all_achieved = sw_bytes / (sw_ms / 1000.0) / 1e9 if sw_ms > 0 else 0.0
    src_sha = kernel_source_sha(os.path.join(ROOT, "paper_1812_08942_gb300", "csrc",
                                             SWEEP_KERNEL_SOURCES[sweep_kernels[0]]))
    traffic = traffic_from_profile(args.workload, src_sha)
    roofline = {
        "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
        "peak_kind": peak_kind,
        "kernel": "%s (weighted-Jacobi multi-vector SpMM, level 0)" % sweep_kernels[0],
        "bytes_per_launch": b0, "traffic": traffic, "launches": l0_launches,
        "avg_launch_ms": l0_ms / max(l0_launches, 1),
        "all_levels": {"kernels": sweep_kernels, "achieved": all_achieved, "frac": all_achieved / peak,
                       "launches": sw_launches, "avg_launch_ms": sw_ms / max(sw_launches, 1)},
    }
    per_level = []
    for s in all_stats[-1]:
        t = s["t_smooth"] + s["t_affinity"] + s["t_aggregate"] + s["t_coarsen"]
        per_level.append({"n": s["n"], "m": s["m"], "nc": s["nc"], "mc": s["mc"], "proposals": s["proposals"],
                          "t_smooth_ms": round(s["t_smooth"], 4), "t_affinity_ms": round(s["t_affinity"], 4),
                          "t_aggregate_ms": round(s["t_aggregate"], 4), "t_coarsen_ms": round(s["t_coarsen"], 4),
                          "edges_per_s": s["m"] / (t / 1000.0) if t > 0 else None})

    # the other phases against the same HBM peak: algorithmic bytes (the
    # helpers above) over each phase's event time (all its kernels and host
    # synchronisations), summed over levels and steps
    dbytes = 8 if wl.precision == "f64" else 4
    acc = {"affinity": [0.0, 0.0], "aggregate": [0.0, 0.0], "coarsen": [0.0, 0.0]}
    for stats in all_stats:
        for s in stats:
            acc["affinity"][0] += affinity_bytes(s["n"], s["m"], wl.K, xbytes, dbytes)
            acc["affinity"][1] += s["t_affinity"]
            acc["aggregate"][0] += aggregate_bytes(s["n"], s["m"], dbytes)
            acc["aggregate"][1] += s["t_aggregate"]
            acc["coarsen"][0] += galerkin_bytes(s["n"], s["m"], s["mc"])
            acc["coarsen"][1] += s["t_coarsen"]
    phases = {}
    for k, (b, t) in acc.items():
        gbs = b / (t / 1000.0) / 1e9 if t > 0 else 0.0
        phases[k] = {"bytes_per_step": b / args.steps, "ms_per_step": t / args.steps, "achieved_gbs": gbs,
                     "frac": gbs / peak, "unit": "GB/s", "bound": "hbm"}
    roofline["phases"] = phases

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        uh = torch.from_numpy(g.u).pin_memory()
        vh = torch.from_numpy(g.v).pin_memory()
        wh = torch.from_numpy(g.w).pin_memory()
        h2d = g.m * (4 + 4 + 8)
        d2h = 0
        k_e2e = max(1, args.steps)
        # each step's edge list goes up from pinned host memory on a side
        # stream while the previous step is reduced (double-buffered), and
        # its results go down on another side stream while the next step is
        # reduced, the way a pipeline feeding graphs to the library would
        # run; the timed region ends when the last results are on the host
        cs = torch.cuda.Stream(device=dev)
        ds = torch.cuda.Stream(device=dev)
        main = torch.cuda.current_stream(dev)
        bufs = [tuple(torch.empty(x.shape, dtype=x.dtype, device=dev) for x in (uh, vh, wh)) for _ in range(2)]
        evs = [torch.cuda.Event() for _ in range(2)]

        def upload(i):
            with torch.cuda.stream(cs):
                for dst, src in zip(bufs[i % 2], (uh, vh, wh)):
                    dst.copy_(src, non_blocking=True)
                evs[i % 2].record(cs)

        # results: the final reduced edge list (at most the input's size) and
        # the composed map, staged on the device (two sets) and copied into
        # pinned host buffers kept across steps
        out_d = [(torch.empty(g.m, dtype=torch.int32, device=dev), torch.empty(g.m, dtype=torch.int32, device=dev),
                  torch.empty(g.m, dtype=torch.float64, device=dev), torch.empty(g.n, dtype=torch.int32, device=dev))
                 for _ in range(2)]
        out_h = (torch.empty(g.m, dtype=torch.int32).pin_memory(), torch.empty(g.m, dtype=torch.int32).pin_memory(),
                 torch.empty(g.m, dtype=torch.float64).pin_memory(), torch.empty(g.n, dtype=torch.int32).pin_memory())
        ev_res = [torch.cuda.Event() for _ in range(2)]
        ev_down = [torch.cuda.Event() for _ in range(2)]
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        upload(0)
        for st in range(k_e2e):
            evs[st % 2].synchronize()
            if st + 1 < k_e2e:
                upload(st + 1)
            G = gr.graph_reduce_create(g.n, *bufs[st % 2])
            levels, _ = gr.graph_reduce_multilevel(G, params, want_stats=False)
            du, dv, dw, dc = out_d[st % 2]
            if st >= 2:  # the copies out of this staging set two steps ago are done
                main.wait_event(ev_down[st % 2])
            mc = levels[-1].m
            gr.graph_reduce_get_edges(levels[-1], on_host=False, out=(du, dv, dw))
            dc.copy_(gr.graph_reduce_compose_maps(levels))
            ev_res[st % 2].record(main)
            with torch.cuda.stream(ds):
                ds.wait_event(ev_res[st % 2])
                for h, d in zip(out_h[:3], (du, dv, dw)):
                    h[:mc].copy_(d[:mc], non_blocking=True)
                out_h[3].copy_(dc, non_blocking=True)
                ev_down[st % 2].record(ds)
            d2h = mc * 16 + g.n * 4
            del G, levels
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": edges_per_step * k_e2e * world / te, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": k_e2e,
               "inputs": "pinned host edge list, uploaded on a side stream during the previous step",
               "outputs": "final reduced edge list and composed map, read back on a side stream during the next step"}

    # The oracle's level loop on the full configuration, once, outside the
    # timed regions: the CPU baseline (one host core) and the reference the
    # GPU paths' reduced graphs are checked against
    orc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as _orc
        _orc.build()
        t0 = time.perf_counter()
        orc_levels = _orc.reduce_multilevel(g.n, g.u, g.v, g.w, wl.K, wl.sweeps, wl.omega,
                                            final_target=wl.final_target)
        orc = (orc_levels, time.perf_counter() - t0)

    # FP32 (or BF16) path against the plain FP64 GPU path on the same graph:
    # step-time speedup; the 10 smallest nontrivial eigenvalues of each final
    # reduced graph (FP64 solver on the host) against the oracle's reduced
    # graph of the same configuration (the GPU FP64 graph when the oracle is
    # skipped)
    cmp64 = None
    if rank == 0 and world == 1 and not args.no_fp64 and prec != gr.GR_F64:
        p64 = gr.ReduceParams(K=wl.K, sweeps=wl.sweeps, omega=wl.omega, seed=0, prec=gr.GR_F64, passes=2,
                              level_ratio=4, final_target=wl.final_target, max_levels=32)

        def step64():
            G = gr.graph_reduce_create(g.n, u_d, v_d, w_d)
            levels, _ = gr.graph_reduce_multilevel(G, p64, want_stats=False)
            return G, levels

        G64, lv64 = step64()  # warm-up (FP64 slot packing, scratch)
        del G64, lv64
        k64 = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k64):
            G64, lv64 = step64()
            if _ < k64 - 1:
                del G64, lv64
        e1.record()
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / k64
        import oracle as _or  # host FP64 eigen solver only
        G32 = gr.graph_reduce_create(g.n, u_d, v_d, w_d)
        lv32, _ = gr.graph_reduce_multilevel(G32, params, want_stats=False)
        ev = []
        for lv in (lv32, lv64):
            fu, fv, fw = (t.numpy() for t in gr.graph_reduce_get_edges(lv[-1], on_host=True))
            ev.append(_or.smallest_nontrivial_eigs(lv[-1].n, fu, fv, fw, 10))
        if orc is not None:
            last = orc[0][-1]
            ev_ref = _or.smallest_nontrivial_eigs(last.nc, last.uc, last.vc, last.wc, 10)
            ref_kind = "oracle reduced graph (FP64 CPU level loop, same configuration)"
        else:
            ev_ref = ev[1]
            ref_kind = "GPU FP64 reduced graph (oracle skipped)"
        rel = float(np.max(np.abs(ev[0] - ev_ref) / np.abs(ev_ref)))
        rel64 = float(np.max(np.abs(ev[1] - ev_ref) / np.abs(ev_ref)))
        same_maps = all(torch.equal(gr.graph_reduce_get_map(a), gr.graph_reduce_get_map(b))
                        for a, b in zip(lv32, lv64)) and len(lv32) == len(lv64)
        cmp64 = {"ms_per_step_fp64": t64, "ms_per_step": t_max / args.steps,
                 "speedup": t64 / (t_max / args.steps), "lambda_reference": ref_kind,
                 "lambda10_max_rel_err": rel, "at_accuracy": bool(rel <= 1e-3),
                 "fp64_lambda10_max_rel_err": rel64,
                 "fp32_vs_gpu_fp64_lambda10_max_rel_err": float(np.max(np.abs(ev[0] - ev[1]) / np.abs(ev[1]))),
                 "aggregates_identical_fp32_fp64": bool(same_maps),
                 "lambda10_reference": [float(x) for x in ev_ref]}
        if orc is not None:
            cmp64["fp64_maps_identical_to_oracle"] = bool(
                len(orc[0]) == len(lv64)
                and all(np.array_equal(gr.graph_reduce_get_map(b).cpu().numpy(), a.agg) for a, b in zip(orc[0], lv64)))
        # BF16 storage of the test vectors (FP32 accumulation), same comparison
        if prec != gr.GR_BF16:
            pb = gr.ReduceParams(K=wl.K, sweeps=wl.sweeps, omega=wl.omega, seed=0, prec=gr.GR_BF16, passes=2,
                                 level_ratio=4, final_target=wl.final_target, max_levels=32)
            Gb = gr.graph_reduce_create(g.n, u_d, v_d, w_d)
            lvb, _st = gr.graph_reduce_multilevel(Gb, pb, want_stats=False)
            del lvb, Gb
            torch.cuda.synchronize()
            e0.record()
            for ib in range(k64):
                Gb = gr.graph_reduce_create(g.n, u_d, v_d, w_d)
                lvb, _st = gr.graph_reduce_multilevel(Gb, pb, want_stats=False)
                if ib < k64 - 1:
                    del Gb, lvb
            e1.record()
            torch.cuda.synchronize()
            tb = e0.elapsed_time(e1) / k64
            fu, fv, fw = (t.numpy() for t in gr.graph_reduce_get_edges(lvb[-1], on_host=True))
            evb = _or.smallest_nontrivial_eigs(lvb[-1].n, fu, fv, fw, 10)
            relb = float(np.max(np.abs(evb - ev_ref) / np.abs(ev_ref)))
            m0 = gr.graph_reduce_get_map(lvb[0]).cpu().numpy()
            m64 = gr.graph_reduce_get_map(lv64[0]).cpu().numpy()
            cmp64["bf16_storage"] = {"ms_per_step": tb, "speedup_vs_fp64": t64 / tb, "lambda10_max_rel_err": relb,
                                     "at_accuracy": bool(relb <= 1e-3), "levels": len(lvb),
                                     "level0_map_agreement": float(np.mean(m0 == m64)) if len(m0) == len(m64) else None}
            del Gb, lvb
        del G32, lv32, G64, lv64

    # Multilevel Laplacian eigensolver (Alg. 5) on a deeper reduction of the
    # same graph (down to 1,024 nodes, where the coarsest eigenpairs are found):
    # k = 8 ratio-cut eigenvectors, 10 shifted Jacobi iterations
    # per level.  The smoothing time is the difference against 0 iterations;
    # its memory roofline counts, per iteration on each level, the CSR slots
    # (column + FP64 weight), row pointers and the per-entry gains, and the
    # block read and written once (2 n k 8 bytes); its FP64 roofline counts a
    # multiply-add per slot and column and a multiply plus a multiply-add per
    # entry (the per-level gains, once per level, are left out) against the
    # nominal FP64 rate: the iteration runs in FP64 throughout and this part's
    # FP64 units, not its memory, bound it.
    eig = None
    if rank == 0 and world == 1 and not args.no_eigen:
        keig, iters = 8, 10
        pe = gr.ReduceParams(K=wl.K, sweeps=wl.sweeps, omega=wl.omega, seed=0, prec=prec, passes=2,
                             level_ratio=4, final_target=1024, max_levels=32)
        Ge = gr.graph_reduce_create(g.n, u_d, v_d, w_d)
        lve, _ = gr.graph_reduce_multilevel(Ge, pe, want_stats=False)
        hier = [Ge] + list(lve)

        def teig(it, reps=3):
            gr.graph_reduce_eigensolve(hier, keig, False, 0.7, it, want_rayleigh=False)
            ts = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                gr.graph_reduce_eigensolve(hier, keig, False, 0.7, it, want_rayleigh=False)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return min(ts)

        t_full = teig(iters)
        t_none = teig(0)
        U, lam, rq = gr.graph_reduce_eigensolve(hier, keig, False, 0.7, iters)
        sm_bytes = sum(iters * (2 * L.m * (4 + 8) + 8 * (L.n + 1) + 3 * L.n * keig * 8)
                       for L in hier[:-1])
        sm_flops = sum(iters * (2 * keig * 2 * L.m + 3 * L.n * keig) for L in hier[:-1])
        t_sm = max(t_full - t_none, 1e-6)
        ach = sm_bytes / (t_sm / 1000.0) / 1e9
        ach_f = sm_flops / (t_sm / 1000.0) / 1e12
        eig = {"k": keig, "normalized": False, "iters_per_level": iters, "levels": len(hier),
               "coarsest_n": hier[-1].n, "ms": t_full, "ms_without_smoothing": t_none,
               "smoothing_roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                      "frac": ach / peak, "bytes": sm_bytes},
               "smoothing_fp64": {"bound": "alu", "achieved": ach_f, "peak": FP64_NOMINAL_TFLOPS,
                                  "unit": "TFLOP/s", "frac": ach_f / FP64_NOMINAL_TFLOPS,
                                  "peak_kind": "nominal FP64 rate", "flops": sm_flops},
               "lambda_coarsest": [float(x) for x in lam], "rayleigh": [float(x) for x in rq]}
        # the same with the Galerkin-consistent mass B_l = P^T B_(l-1) P: the
        # coarsest eigenvalues are then Rayleigh-Ritz values of the finest
        # problem (upper bounds of its eigenvalues), and the returned Rayleigh
        # quotients show how close the refined vectors come to its low spectrum
        gr.graph_reduce_eigensolve(hier, keig, False, 0.7, iters, want_rayleigh=False, galerkin_mass=True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        Ug, lamg, rqg = gr.graph_reduce_eigensolve(hier, keig, False, 0.7, iters, galerkin_mass=True)
        e1.record()
        torch.cuda.synchronize()
        eig["galerkin_mass"] = {"ms": e0.elapsed_time(e1), "lambda_coarsest": [float(x) for x in lamg],
                                "rayleigh": [float(x) for x in rqg]}
        del U, Ug, hier, lve, Ge

    # Spectral-mismatch loss and its adjoint (the differentiable edge-weight
    # objective): fine graph against the final reduced graph through the
    # composed map, the FP32 smoothed block of the step's first level,
    # 5 coarse sweeps; forward and forward + backward times.
    lossm = None
    if rank == 0 and world == 1 and not args.no_eigen and prec != gr.GR_F64:
        Gl = gr.graph_reduce_create(g.n, u_d, v_d, w_d)
        lvl, _ = gr.graph_reduce_multilevel(Gl, params, want_stats=False)
        comp = gr.graph_reduce_compose_maps(lvl)
        Cl = lvl[-1]
        Xl = torch.empty(g.n, wl.K, dtype=torch.float32, device=dev)
        gr.graph_reduce_smooth(Gl, Xl, wl.sweeps, wl.omega, 0, 0)
        _, _, wcl = gr.graph_reduce_get_edges(Cl)
        wc32 = wcl.float().contiguous()

        def tloss(backward, reps=5):
            ts = []
            for _ in range(reps + 1):
                w = wc32.clone().requires_grad_(backward)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                L = gr.spectral_mismatch_loss(w, Gl, Cl, comp, Xl, 5, wl.omega)
                if backward:
                    L.backward()
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return min(ts[1:]), float(L.item())

        t_f, lval = tloss(False)
        t_fb, _ = tloss(True)
        bf, bb = loss_bytes(g.n, g.m, Cl.n, Cl.m, wl.K, 5)
        lossm = {"fine_n": g.n, "coarse_n": Cl.n, "coarse_m": Cl.m, "K": wl.K, "coarse_sweeps": 5, "loss": lval,
                 "ms_forward": t_f, "ms_forward_backward": t_fb,
                 "bytes_forward": bf, "bytes_backward": bb,
                 "achieved_gbs_forward": bf / (t_f / 1000.0) / 1e9,
                 "achieved_gbs_forward_backward": (bf + bb) / (t_fb / 1000.0) / 1e9,
                 "frac_forward": bf / (t_f / 1000.0) / 1e9 / peak,
                 "frac_forward_backward": (bf + bb) / (t_fb / 1000.0) / 1e9 / peak}

        # Edge-weight scaling of the reduced graph (Alg. 1 driven by the loss
        # gradient): 10 iterations with eps = 0, eta_max sized so that the
        # first step moves an edge by at most 5 % of the mean weight.  Each
        # iteration is one loss forward + adjoint, the per-edge update, the
        # degree and lambda_1 recomputation and two small host reads.
        wg = wc32.clone().requires_grad_(True)
        gr.spectral_mismatch_loss(wg, Gl, Cl, comp, Xl, 5, wl.omega).backward()
        eta_s = 0.05 * float(wc32.mean()) / max(float(wg.grad.abs().max()), 1e-30)
        ks = 10
        gr.graph_reduce_scale_edges(Gl, Cl, comp, Xl, wc32.clone(), 5, wl.omega, eta_max=eta_s, kmax=2, eps=0.0)
        ws = wc32.clone()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ws, hist = gr.graph_reduce_scale_edges(Gl, Cl, comp, Xl, ws, 5, wl.omega, eta_max=eta_s, kmax=ks, eps=0.0)
        torch.cuda.synchronize()
        t_sc = (time.perf_counter() - t0) * 1000.0
        moved = float(((ws - wc32) > 0).float().mean())
        lossm["edge_scaling"] = {"iterations": len(hist), "eta_max": eta_s, "alpha": 0.5, "delta_bar": 0.5,
                                 "ms": t_sc, "ms_per_iteration": t_sc / max(len(hist), 1),
                                 "loss_first": hist[0][0] if hist else None,
                                 "loss_last": hist[-1][0] if hist else None,
                                 "lambda1_last": hist[-1][1] if hist else None, "edges_scaled_frac": moved}
        del Xl, Cl, lvl, Gl, comp, wc32, wg, ws

    # Multicolour Gauss-Seidel smoothing (Sec. 3.2.1) on the fine graph:
    # colouring time (first call), and per sweep (S = 8 minus S = 0) with its
    # roofline.  Bytes per sweep: the CSR slots, row pointers and the block
    # read and written once by the colour-class kernels (as the Jacobi sweep),
    # plus the statistics read and the in-place scaling of the block.
    gsm = None
    if rank == 0 and world == 1 and not args.no_eigen:
        Gg = gr.graph_reduce_create(g.n, u_d, v_d, w_d)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, ncol = gr.graph_reduce_colour(Gg, 0)
        t_col = (time.perf_counter() - t0) * 1000.0
        Xg = torch.empty(g.n, wl.K, dtype={"f64": torch.float64, "f32": torch.float32,
                                           "bf16": torch.bfloat16}[wl.precision], device=dev)

        def tgs(S, reps=3):
            gr.graph_reduce_smooth_gs(Gg, Xg, S, wl.omega, 0, 0, 0)
            ts = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                gr.graph_reduce_smooth_gs(Gg, Xg, S, wl.omega, 0, 0, 0)
                e1.record()
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            return min(ts)

        per = (tgs(8) - tgs(0)) / 8
        gbytes = sweep_bytes(g.n, g.m, wl.K, xbytes, wbytes) + 3 * g.n * wl.K * xbytes
        gach = gbytes / (per / 1000.0) / 1e9 if per > 0 else 0.0
        gsm = {"colours": ncol, "colouring_ms": t_col, "ms_per_sweep": per,
               "jacobi_ms_per_sweep_level0": all_stats[-1][0]["t_sweeps"] / max(wl.sweeps, 1),
               "roofline": {"bound": "hbm", "achieved": gach, "peak": peak, "unit": "GB/s", "frac": gach / peak,
                            "bytes_per_sweep": gbytes}}
        del Xg, Gg

    # Reduced data set F_R = P^T F (Alg. 6, step 4) over the bench step's
    # levels: 16 FP32 features per fine node.  Algorithmic bytes: F read
    # once, F_R written once, the per-level maps read once.
    rdata = None
    if rank == 0 and world == 1 and not args.no_eigen:
        Gd = gr.graph_reduce_create(g.n, u_d, v_d, w_d)
        lvd, _ = gr.graph_reduce_multilevel(Gd, params, want_stats=False)
        Fd = torch.randn(g.n, 16, dtype=torch.float32, device=dev)
        gr.graph_reduce_reduce_data(lvd, Fd)
        tds = []
        for _ in range(5):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            Rd = gr.graph_reduce_reduce_data(lvd, Fd)
            e1.record()
            torch.cuda.synchronize()
            tds.append(e0.elapsed_time(e1))
        tdm = min(tds)
        dbytes = g.n * 16 * 4 + lvd[-1].n * 16 * 4 + 4 * (g.n + sum(L.n for L in lvd[:-1]))
        rdata = {"d": 16, "dtype": "f32", "rows_in": g.n, "rows_out": lvd[-1].n, "ms": tdm,
                 "algorithmic_bytes": dbytes, "achieved_gbs": dbytes / (tdm / 1000.0) / 1e9}
        del Rd, Fd, lvd, Gd

    cpu = None
    if orc is not None:
        e = sum(lv.m for lv in orc[0])
        cpu = dict({"value": e / orc[1], "unit": UNIT, "cores": 1, "kind": "oracle", "same_config": True,
                    "sample": "FP64 C oracle, one host core, one full step of this configuration (%d levels, "
                              "%.1f s)" % (len(orc[0]), orc[1])}, **cpu_info())

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": wl.precision, "data": "synthetic",
            "config": {"workload": wl.name, "n": g.n, "m": g.m, "K": wl.K, "sweeps": wl.sweeps,
                       "omega": wl.omega, "passes": 2, "level_ratio": 4, "final_target": wl.final_target,
                       "levels": len(all_stats[-1]), "edges_per_step": edges_per_step,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (edge list %.0f MB + CSR %.0f MB vs 129 MB); no flush"
                             % (g.m * 16 / 1e6, g.m * 2 * 24 / 1e6)},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
            "fp32_vs_fp64": cmp64, "multilevel_eigensolver": eig, "reduced_dataset": rdata,
            "gauss_seidel": gsm, "spectral_mismatch_loss": lossm,
            "clocks": clocks, "levels": per_level,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
