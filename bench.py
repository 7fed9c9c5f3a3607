#!/usr/bin/env python
"""Benchmark: fwd+bwd views/s of the differentiable tile rasterizer on one GB300.

A step is one training view through the whole hot path: gs_project (EWA + SH3
colour) -> gs_bin_sort -> gs_raster_fwd (Eq. 2) -> gs_l1_loss_grad ->
gs_raster_bwd -> gs_project_bwd (parameter gradients, with the densification
statistic fused); by default the raster stages are the per-splat pair
gs_raster_fwd_ckpt / gs_raster_bwd_splat (--backward pixel: the per-pixel pair,
same gradients up to summation order). Workload: 1.5M Gaussians on 20 surface patches + background,
SH degree 3, one 1246x826 view per step on a radius-4 orbit, 16x16 tiles (the
synthetic stand-in for the paper's MipNeRF-360-scale scenes). Inputs are resident
in HBM; the parameters (354 MB resident; the projection reads the geometry of all
Gaussians and the SH rows of the visible ones) exceed the 129 MB L2.

Also reported: the same metric end to end (camera and target image copied from
pinned host memory, loss read back, every step), the roofline of the dominant
kernel, per-stage times, the batched mixed-resolution form (12 views in one
launch per stage, CUDA graph, knobs picked by the autotuner) beside its per-view
form, the large scene (5M Gaussians, 4 views at 1600x1060) with stored and
recomputed stop indices and with the per-splat backward, and their device memory, and the FP64 oracle timed on the
host cores on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 (torchrun), every rank renders its own view of its own replica (the
path has no exchange step inside a view); value = views of all ranks / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd+bwd views/s at 1.5M Gaussians 1246x826"
UNIT = "views/s"
WORKLOAD = "orbit-1.5M-sh3-1246x826"
# FLOPs per (pixel, list entry) pair, counted from the oracle's operation list:
# every examined entry costs the falloff (16); a composited entry adds 10 in the
# forward (transmittance update, weight, 3 colour FMAs) and 46 in the backward.
# The forward examines a pixel's entries up to its transmittance cut-off (or the
# list end); the backward only up to its last composited entry (the stop index).
FWD_FLOP_EXAM, FWD_FLOP_CONTRIB = 16, 10
BWD_FLOP_EXAM, BWD_FLOP_CONTRIB = 16, 46
# FP32 lanes per SM of compute capability 10.x (four sub-partitions of 32); the SM
# count and the maximum SM clock are read from the device at run time
FP32_LANES_PER_SM = 128


def fp32_peak_tflops(dev, clk, peaks):
    """FP32 issue peak = SMs x 128 lanes x 2 (FMA) x maximum SM clock, with the SM
    count from the device properties and the clock the maximum nvidia-smi reported
    during the timed region (else MEASURED_PEAKS.json's sm_max_mhz)."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    sms = int(props.multi_processor_count)
    mhz, src = clk.get("sm_max_mhz"), "nvidia-smi clocks.max.sm during the timed region"
    if not mhz:
        mhz, src = peaks.get("sm_max_mhz"), "MEASURED_PEAKS.json sm_max_mhz"
    mhz = float(mhz)
    peak = sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
    return peak, {"sms": sms, "fp32_lanes_per_sm": FP32_LANES_PER_SM, "flop_per_lane_cycle": 2,
                  "sm_max_mhz": mhz, "sms_source": "torch.cuda.get_device_properties().multi_processor_count",
                  "mhz_source": src}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-large", action="store_true", help="skip the 5M-Gaussian, 4-view section")
    ap.add_argument("--no-densify", action="store_true", help="skip the densification section")
    ap.add_argument("--cpu-sample-tiles", type=int, default=160)
    ap.add_argument("--n", type=int, default=1_500_000)
    ap.add_argument("--tile", default="16x16", help="tile shape WxH (16x16, 8x8, 16x32, 32x16)")
    ap.add_argument("--backward", choices=["pixel", "splat"], default="splat",
                    help="per-pixel gs_raster_bwd or per-splat gs_raster_bwd_splat")
    ap.add_argument("--quick", action="store_true",
                    help="timed region only (no e2e, batched or CPU legs): for profiler runs")
    return ap.parse_args()


def dist_info():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


# ----------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.index)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------
def make_scene(n, rank):
    from paper_2507_20239_gb300 import synth
    sc = synth.orbit_scene(1, n=n)
    if rank:
        # each rank renders its own orbit view of the same scene
        cam = sc.cameras[0]
        az = 2 * math.pi * rank / 8
        sc.cameras = [synth.orbit_camera(4.0, az + 0.7, 15.0, cam.width, cam.height, cam.fx)]
    return sc


STAGES = ["project", "bin_sort", "raster_fwd", "l1_loss_grad", "raster_bwd", "project_bwd"]


def measure_capacity(sc, frame, P):
    """Duplicates M and the per-pixel work of Eq. 2: entries examined by the forward,
    entries composited, and entries the backward walks (sum of the stop indices)."""
    from paper_2507_20239_gb300 import rasterizer as R
    proj = R.project(P, sc.sh_degree, frame)
    bins = R.bin_sort(proj, frame)
    M = int(bins.count.item())
    counts = R.raster_count(proj, bins, frame)
    c = counts.double().sum(0).cpu().numpy()
    _, _, stop = R.raster_fwd(proj, bins, frame, store_stop=True)
    measure_capacity.last_counts = counts
    # Gaussians visible in some view (only their SH rows are read by the projection
    # and its VJP)
    n = P["means"].shape[0]
    measure_capacity.n_visible = int((proj.radius.view(frame.n_views, n) > 0).any(0).sum().item())
    return M, float(c[0]), float(c[1]), float(stop.double().sum().item())


def splat_bucket_stats(step):
    """Work of the per-splat backward on view 0 from the forward's stop indices:
    64-entry buckets walked (per tile, up to its largest stop index) and live
    (pixel, bucket) pairs (per pixel, ceil(stop / 64)); a bucket takes its live
    pixels + 31 warp steps."""
    import torch
    if step.stop is None:
        return None
    f = step.frame
    tw, th = f.tile
    st = f.view_pixels(step.stop, 0).to(torch.int64)
    H, W = st.shape
    gy, gx = (H + th - 1) // th, (W + tw - 1) // tw
    pad = torch.zeros(gy * th, gx * tw, dtype=torch.int64, device=st.device)
    pad[:H, :W] = st
    tmax = pad.view(gy, th, gx, tw).amax(dim=(1, 3))
    return {"bucket_entries": 64, "buckets": int(((tmax + 63) // 64).sum()),
            "live_pixel_buckets": int(((st + 63) // 64).sum()), "pixels": int(H * W)}


def bench_ours(args, rank, local_rank, world):
    import torch
    import torch.distributed as dist
    from paper_2507_20239_gb300 import build as gbuild
    gbuild.build()
    from paper_2507_20239_gb300 import rasterizer as R, _abi, replicas
    from paper_2507_20239_gb300.step import StepConfig, TrainStep
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    sc = make_scene(args.n, rank)
    tile = tuple(int(x) for x in args.tile.split("x"))
    frame = R.Frame(sc.cameras, tile=tile, device=dev)
    P = R.to_device_params(sc.params(), dev)
    M, p_exam, p_contrib, p_walk_bwd = measure_capacity(sc, frame, P)
    step = TrainStep(P, sc.sh_degree, sc.cameras, sc.targets, StepConfig(tile=tile, backward=args.backward),
                     device=dev, capacity=int(M * 1.25) + 4096)
    for _ in range(max(args.warmup, 3)):
        step.run()
    torch.cuda.synchronize()
    assert step.error() == 0, "duplicate capacity exceeded"

    # ---- per-stage breakdown: the same step launched eagerly, CUDA events between stages
    events = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(args.steps)]
    launches0 = _abi.load().gs_launch_count()
    for k in range(args.steps):
        step.run(events[k])
    torch.cuda.synchronize()
    launches = (_abi.load().gs_launch_count() - launches0) // args.steps
    stage_ms = {s: statistics.mean(events[k][i].elapsed_time(events[k][i + 1]) for k in range(args.steps))
                for i, s in enumerate(STAGES)}
    eager_ms = statistics.mean(events[k][0].elapsed_time(events[k][6]) for k in range(args.steps))

    # ---- device-resident timed region: the step captured once into a CUDA graph
    graph = step.capture()
    for _ in range(3):
        graph.replay()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        graph.replay()
    t1.record()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = replicas.slowest(t0.elapsed_time(t1) / args.steps, dev)

    if args.quick:
        print(json.dumps({"quick": True, "ms_per_step": round(ms, 4), "eager_ms_per_step": round(eager_ms, 4),
                          "stages": stage_ms, "M": M, "pairs_walked_bwd": p_walk_bwd,
                          "pairs_examined": p_exam, "pairs_composited": p_contrib,
                          "tile_sync": tile_sync_stats(frame, measure_capacity.last_counts),
                          "splat_buckets": splat_bucket_stats(step)}), flush=True)
        return None
    # ---- end to end: camera + target H2D from pinned memory, loss D2H, every step
    # Two input buffers (camera block and target image), each with the step captured
    # over it: while one graph runs, the next step's camera and target are copied from
    # pinned host memory straight into the other buffer on a side stream (as a
    # training loop prefetches its next view), so the compute stream carries no
    # device-to-device move. Every one of the K host-to-device copies is issued after
    # e0 and waited for before e1; each step's loss is copied back to pinned memory.
    tgt_host = step.target.cpu().pin_memory()
    cam_host = step.frame.cams_dev.cpu().pin_memory()
    loss_host = torch.empty(frame.n_views, pin_memory=True)
    cams_a, tgt_a, ptr_a = step.frame.cams_dev, step.target, step.frame.frame.cams_dev
    cams_b, tgt_b = cams_a.clone(), tgt_a.clone()
    step.frame.frame.cams_dev, step.target = cams_b.data_ptr(), tgt_b
    graph_b = step.capture()
    step.frame.frame.cams_dev, step.target = ptr_a, tgt_a
    bufs = [(cams_a, tgt_a, graph), (cams_b, tgt_b, graph_b)]
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for cams_i, tgt_i, g_i in bufs:
        cams_i.copy_(cam_host, non_blocking=True)
        tgt_i.copy_(tgt_host, non_blocking=True)
        g_i.replay()
    torch.cuda.synchronize()
    cur = torch.cuda.current_stream()
    side = torch.cuda.Stream(device=dev)
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    done = [torch.cuda.Event(), torch.cuda.Event()]

    def prefetch(i):
        with torch.cuda.stream(side):
            bufs[i][0].copy_(cam_host, non_blocking=True)
            bufs[i][1].copy_(tgt_host, non_blocking=True)
            ready[i].record(side)

    e0.record()
    side.wait_stream(cur)
    prefetch(0)
    for k in range(args.steps):
        i = k % 2
        if k + 1 < args.steps:
            if k >= 1:
                side.wait_event(done[1 - i])   # the step that last read that buffer
            prefetch(1 - i)
        cur.wait_event(ready[i])
        bufs[i][2].replay()
        done[i].record(cur)
        loss_host.copy_(step.loss, non_blocking=True)
    e1.record()
    torch.cuda.synchronize()
    e2e_ms = replicas.slowest(e0.elapsed_time(e1) / args.steps, dev)

    # ---- roofline of the dominant kernel
    peaks = load_peaks()
    fp32_peak, peak_inputs = fp32_peak_tflops(dev, clk, peaks)                   # TFLOP/s
    dom = max(stage_ms, key=stage_ms.get)
    flops = {"raster_fwd": FWD_FLOP_EXAM * p_exam + FWD_FLOP_CONTRIB * p_contrib,
             "raster_bwd": BWD_FLOP_EXAM * p_walk_bwd + BWD_FLOP_CONTRIB * p_contrib}
    n_rec = sc.n * frame.n_views
    sh_k = sc.sh.shape[1]
    param_bytes = sc.n * 4 * (3 + 3 + 4 + 1 + 3 * sh_k)
    # parameters read: every Gaussian's geometry and opacity, SH rows of visible ones
    read_bytes = sc.n * 4 * (3 + 3 + 4 + 1) + measure_capacity.n_visible * 4 * 3 * sh_k
    bytes_ = {"project": read_bytes + n_rec * 57,
              "bin_sort": 8 * n_rec * 4 + 8 * M * 2 * 3,
              "l1_loss_grad": 3 * frame.n_pixels * 4 * 3,
              "project_bwd": read_bytes + param_bytes + n_rec * (40 + 57)}
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    stages = {}
    for s in STAGES:
        d = {"ms": round(stage_ms[s], 4)}
        if s in flops:
            a = flops[s] / (stage_ms[s] * 1e-3) / 1e12
            d.update(bound="alu", achieved_tflops=round(a, 3), frac=round(a / fp32_peak, 4))
        elif s in bytes_:
            a = bytes_[s] / (stage_ms[s] * 1e-3) / 1e9
            d.update(bound="hbm", achieved_gbs=round(a, 1), frac=round(a / hbm_peak, 4))
        stages[s] = d
    if dom in flops:
        ach = flops[dom] / (stage_ms[dom] * 1e-3) / 1e12
        conv = ({"flop_per_examined_pair": FWD_FLOP_EXAM, "flop_per_composited_pair": FWD_FLOP_CONTRIB,
                 "pairs_examined": p_exam, "pairs_composited": p_contrib} if dom == "raster_fwd" else
                {"flop_per_walked_pair": BWD_FLOP_EXAM, "flop_per_composited_pair": BWD_FLOP_CONTRIB,
                 "pairs_walked": p_walk_bwd, "pairs_composited": p_contrib})
        roof = {"kernel": dom, "bound": "alu", "achieved": round(ach, 3), "peak": round(fp32_peak, 2),
                "unit": "TFLOP/s", "frac": round(ach / fp32_peak, 4),
                "peak_source": (f"derived: {peak_inputs['sms']} SMs (device properties) x {FP32_LANES_PER_SM} FP32 "
                                f"lanes x 2 x {peak_inputs['sm_max_mhz']:.0f} MHz ({peak_inputs['mhz_source']}); "
                                "MEASURED_PEAKS.json has no FP32 figure"),
                "peak_inputs": peak_inputs,
                "flop_per_launch": flops[dom], "flop_convention": conv,
                "kernel_ms": round(stage_ms[dom], 4), "traffic": None}
    else:
        ach = bytes_.get(dom, 0) / (stage_ms[dom] * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(ach / hbm_peak, 4), "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                "traffic": None}
    if dom == "raster_bwd":
        roof["kernel"] = "raster_bwd_splat" if args.backward == "splat" else "raster_bwd"
    traffic = load_traffic(roof["kernel"])
    if traffic is not None:
        roof["traffic"] = traffic

    out = {
        "metric": METRIC, "value": round(replicas.job_rate(frame.n_views, world, ms), 2), "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": round(ms, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded surface-patch scene standing in for MipNeRF-360-scale captures)",
        "config": {"workload": WORKLOAD, "n_gaussians": sc.n, "sh_degree": sc.sh_degree,
                   "width": sc.cameras[0].width, "height": sc.cameras[0].height, "tile": args.tile,
                   "backward": args.backward, "views_per_step": frame.n_views, "duplicates_M": M, "pairs_examined": p_exam,
                   "pairs_walked_bwd": p_walk_bwd,
                   "pairs_composited": p_contrib, "visible_gaussians": measure_capacity.n_visible,
                   "parallelism": f"replicas x{world}",
                   "l2": f"inputs larger than L2 ({read_bytes / 1e6:.0f} MB of parameters read by the "
                         f"projection per step, {param_bytes / 1e6:.0f} MB resident)"},
        "e2e": {"value": round(replicas.job_rate(frame.n_views, world, e2e_ms), 2), "unit": UNIT,
                "h2d_bytes_per_step": int(step.target.numel() * 4 + step.frame.cams_dev.numel()),
                "d2h_bytes_per_step": int(step.loss.numel() * 4)},
        "gpu_launches": int(launches) * args.steps,
        "gpu_launches_per_step": int(launches),
        "timing": {"value": "CUDA-graph replay of the step, events around the K replays",
                   "e2e": "every step: camera and target image from pinned host memory (the next "
                          "step's copied on a side stream into the second of two input buffers, each "
                          "with its own captured graph, while the current step runs), loss read back",
                   "stages": "the same step launched eagerly for K steps just before, events between stages",
                   "eager_ms_per_step": round(eager_ms, 4)},
        "roofline": roof,
        "stages": stages,
        "clocks": clk,
        "memory": {**{k + "_mb": round(v / 1e6, 1) for k, v in step.memory_bytes().items()},
                   "peak_allocated_gb": round(torch.cuda.max_memory_allocated(dev) / 1e9, 3)},
    }
    if rank == 0 and not args.no_batched:
        out["batched"] = bench_batched(args, dev)
        out["batched_orbit"] = bench_batched_orbit(args, dev)
    if rank == 0 and not args.no_densify:
        out["densify"] = bench_densify(args, dev)
    if rank == 0 and not args.no_large:
        out["large"] = bench_large(args, dev)
    return out


def tile_sync_stats(frame, counts):
    """Entries a tile's CTA walks (its pixels' maximum examined count, for every
    pixel) against the entries its pixels need (their own examined counts)."""
    import torch
    W, H = frame.views[0][:2]
    tw, th = frame.tile
    ex = counts[:, 0].view(H, W).double()
    gx, gy = (W + tw - 1) // tw, (H + th - 1) // th
    pad = torch.zeros(gy * th, gx * tw, dtype=torch.float64, device=ex.device)
    pad[:H, :W] = ex
    t = pad.view(gy, th, gx, tw).permute(0, 2, 1, 3).reshape(gy * gx, th * tw)
    walked = float(t.max(1).values.sum() * th * tw)
    need = float(ex.sum())
    # the same at warp granularity (16 x 4 pixel strips of a 16x16 tile)
    wv = pad.view(gy, th // 4, 4, gx, tw).permute(0, 3, 1, 2, 4).reshape(-1, 4 * tw)
    walked_w = float(wv.max(1).values.sum() * 4 * tw)
    return {"needed": need, "walked_tile": walked, "walked_warp": walked_w}


def rasterizer_code_hash():
    """sha256 of the rasterizer's code (raster.cu and gs_common.cuh without // comments,
    trailing blanks and empty lines): what the recorded DRAM counters were taken on."""
    import hashlib
    import re
    csrc = os.path.join(ROOT, "paper_2507_20239_gb300", "csrc")
    lines = []
    for name in ("raster.cu", "gs_common.cuh"):
        with open(os.path.join(csrc, name)) as f:
            for line in f:
                code = re.sub(r"//.*$", "", line.rstrip("\n")).rstrip()
                if code:
                    lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def load_traffic(kernel):
    """Per-launch DRAM bytes of a kernel from the committed ncu summary, used only
    while the rasterizer code is the one the counters were taken on."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        if rasterizer_code_hash() != t.get("code_sha256"):
            return None
        return t.get(kernel)
    except Exception:
        return None


def bench_batched(args, dev):
    """12 mixed-resolution views (4 x 312x207, 4 x 623x413, 4 x 1246x826) of a
    500k-Gaussian scene: the autotuner picks tile shape, fused sort bits and the
    backward's staging depth; then one launch per stage, CUDA-graph captured, against
    the same kernels launched view by view."""
    import torch
    from paper_2507_20239_gb300 import rasterizer as R, synth
    from paper_2507_20239_gb300.autotune import autotune
    from paper_2507_20239_gb300.step import TrainStep
    sc = synth.batched_scene(2)
    P = R.to_device_params(sc.params(), dev)
    tune = autotune(P, sc.sh_degree, sc.cameras, sc.targets, device=dev)
    cfg = tune.best
    step = TrainStep(P, sc.sh_degree, sc.cameras, sc.targets, cfg, device=dev)
    g = step.capture(warmup=3)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = max(5, args.steps // 2)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1) / reps
    # per-view form: the same kernels and knobs, one view per launch
    singles = [TrainStep(P, sc.sh_degree, [cam], [sc.targets[v]], cfg, device=dev)
               for v, cam in enumerate(sc.cameras)]
    for s1 in singles:
        s1.run()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        for s1 in singles:
            s1.run()
    e1.record()
    torch.cuda.synchronize()
    per_view_ms = e0.elapsed_time(e1) / reps
    # same accuracy: the batched images equal the per-view images
    step.run()
    torch.cuda.synchronize()
    same = all(torch.equal(step.frame.view_image(step.image, v), s1.frame.view_image(s1.image, 0))
               for v, s1 in enumerate(singles))
    nv = len(sc.cameras)
    return {"workload": "batched-500k-sh3-12views-mixed-res", "views_per_launch": nv,
            "batched_views_per_s": round(nv * 1000.0 / batched_ms, 2),
            "per_view_views_per_s": round(nv * 1000.0 / per_view_ms, 2),
            "batched_ms": round(batched_ms, 4), "per_view_ms": round(per_view_ms, 4),
            "images_identical": bool(same), "graph": True, "autotune": tune.as_dict()}


def bench_large(args, dev):
    """5M Gaussians, 4 views at 1600x1060 in one launch per stage (graph-replayed),
    with the per-pixel stop index stored by the forward and, as where memory binds,
    recomputed by the backward, and with the per-splat backward (which also holds
    the forward's checkpoints); device memory beside views/s for each."""
    import gc
    import torch
    from paper_2507_20239_gb300 import rasterizer as R, synth
    from paper_2507_20239_gb300.step import StepConfig, TrainStep, duplicates
    sc = synth.large_scene(4)
    P = R.to_device_params(sc.params(), dev)
    M = duplicates(P, sc.sh_degree, R.Frame(sc.cameras, device=dev))
    out = {"workload": "large-5M-sh3-4views-1600x1060", "n_gaussians": sc.n, "views_per_launch": len(sc.cameras),
           "duplicates_M": M}
    for mode, store, bwd in (("stop_stored", True, "pixel"), ("stop_recomputed", False, "pixel"),
                             ("per_splat", True, "splat")):
        gc.collect()
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        torch.cuda.reset_peak_memory_stats(dev)
        free0, _ = torch.cuda.mem_get_info(dev)
        base = torch.cuda.memory_allocated(dev)
        step = TrainStep(P, sc.sh_degree, sc.cameras, sc.targets, StepConfig(backward=bwd), device=dev,
                         capacity=int(M * 1.1) + 4096, store_stop=store)
        g = step.capture(warmup=2)
        for _ in range(2):
            g.replay()
        torch.cuda.synchronize()
        assert step.error() == 0, "duplicate capacity exceeded"
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = max(3, args.steps // 4)
        e0.record()
        for _ in range(reps):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        free1, _ = torch.cuda.mem_get_info(dev)
        out[mode] = {"views_per_s": round(len(sc.cameras) * 1000.0 / ms, 2), "ms_per_launch": round(ms, 4),
                     "peak_allocated_gb": round((torch.cuda.max_memory_allocated(dev) - base) / 1e9, 3),
                     "mem_get_info_delta_gb": round((free0 - free1) / 1e9, 3),
                     "ckpt_gb": round(step.memory_bytes()["ckpt"] / 1e9, 3)}
        del g, step
    return out


def bench_batched_orbit(args, dev, n_views=4):
    """The metric's own configuration batched: n_views orbit views of the 1.5M-Gaussian
    scene at 1246x826 rendered in one launch per stage (CUDA graph), beside the same
    views each in a single-view step (each its own CUDA graph, replayed one after
    the other); images identical."""
    import torch
    from paper_2507_20239_gb300 import rasterizer as R, synth
    from paper_2507_20239_gb300.step import StepConfig, TrainStep
    sc = make_scene(args.n, 0)
    cam0 = sc.cameras[0]
    rng = np.random.default_rng(7)
    c = cam0.center                               # (r cos e sin az, -r sin e, -r cos e cos az)
    az0 = math.atan2(float(c[0]), float(-c[2]))
    cams = [synth.orbit_camera(4.0, az0 + 2 * math.pi * k / n_views, 15.0, cam0.width, cam0.height, cam0.fx)
            for k in range(n_views)]
    targets = [rng.uniform(0, 1, (3, c.height, c.width)).astype(np.float32) for c in cams]
    P = R.to_device_params(sc.params(), dev)
    tile = tuple(int(x) for x in args.tile.split("x"))
    cfg = StepConfig(tile=tile, backward=args.backward)
    step = TrainStep(P, sc.sh_degree, cams, targets, cfg, device=dev)
    singles = [TrainStep(P, sc.sh_degree, [c], [t], cfg, device=dev) for c, t in zip(cams, targets)]
    g = step.capture(warmup=3)
    gs = [s1.capture(warmup=3) for s1 in singles]
    for _ in range(3):
        g.replay()
        for g1 in gs:
            g1.replay()
    torch.cuda.synchronize()
    assert step.error() == 0 and all(s1.error() == 0 for s1 in singles), "duplicate capacity exceeded"
    reps = max(5, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    batched_ms = e0.elapsed_time(e1) / reps
    e0.record()
    for _ in range(reps):
        for g1 in gs:
            g1.replay()
    e1.record()
    torch.cuda.synchronize()
    per_view_ms = e0.elapsed_time(e1) / reps
    same = all(torch.equal(step.frame.view_image(step.image, v), s1.frame.view_image(s1.image, 0))
               for v, s1 in enumerate(singles))
    M = int(step.bins.count.item())
    return {"workload": f"orbit-1.5M-sh3-{n_views}x1246x826", "n_gaussians": sc.n, "views_per_launch": n_views,
            "duplicates_M": M, "config": cfg.label(),
            "batched_views_per_s": round(n_views * 1000.0 / batched_ms, 2),
            "per_view_views_per_s": round(n_views * 1000.0 / per_view_ms, 2),
            "batched_ms": round(batched_ms, 4), "per_view_ms": round(per_view_ms, 4),
            "images_identical": bool(same), "graph": "both forms CUDA-graph replayed"}


def bench_densify(args, dev, n=1_200_000):
    """Densification event at the training workload's size (~1.2M Gaussians, SH degree
    3, Adam moments of all five groups carried through): gs_densify_select (fixed
    and adaptive pruning threshold) and gs_densify_apply, CUDA events around each,
    against the bytes they must move (select: log-scales, statistics, logits, masks;
    apply: N x 708 B read and N' x 708 B written: parameters and both moments, plus
    the masks)."""
    import torch
    from paper_2507_20239_gb300 import rasterizer as R, synth
    sc = synth.surface_scene(3, n, 3)
    P = R.to_device_params(sc.params(), dev)
    rng = np.random.default_rng(8)
    # view-space gradient statistic: visible in 0-11 views, average norm log-normal
    # around half the 2e-4 threshold (about 6% of the Gaussians exceed it)
    count = rng.integers(0, 12, n).astype(np.int32)
    avg = np.exp(rng.normal(math.log(1e-4), 0.45, n))
    accum = torch.as_tensor((avg * count).astype(np.float32), device=dev)
    count = torch.as_tensor(count, device=dev)
    moments = {f"{w}_{k}": torch.as_tensor(rng.normal(0, 1e-3, tuple(P[k].shape)).astype(np.float32)).to(dev)
               for w in ("m", "v") for k in R.PARAM_KEYS}
    thr_s = float(np.float32(math.log(0.01 * 4.4)))
    fixed = R.densify_cfg(mode=R.DENSIFY_ADAPTIVE, log_scale_threshold=thr_s,
                          prune_logit=float(np.float32(math.log(0.005 / 0.995))), seed=3, event=1)
    adaptive = R.densify_cfg(mode=R.DENSIFY_ADAPTIVE, log_scale_threshold=thr_s, prune_ratio=0.03,
                             prune_upper_logit=float(np.float32(math.log(0.05 / 0.95))), seed=3, event=1)
    split, clone, tau, new_n, ws = R.densify_select(fixed, P, accum, count)
    torch.cuda.synchronize()
    cap = int(new_n.item())
    out = {k: torch.empty((cap,) + tuple(P[k].shape[1:]), device=dev) for k in R.PARAM_KEYS}
    ex_out = {k: torch.empty((cap,) + tuple(v.shape[1:]), device=dev) for k, v in moments.items()}
    got_n = torch.empty(1, dtype=torch.int64, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    sel_out = (split, clone, tau, new_n)
    reps = 20

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    sel_ms = timed(lambda: R.densify_select(fixed, P, accum, count, ws=ws, out=sel_out))
    apply_ms = timed(lambda: R.densify_apply(fixed, P, sc.sh_degree, split, clone, tau, cap, extra=moments, ws=ws,
                                             out=out, ex_out=ex_out, new_n=got_n, err=err))
    assert int(err.item()) == 0 and int(got_n.item()) == cap
    n_split, n_clone = int(split.sum().item()), int(clone.sum().item())
    sel_ad_ms = timed(lambda: R.densify_select(adaptive, P, accum, count, ws=ws, out=sel_out))
    hbm = float(load_peaks().get("hbm_gbs", 6800.0))
    row = 4 * (3 + 3 + 4 + 1 + 3 * sc.sh.shape[1])          # 236 B of parameters per Gaussian
    sel_bytes = n * (12 + 4 + 4 + 2 + 4 + 2)
    apply_bytes = n * 3 * row + cap * 3 * row + 2 * n
    return {"workload": f"densify-{n / 1e6:.1f}M-sh3-adam", "n": n, "n_after": cap, "splits": n_split,
            "clones": n_clone, "select_ms": round(sel_ms, 4), "select_adaptive_ms": round(sel_ad_ms, 4),
            "apply_ms": round(apply_ms, 4),
            "select_bytes": sel_bytes, "apply_bytes": apply_bytes,
            "select_frac": round(sel_bytes / (sel_ms * 1e-3) / 1e9 / hbm, 4),
            "apply_frac": round(apply_bytes / (apply_ms * 1e-3) / 1e9 / hbm, 4),
            "frac": round(apply_bytes / (apply_ms * 1e-3) / 1e9 / hbm, 4),
            "peak": "MEASURED_PEAKS.json hbm_gbs (of measured)"}


# ----------------------------------------------------------------------------------------
def oracle_view_seconds(sc, n_tiles_sample, seed=0, vjp_sample=100_000):
    """Time the FP64 oracle on a bounded sample of one training view and scale it to
    a whole view: projection of all Gaussians, tile binning, compositing + backward of
    n_tiles_sample tiles (scaled by tiles), projection VJP of a Gaussian sample
    (scaled by count). Returns (seconds per whole view, wall seconds spent, sample
    description, threads torch was allowed, cores actually used = process CPU
    time / wall time over the sample)."""
    import torch
    from oracle import project as oproj, raster as oras, pipeline as opipe
    cam = sc.cameras[0]
    cpu0 = time.process_time()
    w0 = time.perf_counter()
    t0 = time.perf_counter()
    pr = oproj.project_np(sc.params(), sc.sh_degree, cam)
    t_proj = time.perf_counter() - t0
    gx, gy = pr["grid"]
    t0 = time.perf_counter()
    lists = oras.tile_lists(opipe.proj_record_arrays(pr), cam.width, cam.height)
    t_bin = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    busy = [t for t, l in lists.items() if len(l)]
    tiles = sorted(rng.choice(busy, min(n_tiles_sample, len(busy)), replace=False).tolist())
    d_image = rng.normal(0, 1, (3, cam.height, cam.width))
    t0 = time.perf_counter()
    oras.raster_vjp(pr["mean2d"], pr["conic_f"], pr["opacity"], pr["rgb"], lists, cam.width, cam.height, d_image,
                    tiles=tiles)
    t_tiles = time.perf_counter() - t0
    n_s = min(sc.n, vjp_sample)
    sub = {k: v[:n_s] for k, v in sc.params().items()}
    g = dict(d_mean2d=rng.normal(size=(n_s, 2)), d_conic=rng.normal(size=(n_s, 3)), d_opacity=rng.normal(size=n_s),
             d_rgb=rng.normal(size=(n_s, 3)))
    t0 = time.perf_counter()
    opipe.project_vjp(sub, sc.sh_degree, [cam], [g])
    t_vjp = time.perf_counter() - t0
    total = t_proj + t_bin + t_tiles * gx * gy / len(tiles) + t_vjp * sc.n / n_s
    spent = t_proj + t_bin + t_tiles + t_vjp
    used = (time.process_time() - cpu0) / max(time.perf_counter() - w0, 1e-9)
    sample = (f"1 view of {WORKLOAD}: projection of all {sc.n} Gaussians, binning, Eq. 2 forward+backward on "
              f"{len(tiles)} of {gx * gy} tiles (x{gx * gy / len(tiles):.1f}), projection VJP on {n_s} Gaussians "
              f"(x{sc.n / n_s:.1f}); {spent:.1f} s wall")
    return total, spent, sample, torch.get_num_threads(), used


def cpu_baseline(sc, n_tiles):
    """The oracle with every host core torch may use, then on one thread (a smaller
    sample, scaled the same way); cores = CPU time / wall time actually measured."""
    import torch
    total, spent, sample, threads, used = oracle_view_seconds(sc, n_tiles)
    nthreads = torch.get_num_threads()
    torch.set_num_threads(1)
    try:
        t1, s1, sample1, _, used1 = oracle_view_seconds(sc, max(8, n_tiles // 4), vjp_sample=25_000)
    finally:
        torch.set_num_threads(nthreads)
    return {"value": round(1.0 / total, 6), "unit": UNIT, "cores": round(used, 1), "kind": "oracle",
            "sample": sample, "threads_allowed": threads, "host_cores": len(os.sched_getaffinity(0)),
            "single_thread": {"value": round(1.0 / t1, 6), "unit": UNIT, "cores": round(used1, 1),
                              "sample": sample1}}


class OracleReference:
    """The FP64 oracle as the reference arm's program. Set-up runs the projection of
    all Gaussians and the tile binning once (timed: the binning's time enters every
    step's estimate, and its lists are what the sampled tiles walk); each step then
    times a fresh bounded sample of the view -- the projection of a random tenth of
    the Gaussians, Eq. 2 forward + backward on sampled tiles, the projection VJP on a
    Gaussian sample -- and scales each part to the whole view."""

    def __init__(self, sc, tiles=20, proj_frac=0.1, vjp_sample=25_000):
        from oracle import project as oproj, raster as oras, pipeline as opipe
        self.sc, self.cam = sc, sc.cameras[0]
        self.tiles, self.proj_n, self.vjp_n = tiles, max(1, int(sc.n * proj_frac)), min(sc.n, vjp_sample)
        self.params = sc.params()
        self.pr = oproj.project_np(self.params, sc.sh_degree, self.cam)
        t0 = time.perf_counter()
        self.lists = oras.tile_lists(opipe.proj_record_arrays(self.pr), self.cam.width, self.cam.height)
        self.t_bin = time.perf_counter() - t0
        self.busy = [t for t, l in self.lists.items() if len(l)]
        self.n_tiles = self.pr["grid"][0] * self.pr["grid"][1]

    def step(self, seed):
        """(seconds per whole view, wall seconds of this step, cores used)."""
        from oracle import project as oproj, raster as oras, pipeline as opipe
        sc, cam, rng = self.sc, self.cam, np.random.default_rng(seed)
        cpu0, w0 = time.process_time(), time.perf_counter()
        idx = np.sort(rng.choice(sc.n, self.proj_n, replace=False))
        sub = {k: v[idx] for k, v in self.params.items()}
        t0 = time.perf_counter()
        oproj.project_np(sub, sc.sh_degree, cam)
        t_proj = time.perf_counter() - t0
        tiles = sorted(rng.choice(self.busy, min(self.tiles, len(self.busy)), replace=False).tolist())
        d_image = rng.normal(0, 1, (3, cam.height, cam.width))
        pr = self.pr
        t0 = time.perf_counter()
        oras.raster_vjp(pr["mean2d"], pr["conic_f"], pr["opacity"], pr["rgb"], self.lists, cam.width, cam.height,
                        d_image, tiles=tiles)
        t_tiles = time.perf_counter() - t0
        vi = np.sort(rng.choice(sc.n, self.vjp_n, replace=False))
        vsub = {k: v[vi] for k, v in self.params.items()}
        n_s = self.vjp_n
        g = dict(d_mean2d=rng.normal(size=(n_s, 2)), d_conic=rng.normal(size=(n_s, 3)),
                 d_opacity=rng.normal(size=n_s), d_rgb=rng.normal(size=(n_s, 3)))
        t0 = time.perf_counter()
        opipe.project_vjp(vsub, sc.sh_degree, [cam], [g])
        t_vjp = time.perf_counter() - t0
        total = (t_proj * sc.n / self.proj_n + self.t_bin + t_tiles * self.n_tiles / len(tiles)
                 + t_vjp * sc.n / n_s)
        wall = time.perf_counter() - w0
        return total, wall, (time.process_time() - cpu0) / max(wall, 1e-9), len(tiles)

    def sample(self, n_tiles_used, wall):
        return (f"1 view of {WORKLOAD} per step: projection of {self.proj_n} of {self.sc.n} Gaussians "
                f"(x{self.sc.n / self.proj_n:.1f}), the tile binning of all of them timed once at set-up "
                f"({self.t_bin:.1f} s), Eq. 2 forward+backward on {n_tiles_used} of {self.n_tiles} tiles "
                f"(x{self.n_tiles / n_tiles_used:.1f}), projection VJP on {self.vjp_n} Gaussians "
                f"(x{self.sc.n / self.vjp_n:.1f}); {wall:.1f} s wall per step")


def bench_reference(args, rank, world):
    """The FP64 oracle as the reference arm, on the host cores: W warm-up and K timed
    steps, each a bounded sample of the view (OracleReference)."""
    if rank != 0:
        return None
    sc = make_scene(args.n, 0)
    ref = OracleReference(sc)
    for k in range(args.warmup):
        ref.step(seed=1000 + k)
    times, walls, used_all, nt = [], [], [], 0
    for k in range(args.steps):
        total, wall, used, nt = ref.step(seed=k)
        times.append(total)
        walls.append(wall)
        used_all.append(used)
    # value: the views/s that the steps' samples imply for whole views; ms_per_step:
    # the measured wall time of a step (one sample)
    v = round(1.0 / statistics.mean(times), 6)
    sample = ref.sample(nt, statistics.mean(walls))
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1000.0 * statistics.mean(walls), 1), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "n_gaussians": sc.n, "width": sc.cameras[0].width,
                       "height": sc.cameras[0].height, "tile": "16x16"},
            "view_fraction_per_step": round(statistics.mean(walls) / statistics.mean(times), 4),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": round(statistics.mean(used_all), 1), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, local_rank, world = dist_info()
    if args.impl == "reference":
        if world > 1 and rank != 0:
            return
        out = bench_reference(args, rank, world)
        print(json.dumps(out), flush=True)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    out = bench_ours(args, rank, local_rank, world)
    if out is not None and rank == 0:
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_baseline(make_scene(args.n, 0), args.cpu_sample_tiles)
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
