"""One training view through the hot path, with every buffer preallocated.

TrainStep runs, on the current stream: gs_project -> gs_bin_sort -> gs_raster_fwd
(Eq. 2) -> gs_l1_loss_grad (the L1 term of Eq. 3) -> gs_raster_bwd ->
gs_project_bwd (parameter gradients and the densification statistic); with the
per-splat backward, gs_raster_fwd_ckpt and gs_raster_bwd_splat take the raster
stages. With store_stop the forward stores each pixel's stop index and the
backward walks only up to it; without, no per-pixel index is kept and the
backward recomputes the cut-off (4 bytes per pixel less). No count returns to the host inside run(), so
the sequence can be captured once into a CUDA graph (capture()) and replayed.

The duplicate capacity of the per-tile lists is sized from a measured M with
headroom, and the per-splat forward's checkpoint slots from a measured count with
the same headroom; gs_bin_sort raises its device error word if a later view exceeds
the capacity, and error() also reports a forward that ran out of checkpoint slots
(check it outside any graph).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import rasterizer as R
from .autograd import DensifyStats


BACKWARDS = ("pixel", "splat")


@dataclass(frozen=True)
class StepConfig:
    """Tuning knobs of one step (none changes the images; gradients agree up to
    summation order): tile shape, low tile-id bits sorted during emission
    (0 = the library's choice), the backward's staging depth (0 = one list entry
    per thread per CTA step, 1 = half as many) and the backward itself ("pixel":
    gs_raster_bwd, parallel over pixels; "splat": gs_raster_bwd_splat, parallel over
    list entries from checkpoints the forward stores; the staging depth does not
    apply to it)."""
    tile: tuple = (16, 16)
    sort_fused_bits: int = 0
    stage_depth: int = 0
    backward: str = "pixel"
    queue: bool = False      # the forward as a persistent grid claiming (tile, block) units

    def __post_init__(self):
        if self.backward not in BACKWARDS:
            raise ValueError(f"backward must be one of {BACKWARDS}, not {self.backward!r}")

    def label(self) -> str:
        q = "/queue" if self.queue else ""
        if self.backward == "splat":
            return f"{self.tile[0]}x{self.tile[1]}/f{self.sort_fused_bits}/splat{q}"
        return f"{self.tile[0]}x{self.tile[1]}/f{self.sort_fused_bits}/s{self.stage_depth}{q}"


def duplicates(params: dict, sh_degree: int, frame: R.Frame) -> int:
    """M for these parameters on this frame (one projection and binning, synchronising)."""
    proj = R.project(params, sh_degree, frame)
    bins = R.bin_sort(proj, frame)
    return int(bins.count.item())


class TrainStep:
    def __init__(self, params: dict, sh_degree: int, cameras, target_images, config: StepConfig = StepConfig(),
                 device="cuda", capacity: int | None = None, headroom: float = 1.25, store_stop: bool = True,
                 slots: int | None = None):
        self.P, self.sh_degree, self.config = params, int(sh_degree), config
        self.splat = config.backward == "splat"
        self.store_stop = bool(store_stop) or self.splat   # the per-splat backward needs the stop indices
        self.frame = R.Frame(cameras, tile=config.tile, device=device, sort_fused_bits=config.sort_fused_bits)
        f = self.frame
        n = params["means"].shape[0]
        if capacity is None:
            capacity = int(duplicates(params, sh_degree, f) * headroom) + 4096
        Rn = f.n_views * n
        self.proj = R.Projected.empty(Rn, f.device)
        self.bins = R.alloc_bins(f, Rn, capacity)
        self.image = torch.empty(3 * f.n_pixels, device=f.device)
        self.T = torch.empty(f.n_pixels, device=f.device)
        self.stop = torch.empty(f.n_pixels, dtype=torch.int32, device=f.device) if self.store_stop else None
        self.ckpt = None
        if self.splat:
            # checkpoint slots for the (bucket, block) pairs the forward walks, measured
            # on the step's own buffers (a forward into a checkpoint buffer without
            # slots reports the count), reserved with headroom; -1: one per possible pair
            self.ckpt_use = torch.zeros(2, dtype=torch.int64, device=f.device)
            if slots is None:
                probe = R.alloc_ckpt(f, self.bins, 0)
                R.project(params, sh_degree, f, out=self.proj)
                R.bin_sort_into(self.proj, f, self.bins)
                R.raster_fwd_ckpt(self.proj, self.bins, f, probe, image=self.image, T_final=self.T, stop=self.stop)
                R.ckpt_usage(f, self.bins, probe, out=self.ckpt_use)
                if int(self.bins.error.item()) != 0:
                    raise RuntimeError("TrainStep: duplicate capacity exceeded while sizing the checkpoints")
                slots = int(int(self.ckpt_use[0].item()) * headroom) + 4 * 256
                del probe
            self.ckpt = R.alloc_ckpt(f, self.bins, slots)
        self.queue = torch.zeros(1, dtype=torch.int32, device=f.device) if config.queue else None
        self.d_image = torch.empty_like(self.image)
        self.loss = torch.empty(f.n_views, device=f.device)
        self.target = f.pack_images(target_images).contiguous()
        self.rec = R.RecGrads.zeros(Rn, f.device)
        self.pgrads = R.empty_param_grads(params)
        self.stats = DensifyStats.zeros(n, f.device)

    def run(self, events=None):
        """Enqueue the step; events (7 CUDA events or None) bracket the six stages."""
        f, cfg = self.frame, self.config
        ev = events or [None] * 7
        rec = lambda i: ev[i].record() if ev[i] is not None else None
        rec(0)
        R.project(self.P, self.sh_degree, f, out=self.proj)
        rec(1)
        R.bin_sort_into(self.proj, f, self.bins)
        rec(2)
        if self.splat:
            R.raster_fwd_ckpt(self.proj, self.bins, f, self.ckpt, image=self.image, T_final=self.T, stop=self.stop,
                              queue=self.queue)
        else:
            R.raster_fwd(self.proj, self.bins, f, image=self.image, T_final=self.T, store_stop=self.store_stop,
                         stop=self.stop, queue=self.queue)
        rec(3)
        R.l1_loss_grad(f, self.image, self.target, d_image=self.d_image, loss=self.loss)
        rec(4)
        if self.splat:
            R.raster_bwd_splat(self.proj, self.bins, f, self.image, self.d_image, self.stop, self.ckpt,
                               grads=self.rec)
        else:
            R.raster_bwd(self.proj, self.bins, f, self.image, self.d_image, grads=self.rec, stop=self.stop,
                         stage_depth=cfg.stage_depth)
        rec(5)
        R.project_bwd(self.P, self.sh_degree, f, self.proj, self.rec, out=self.pgrads,
                      accum=self.stats.accum, count=self.stats.count)
        rec(6)

    def capture(self, warmup: int = 1) -> torch.cuda.CUDAGraph:
        """The step captured once into a CUDA graph, after warm-up on a side stream
        as capture requires."""
        side = torch.cuda.Stream(device=self.frame.device)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(max(1, warmup)):
                self.run()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run()
        return g

    def error(self) -> int:
        """gs_bin_sort's device error word (0: every list fitted the capacity), with
        GS_ERR_CAPACITY also set when the per-splat forward ran out of checkpoint slots."""
        err = int(self.bins.error.item())
        if self.ckpt is not None:
            R.ckpt_usage(self.frame, self.bins, self.ckpt, out=self.ckpt_use)
            if int(self.ckpt_use[1].item()):
                err |= 2
        return err

    def memory_bytes(self) -> dict:
        """Device bytes of the step's largest buffers."""
        nb = lambda t: 0 if t is None else t.numel() * t.element_size()
        return {"bins": nb(self.bins.vals) + nb(self.bins.ws) + nb(self.bins.keys), "ckpt": nb(self.ckpt),
                "records": sum(nb(getattr(self.proj, k)) for k in ("mean2d", "conic_opacity", "rgb", "depth",
                                                                     "radius", "rect", "clamped"))}
