"""torch.autograd.Function around the CUDA rasterizer.

forward: gs_project -> gs_bin_sort -> gs_raster_fwd (images of every view, planar,
concatenated). backward: gs_raster_bwd (record gradients) -> gs_project_bwd
(parameter gradients, summed over views), with the densification statistic
accumulated on the way when a DensifyStats object is passed. With
backward="splat" the raster stages are gs_raster_fwd_ckpt / gs_raster_bwd_splat
(the same gradients up to summation order; the forward's checkpoints are held
until the backward).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import torch

from . import rasterizer as R


@dataclass
class DensifyStats:
    accum: torch.Tensor    # [N] float32
    count: torch.Tensor    # [N] int32
    radius: Optional[torch.Tensor] = None   # [V * N] int32: the last forward's record radii

    @staticmethod
    def zeros(n, device="cuda"):
        return DensifyStats(torch.zeros(n, dtype=torch.float32, device=device),
                            torch.zeros(n, dtype=torch.int32, device=device))


class _Rasterize(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logits, sh, sh_degree, frame, bg, stats, splat):
        params = dict(means=means.contiguous(), log_scales=log_scales.contiguous(), quats=quats.contiguous(),
                      opacity_logits=opacity_logits.contiguous(), sh=sh.contiguous())
        proj = R.project(params, sh_degree, frame)
        bins = R.bin_sort(proj, frame)
        ckpt = None
        if splat:
            ckpt = R.alloc_ckpt(frame, bins)
            image, T_final, stop = R.raster_fwd_ckpt(proj, bins, frame, ckpt, bg)
        else:
            image, T_final, stop = R.raster_fwd(proj, bins, frame, bg, store_stop=True)
        if stats is not None:
            stats.radius = proj.radius
        ctx.save_for_backward(*[params[k] for k in R.PARAM_KEYS])
        ctx.state = (proj, bins, frame, bg, sh_degree, stats, image, stop, ckpt)
        ctx.mark_non_differentiable(T_final)
        return image, T_final

    @staticmethod
    def backward(ctx, d_image, _d_T):
        proj, bins, frame, bg, sh_degree, stats, image, stop, ckpt = ctx.state
        params = dict(zip(R.PARAM_KEYS, ctx.saved_tensors))
        if ckpt is not None:
            rec = R.raster_bwd_splat(proj, bins, frame, image, d_image.contiguous(), stop, ckpt)
        else:
            rec = R.raster_bwd(proj, bins, frame, image, d_image.contiguous(), bg, stop=stop)
        acc = cnt = None
        if stats is not None:
            acc, cnt = stats.accum, stats.count
        g = R.project_bwd(params, sh_degree, frame, proj, rec, accum=acc, count=cnt)
        ctx.state = None
        return g["means"], g["log_scales"], g["quats"], g["opacity_logits"], g["sh"], None, None, None, None, None


def rasterize(params: dict, sh_degree: int, frame, bg=(0.0, 0.0, 0.0), stats: DensifyStats = None,
              backward: str = "pixel"):
    """Differentiable render of every view of `frame`; returns (image, T_final), the
    image planar per view and concatenated (see Frame.view_image). backward: "pixel"
    (gs_raster_bwd) or "splat" (gs_raster_bwd_splat)."""
    if backward not in ("pixel", "splat"):
        raise ValueError(f"backward must be 'pixel' or 'splat', not {backward!r}")
    return _Rasterize.apply(params["means"], params["log_scales"], params["quats"], params["opacity_logits"],
                            params["sh"], int(sh_degree), frame, tuple(float(b) for b in bg), stats,
                            backward == "splat")
