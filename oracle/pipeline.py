"""One training view end to end (FP64) -- test infrastructure only.

project (EWA, SH colour) -> tile lists (rect decided in FP64, key = FP32 depth)
-> Eq. 2 compositing -> L1 loss (the L1 part of Eq. 3) -> gradients of the loss
w.r.t. every Gaussian parameter, by the chain rule: the compositing VJP gives
gradients of the projected records, and reverse-mode differentiation of the
projection carries them to means, log-scales, quaternions, opacity logits and SH.
"""
from __future__ import annotations

import numpy as np
import torch

from .project import project, params_to_torch
from .raster import tile_lists, raster_vjp, rasterize, records_to_torch
from .loss import l1_loss_grad

PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")


def project_vjp(params: dict, sh_degree: int, cams: list, rec_grads: list, tile_w=16, tile_h=16):
    """Gradients of sum_v <records_v, rec_grads_v> w.r.t. the parameters.

    rec_grads[v] is a dict d_mean2d [N,2], d_conic [N,3] (w.r.t. the factored conic
    (A, beta, gamma)), d_opacity [N], d_rgb [N,3] for view v; the parameter gradients are summed over views. Also returns the
    per-view NDC-space mean2D gradients (d_u W/2, d_v H/2)."""
    p = params_to_torch(params, requires_grad=True)
    outs, grads = [], []
    for cam, g in zip(cams, rec_grads):
        pr = project(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["sh"],
                     sh_degree, cam, tile_w, tile_h)
        outs += [pr["mean2d"], pr["conic_f"], pr["opacity"], pr["rgb"]]
        grads += [torch.as_tensor(np.asarray(g[k], np.float64))
                  for k in ("d_mean2d", "d_conic", "d_opacity", "d_rgb")]
    torch.autograd.backward(outs, grads)
    return {k: (p[k].grad.numpy() if p[k].grad is not None else np.zeros(p[k].shape))
            for k in PARAM_KEYS}


def proj_record_arrays(proj: dict) -> dict:
    """The arrays binning needs, in FP64 (depth keys are FP32 by definition)."""
    return dict(mean2d=proj["mean2d"], conic_f=proj["conic_f"], q_max=proj["q_max"], rect=proj["rect"],
                depth=proj["depth"].astype(np.float32))


def render_view(params: dict, sh_degree: int, cam, target=None, tile_w=16, tile_h=16,
                bg=(0.0, 0.0, 0.0), tiles=None, d_image=None, rec_delta=None):
    """Forward (and, given a target or d_image, backward) of one view.

    Returns a dict with the projection (numpy), the render outputs, the loss and
    d_image when a target is given, record gradients and parameter gradients.
    rec_delta [N,6]: differences of the records another implementation computed
    (see raster.composite; they widen the straddle flags).
    """
    p = params_to_torch(params)
    with torch.no_grad():
        pr = project(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["sh"],
                     sh_degree, cam, tile_w, tile_h)
    proj = {k: (v.numpy() if isinstance(v, torch.Tensor) else v) for k, v in pr.items()}
    lists = tile_lists(proj_record_arrays(proj), cam.width, cam.height, tile_w, tile_h)
    res = dict(proj=proj, lists=lists)
    if target is None and d_image is None:
        rec = records_to_torch(proj["mean2d"], proj["conic_f"], proj["opacity"], proj["rgb"])
        with torch.no_grad():
            res["render"] = rasterize(rec, lists, cam.width, cam.height, tile_w, tile_h, bg, tiles,
                                      rec_delta=rec_delta)
        return res
    if d_image is None:
        with torch.no_grad():
            rec = records_to_torch(proj["mean2d"], proj["conic_f"], proj["opacity"], proj["rgb"])
            fwd = rasterize(rec, lists, cam.width, cam.height, tile_w, tile_h, bg, tiles, rec_delta=rec_delta)
        loss, d_image = l1_loss_grad(fwd["image"], target)
        res["loss"] = loss
    res["d_image"] = d_image
    out, g = raster_vjp(proj["mean2d"], proj["conic_f"], proj["opacity"], proj["rgb"], lists,
                        cam.width, cam.height, d_image, tile_w, tile_h, bg, tiles, rec_delta)
    res["render"] = out
    res["rec_grads"] = g
    res["param_grads"] = project_vjp(params, sh_degree, [cam], [g], tile_w, tile_h)
    return res
