"""The training step's loss and optimiser on the library's kernels.

photometric_loss_grad: Eq. 3, (1 - lambda) L1 + lambda D-SSIM per view, and its
gradient w.r.t. the rendered image (gs_photometric_loss_grad). Adam: moments held
as device tensors, one fused kernel per step for all five parameter groups
(gs_adam_step), optionally sparse (only Gaussians some view of the step saw).
opacity_reset: the schedule's periodic opacity reset (gs_opacity_reset).
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import torch

from . import _abi
from ._abi import check
from .rasterizer import PARAM_KEYS, Frame, _p, _stream, lib


def photometric_loss_grad(frame: Frame, image: torch.Tensor, target: torch.Tensor, lam: float = 0.2,
                          d_image=None, loss=None, ws=None, stream=None):
    d_image = torch.empty_like(image) if d_image is None else d_image
    loss = torch.empty(frame.n_views, dtype=torch.float32, device=frame.device) if loss is None else loss
    if ws is None:
        ws = torch.empty(lib().gs_photometric_workspace_size(C.byref(frame.frame)), dtype=torch.uint8,
                         device=frame.device)
    check(lib().gs_photometric_loss_grad(C.byref(frame.frame), _p(image), _p(target), float(lam), _p(d_image),
                                         _p(loss), _p(ws), ws.numel(), _stream(stream)), "gs_photometric_loss_grad")
    return d_image, loss


class Adam:
    """Adam over the five parameter groups (means, log_scales, quats,
    opacity_logits, sh) with per-group learning rates."""

    def __init__(self, params: dict, lrs: dict, betas=(0.9, 0.999), eps=1e-15):
        self.lrs = dict(lrs)
        self.betas, self.eps = betas, eps
        self.m = {k: torch.zeros_like(params[k]) for k in PARAM_KEYS}
        self.v = {k: torch.zeros_like(params[k]) for k in PARAM_KEYS}
        self.t = 0

    def _state(self):
        st = _abi.GsAdamState()
        for i, k in enumerate(PARAM_KEYS):
            st.m[i], st.v[i] = self.m[k].data_ptr(), self.v[k].data_ptr()
        return st

    def step(self, params: dict, grads: dict, radius: Optional[torch.Tensor] = None, n_views: int = 1,
             stream=None):
        """In-place update of params from grads; radius ([n_views * N] int32, the
        step's projection) makes it sparse."""
        self.t += 1
        cfg = _abi.GsAdamCfg()
        for i, k in enumerate(PARAM_KEYS):
            cfg.lr[i] = float(self.lrs[k])
        cfg.beta1, cfg.beta2, cfg.eps, cfg.step = self.betas[0], self.betas[1], self.eps, self.t
        po = _abi.GsParamsOut()
        po.means, po.log_scales, po.quats = params["means"].data_ptr(), params["log_scales"].data_ptr(), \
            params["quats"].data_ptr()
        po.opacity_logits, po.sh = params["opacity_logits"].data_ptr(), params["sh"].data_ptr()
        g = _abi.GsParamGrads()
        g.d_means, g.d_log_scales, g.d_quats = grads["means"].data_ptr(), grads["log_scales"].data_ptr(), \
            grads["quats"].data_ptr()
        g.d_opacity_logits, g.d_sh = grads["opacity_logits"].data_ptr(), grads["sh"].data_ptr()
        n = params["means"].shape[0]
        sh_stride = params["sh"].shape[1]
        check(lib().gs_adam_step(C.byref(cfg), C.byref(po), n, sh_stride, C.byref(g), C.byref(self._state()),
                                 _p(radius) if radius is not None else None, int(n_views), _stream(stream)),
              "gs_adam_step")

    def moments(self) -> dict:
        """Moments as [N, width] arrays keyed 'group.m' / 'group.v' (for compaction)."""
        out = {}
        for k in PARAM_KEYS:
            n = self.m[k].shape[0]
            out[k + ".m"] = self.m[k].reshape(n, -1)
            out[k + ".v"] = self.v[k].reshape(n, -1)
        return out

    def set_moments(self, arrays: dict, params: dict):
        for k in PARAM_KEYS:
            self.m[k] = arrays[k + ".m"].reshape(params[k].shape).contiguous()
            self.v[k] = arrays[k + ".v"].reshape(params[k].shape).contiguous()


def opacity_reset(params: dict, adam: Optional[Adam] = None, max_opacity: float = 0.01, stream=None):
    lg = params["opacity_logits"]
    m = adam.m["opacity_logits"] if adam is not None else None
    v = adam.v["opacity_logits"] if adam is not None else None
    check(lib().gs_opacity_reset(_p(lg), _p(m) if m is not None else None, _p(v) if v is not None else None,
                                 lg.shape[0], float(max_opacity), _stream(stream)), "gs_opacity_reset")
