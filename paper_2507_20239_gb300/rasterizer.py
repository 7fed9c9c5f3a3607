"""Torch-facing binding of libgs: tensors in, tensors out, every step in CUDA.

Each function only marshals arguments (device pointers, sizes, the current CUDA
stream) into the matching C-ABI call of include/gs.h; buffers are torch tensors
on the GPU. There is no CPU fallback: a missing library or a non-CUDA tensor
raises.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import torch

from . import _abi
from ._abi import check

PARAM_KEYS = ("means", "log_scales", "quats", "opacity_logits", "sh")
DENSIFY_ADAPTIVE, DENSIFY_SPLIT_ONLY, DENSIFY_ALL_SPLIT, DENSIFY_ALL_CLONE = 0, 1, 2, 3


def lib():
    return _abi.load()


def _p(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(s.cuda_stream)


def _need(t: torch.Tensor, dtype, name, align=4):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.data_ptr() % align:
        raise ValueError(f"{name} must be {align}-byte aligned")
    return t


def _bytes(n, device):
    return torch.empty(max(int(n), 256), dtype=torch.uint8, device=device)


# ----------------------------------------------------------------------------------------
class Frame:
    """A batch of views rendered together (gs_frame_t + a device copy of the cameras)."""

    def __init__(self, cameras, tile=(16, 16), device="cuda", sort_fused_bits=0):
        n = len(cameras)
        arr = (_abi.GsCamera * n)()
        for i, cam in enumerate(cameras):
            c = arr[i]
            R = np.asarray(cam.R, np.float32).reshape(9)
            t = np.asarray(cam.t, np.float32).reshape(3)
            for k in range(9):
                c.R[k] = float(R[k])
            for k in range(3):
                c.t[k] = float(t[k])
            c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
            c.width, c.height = int(cam.width), int(cam.height)
            c.near_plane = float(getattr(cam, "near", 0.2))
        self.frame = _abi.GsFrame()
        check(lib().gs_frame_init(arr, n, int(tile[0]), int(tile[1]), C.byref(self.frame)), "gs_frame_init")
        # low tile-id bits gs_bin_sort sorts while emitting (0 = its own choice)
        self.frame.sort_fused_bits = int(sort_fused_bits)
        self.cams_host = arr
        raw = bytes(C.string_at(C.addressof(arr), C.sizeof(arr)))
        self.cams_dev = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)
        self.frame.cams_dev = self.cams_dev.data_ptr()
        self.cameras = list(cameras)
        self.tile = (int(tile[0]), int(tile[1]))
        self.device = torch.device(device)
        self.views = [(arr[i].width, arr[i].height, arr[i].pixel_offset, arr[i].tile_offset,
                       arr[i].grid_x, arr[i].grid_y) for i in range(n)]

    @property
    def n_views(self):
        return self.frame.n_views

    @property
    def n_tiles(self):
        return self.frame.n_tiles

    @property
    def n_pixels(self):
        return self.frame.n_pixels

    def view_image(self, flat: torch.Tensor, v: int) -> torch.Tensor:
        W, H, off = self.views[v][:3]
        return flat[3 * off: 3 * (off + W * H)].view(3, H, W)

    def view_pixels(self, flat: torch.Tensor, v: int) -> torch.Tensor:
        W, H, off = self.views[v][:3]
        return flat[off: off + W * H].view(H, W)

    def pack_images(self, images) -> torch.Tensor:
        """Concatenate per-view [3,H,W] images into the planar batch layout."""
        return torch.cat([torch.as_tensor(im).reshape(-1) for im in images]).to(self.device)


def params_struct(params: dict, sh_degree: int) -> _abi.GsParams:
    m = _need(params["means"], torch.float32, "means")
    n = m.shape[0]
    _need(params["log_scales"], torch.float32, "log_scales")
    _need(params["quats"], torch.float32, "quats", 16)
    _need(params["opacity_logits"], torch.float32, "opacity_logits")
    sh = _need(params["sh"], torch.float32, "sh")
    s = _abi.GsParams()
    s.means, s.log_scales, s.quats = m.data_ptr(), params["log_scales"].data_ptr(), params["quats"].data_ptr()
    s.opacity_logits, s.sh = params["opacity_logits"].data_ptr(), sh.data_ptr()
    s.n, s.sh_degree, s.sh_stride = n, int(sh_degree), int(sh.shape[1])
    return s


def to_device_params(params: dict, device="cuda") -> dict:
    return {k: torch.as_tensor(np.ascontiguousarray(params[k]), dtype=torch.float32).to(device).contiguous()
            for k in PARAM_KEYS}


# ----------------------------------------------------------------------------------------
@dataclass
class Projected:
    mean2d: torch.Tensor          # [R,2]
    conic_opacity: torch.Tensor   # [R,4]
    rgb: torch.Tensor             # [R,4]
    depth: torch.Tensor           # [R]
    radius: torch.Tensor          # [R] int32
    rect: torch.Tensor            # [R,4] int16 (bits of uint16)
    clamped: torch.Tensor         # [R] uint8

    @staticmethod
    def empty(R, device):
        f = dict(dtype=torch.float32, device=device)
        return Projected(torch.empty(R, 2, **f), torch.empty(R, 4, **f), torch.empty(R, 4, **f),
                         torch.empty(R, **f), torch.empty(R, dtype=torch.int32, device=device),
                         torch.empty(R, 4, dtype=torch.int16, device=device),
                         torch.empty(R, dtype=torch.uint8, device=device))

    def struct(self) -> _abi.GsProj:
        s = _abi.GsProj()
        s.mean2d, s.conic_opacity, s.rgb = self.mean2d.data_ptr(), self.conic_opacity.data_ptr(), self.rgb.data_ptr()
        s.depth, s.radius, s.rect = self.depth.data_ptr(), self.radius.data_ptr(), self.rect.data_ptr()
        s.clamped, s.n_records = self.clamped.data_ptr(), self.mean2d.shape[0]
        return s

    def rect_np(self):
        return self.rect.cpu().numpy().view(np.uint16).astype(np.int64)


def project(params: dict, sh_degree: int, frame: Frame, out: Optional[Projected] = None,
            stream=None) -> Projected:
    ps = params_struct(params, sh_degree)
    R = frame.n_views * ps.n
    out = Projected.empty(R, frame.device) if out is None else out
    check(lib().gs_project(C.byref(ps), C.byref(frame.frame), C.byref(out.struct()), _stream(stream)),
          "gs_project")
    return out


# ----------------------------------------------------------------------------------------
@dataclass
class Bins:
    vals: torch.Tensor            # [capacity] int32 (bits of uint32 record ids)
    ranges: torch.Tensor          # [n_tiles, 2] int32
    count: torch.Tensor           # [1] int64: number of entries M
    keys: Optional[torch.Tensor]  # [capacity] int64 or None
    ws: torch.Tensor
    error: torch.Tensor           # [1] int32 device error word

    @property
    def capacity(self):
        return self.vals.shape[0]

    def struct(self) -> _abi.GsBins:
        s = _abi.GsBins()
        s.vals, s.ranges, s.d_count = self.vals.data_ptr(), self.ranges.data_ptr(), self.count.data_ptr()
        s.keys = None if self.keys is None else self.keys.data_ptr()
        s.capacity = self.vals.shape[0]
        return s


def alloc_bins(frame: Frame, n_records: int, capacity: int, want_keys=False) -> Bins:
    dev = frame.device
    ws_size = lib().gs_bin_sort_workspace_size(n_records, capacity, C.byref(frame.frame))
    if ws_size == 0:
        raise _abi.GsError(1, "gs_bin_sort_workspace_size (sizes or sort_fused_bits)")
    ws = _bytes(ws_size, dev)
    return Bins(torch.empty(max(capacity, 1), dtype=torch.int32, device=dev),
                torch.empty(frame.n_tiles, 2, dtype=torch.int32, device=dev),
                torch.zeros(1, dtype=torch.int64, device=dev),
                torch.empty(max(capacity, 1), dtype=torch.int64, device=dev) if want_keys else None,
                ws, torch.zeros(1, dtype=torch.int32, device=dev))


def bin_sort_into(proj: Projected, frame: Frame, bins: Bins, stream=None):
    """Enqueue gs_bin_sort into preallocated bins (no host synchronisation)."""
    check(lib().gs_bin_sort(C.byref(proj.struct()), C.byref(frame.frame), C.byref(bins.struct()),
                            _p(bins.ws), bins.ws.numel(), _p(bins.error), _stream(stream)), "gs_bin_sort")


def bin_sort(proj: Projected, frame: Frame, capacity: Optional[int] = None, want_keys=False,
             bins: Optional[Bins] = None) -> Bins:
    """Bin and sort; on duplicate-capacity overflow, grow to the reported count and redo."""
    R = proj.mean2d.shape[0]
    if bins is None:
        bins = alloc_bins(frame, R, capacity or max(1 << 16, 8 * R), want_keys)
    for _ in range(3):
        bins.error.zero_()
        bin_sort_into(proj, frame, bins)
        if int(bins.error.item()) == 0:
            return bins
        need = int(bins.count.item())
        bins = alloc_bins(frame, R, int(need * 1.1) + 1024, want_keys)
    raise _abi.GsError(2, "gs_bin_sort capacity")


# ----------------------------------------------------------------------------------------
def raster_cfg(bg=(0.0, 0.0, 0.0), store_stop=False, stage_depth=0, queue=None) -> _abi.GsRasterCfg:
    """queue: None (one CTA per tile) or a device int32 [1] tensor for the forward's
    persistent grid to claim its (tile, block) units from."""
    c = _abi.GsRasterCfg()
    for k in range(3):
        c.bg[k] = float(bg[k])
    c.store_stop = 1 if store_stop else 0
    c.stage_depth = int(stage_depth)
    c.d_queue = None if queue is None else _need(queue, torch.int32, "queue").data_ptr()
    return c


def raster_fwd(proj: Projected, bins: Bins, frame: Frame, bg=(0.0, 0.0, 0.0), store_stop=False,
               image=None, T_final=None, stop=None, stream=None, queue=None):
    dev = frame.device
    image = torch.empty(3 * frame.n_pixels, dtype=torch.float32, device=dev) if image is None else image
    T_final = torch.empty(frame.n_pixels, dtype=torch.float32, device=dev) if T_final is None else T_final
    if store_stop and stop is None:
        stop = torch.empty(frame.n_pixels, dtype=torch.int32, device=dev)
    cfg = raster_cfg(bg, store_stop, queue=queue)
    check(lib().gs_raster_fwd(C.byref(proj.struct()), C.byref(bins.struct()), C.byref(frame.frame),
                              C.byref(cfg), _p(image), _p(T_final), _p(stop) if store_stop else None,
                              _stream(stream)), "gs_raster_fwd")
    return image, T_final, (stop if store_stop else None)


def ckpt_bytes(frame: Frame, capacity: int, n_slots: int = -1) -> int:
    """Bytes of a checkpoint buffer with n_slots 1 KB slots (-1: one for every
    (bucket, 8x8 block) pair the lists can have, which cannot overflow)."""
    n = int(lib().gs_raster_ckpt_size(C.byref(frame.frame), int(capacity), int(n_slots)))
    if n == 0:
        raise _abi.GsError(1, f"gs_raster_ckpt_size (frame or capacity {capacity})")
    return n


def alloc_ckpt(frame: Frame, bins: "Bins", n_slots: int = -1) -> torch.Tensor:
    """Checkpoint buffer (uint8, 16-byte aligned) for raster_fwd_ckpt on these bins."""
    return torch.empty(ckpt_bytes(frame, bins.capacity, n_slots), dtype=torch.uint8, device=frame.device)


def ckpt_usage(frame: Frame, bins: "Bins", ckpt: torch.Tensor, out=None, stream=None) -> torch.Tensor:
    """int64 [2] on the device: (slots the last raster_fwd_ckpt into ckpt needed,
    1 if it ran out of slots)."""
    out = torch.empty(2, dtype=torch.int64, device=frame.device) if out is None else out
    check(lib().gs_raster_ckpt_usage(C.byref(frame.frame), int(bins.capacity), _p(ckpt),
                                     ckpt.numel() * ckpt.element_size(), _p(out), _stream(stream)),
          "gs_raster_ckpt_usage")
    return out


def raster_fwd_ckpt(proj: Projected, bins: Bins, frame: Frame, ckpt: torch.Tensor, bg=(0.0, 0.0, 0.0),
                    image=None, T_final=None, stop=None, stream=None, queue=None):
    """raster_fwd with stop indices and the per-splat backward's checkpoints."""
    dev = frame.device
    image = torch.empty(3 * frame.n_pixels, dtype=torch.float32, device=dev) if image is None else image
    T_final = torch.empty(frame.n_pixels, dtype=torch.float32, device=dev) if T_final is None else T_final
    stop = torch.empty(frame.n_pixels, dtype=torch.int32, device=dev) if stop is None else stop
    cfg = raster_cfg(bg, True, queue=queue)
    check(lib().gs_raster_fwd_ckpt(C.byref(proj.struct()), C.byref(bins.struct()), C.byref(frame.frame),
                                   C.byref(cfg), _p(image), _p(T_final), _p(stop), _p(ckpt),
                                   ckpt.numel() * ckpt.element_size(), _stream(stream)), "gs_raster_fwd_ckpt")
    return image, T_final, stop


def raster_count(proj: Projected, bins: Bins, frame: Frame, counts=None, stream=None):
    """Per-pixel (entries examined, entries composited) of Eq. 2 -> int32 [n_pixels, 2]."""
    counts = torch.empty(frame.n_pixels, 2, dtype=torch.int32, device=frame.device) if counts is None else counts
    check(lib().gs_raster_count(C.byref(proj.struct()), C.byref(bins.struct()), C.byref(frame.frame), _p(counts),
                                _stream(stream)), "gs_raster_count")
    return counts


def l1_loss_grad(frame: Frame, image: torch.Tensor, target: torch.Tensor, d_image=None, loss=None,
                 stream=None):
    d_image = torch.empty_like(image) if d_image is None else d_image
    loss = torch.empty(frame.n_views, dtype=torch.float32, device=frame.device) if loss is None else loss
    check(lib().gs_l1_loss_grad(C.byref(frame.frame), _p(image), _p(_need(target, torch.float32, "target")),
                                _p(d_image), _p(loss), _stream(stream)), "gs_l1_loss_grad")
    return d_image, loss


@dataclass
class RecGrads:
    d_mean2d: torch.Tensor
    d_conic_opacity: torch.Tensor
    d_rgb: torch.Tensor

    @staticmethod
    def zeros(R, device):
        f = dict(dtype=torch.float32, device=device)
        return RecGrads(torch.empty(R, 2, **f), torch.empty(R, 4, **f), torch.empty(R, 4, **f))

    def zero_(self):
        self.d_mean2d.zero_(); self.d_conic_opacity.zero_(); self.d_rgb.zero_()
        return self

    def struct(self):
        s = _abi.GsRecGrads()
        s.d_mean2d, s.d_conic_opacity, s.d_rgb = (self.d_mean2d.data_ptr(), self.d_conic_opacity.data_ptr(),
                                                  self.d_rgb.data_ptr())
        return s


def raster_bwd(proj: Projected, bins: Bins, frame: Frame, image, d_image, bg=(0.0, 0.0, 0.0),
               grads: Optional[RecGrads] = None, stop=None, stage_depth=0, stream=None) -> RecGrads:
    """stop: the forward's per-pixel stop indices (raster_fwd(store_stop=True)), or
    None to recompute them from the transmittance cut-off. stage_depth: 0 stages one
    list entry per thread per CTA step, 1 half as many (a tuning knob)."""
    grads = RecGrads.zeros(proj.mean2d.shape[0], frame.device) if grads is None else grads
    cfg = raster_cfg(bg, stage_depth=stage_depth)
    check(lib().gs_raster_bwd(C.byref(proj.struct()), C.byref(bins.struct()), C.byref(frame.frame), C.byref(cfg),
                              _p(image), _p(_need(d_image, torch.float32, "d_image")),
                              _p(stop) if stop is not None else None, C.byref(grads.struct()),
                              _stream(stream)), "gs_raster_bwd")
    return grads


def empty_param_grads(params: dict) -> dict:
    return {k: torch.empty_like(params[k]) for k in PARAM_KEYS}


def project_bwd(params: dict, sh_degree: int, frame: Frame, proj: Projected, rec: RecGrads, out=None,
                accum=None, count=None, stream=None) -> dict:
    ps = params_struct(params, sh_degree)
    out = empty_param_grads(params) if out is None else out
    g = _abi.GsParamGrads()
    g.d_means, g.d_log_scales, g.d_quats = out["means"].data_ptr(), out["log_scales"].data_ptr(), out["quats"].data_ptr()
    g.d_opacity_logits, g.d_sh = out["opacity_logits"].data_ptr(), out["sh"].data_ptr()
    check(lib().gs_project_bwd(C.byref(ps), C.byref(frame.frame), C.byref(proj.struct()), C.byref(rec.struct()),
                               C.byref(g), _p(accum), _p(count), _stream(stream)), "gs_project_bwd")
    return out


# ----------------------------------------------------------------------------------------
def densify_accum(d_mean2d, radius, frame: Frame, n, accum, count, stream=None):
    check(lib().gs_densify_accum(_p(d_mean2d), _p(radius), C.byref(frame.frame), int(n), _p(accum), _p(count),
                                 _stream(stream)), "gs_densify_accum")


def densify_cfg(mode=DENSIFY_ADAPTIVE, grad_threshold=2e-4, log_scale_threshold=0.0, prune_logit=None,
                prune_ratio=None, prune_upper_logit=None, seed=0, event=0) -> _abi.GsDensifyCfg:
    c = _abi.GsDensifyCfg()
    c.mode = int(mode)
    c.grad_threshold = float(np.float32(grad_threshold))
    c.log_scale_threshold = float(np.float32(log_scale_threshold))
    c.prune_adaptive = 1 if prune_ratio is not None else 0
    c.prune_logit = float(np.float32(prune_logit if prune_logit is not None else -np.inf))
    c.prune_upper_logit = float(np.float32(prune_upper_logit if prune_upper_logit is not None else np.inf))
    c.prune_ratio = float(prune_ratio) if prune_ratio is not None else 0.0
    c.seed, c.event = int(seed), int(event)
    return c


def densify_select(cfg: _abi.GsDensifyCfg, params: dict, accum, count, ws=None, stream=None, out=None):
    """out: optional preallocated (split, clone, tau, new_n)."""
    n = params["means"].shape[0]
    dev = params["means"].device
    ws = _bytes(lib().gs_densify_workspace_size(n), dev) if ws is None else ws
    if out is None:
        split = torch.empty(n, dtype=torch.uint8, device=dev)
        clone = torch.empty(n, dtype=torch.uint8, device=dev)
        tau = torch.empty(1, dtype=torch.float32, device=dev)
        new_n = torch.empty(1, dtype=torch.int64, device=dev)
    else:
        split, clone, tau, new_n = out
    check(lib().gs_densify_select(C.byref(cfg), _p(params["log_scales"]), _p(params["opacity_logits"]),
                                  _p(accum), _p(count), n, _p(split), _p(clone), _p(tau), _p(new_n), _p(ws),
                                  ws.numel(), _stream(stream)), "gs_densify_select")
    return split, clone, tau, new_n, ws


PROV_KEYS = ("origin", "splits", "clones")


def densify_apply(cfg: _abi.GsDensifyCfg, params: dict, sh_degree: int, split, clone, tau, capacity: int,
                  extra: Optional[dict] = None, ws=None, stream=None, out=None, ex_out=None, new_n=None,
                  err=None, prov: Optional[dict] = None):
    """out / ex_out / new_n / err: optional preallocated outputs (capacity rows).
    prov: optional provenance {origin, splits, clones} (int32 [n]); their outputs
    (int32 [capacity]) are returned in out under the same keys."""
    ps = params_struct(params, sh_degree)
    dev = params["means"].device
    ws = _bytes(lib().gs_densify_workspace_size(ps.n), dev) if ws is None else ws
    if out is None:
        out = {k: torch.empty((capacity,) + tuple(params[k].shape[1:]), dtype=torch.float32, device=dev)
               for k in PARAM_KEYS}
    po = _abi.GsParamsOut()
    po.means, po.log_scales, po.quats = out["means"].data_ptr(), out["log_scales"].data_ptr(), out["quats"].data_ptr()
    po.opacity_logits, po.sh = out["opacity_logits"].data_ptr(), out["sh"].data_ptr()
    extra = extra or {}
    given = ex_out is not None
    ex_out = dict(ex_out) if given else {}
    arr = (_abi.GsExtraArray * max(1, len(extra)))()
    for i, (k, src) in enumerate(extra.items()):
        src = _need(src, torch.float32, k)
        dst = ex_out[k] if given else torch.empty((capacity,) + tuple(src.shape[1:]), dtype=torch.float32, device=dev)
        ex_out[k] = dst
        arr[i].src, arr[i].dst, arr[i].width = src.data_ptr(), dst.data_ptr(), int(src[0].numel()) if src.shape[0] else 1
    new_n = torch.empty(1, dtype=torch.int64, device=dev) if new_n is None else new_n
    err = torch.zeros(1, dtype=torch.int32, device=dev) if err is None else err
    pv = None
    if prov is not None:
        pv = _abi.GsProvenance()
        for k in PROV_KEYS:
            src = _need(prov[k], torch.int32, k)
            dst = out.get(k)
            if dst is None:
                dst = torch.empty(capacity, dtype=torch.int32, device=dev)
                out[k] = dst
            setattr(pv, f"{k}_in", src.data_ptr())
            setattr(pv, f"{k}_out", dst.data_ptr())
    check(lib().gs_densify_apply(C.byref(cfg), C.byref(ps), _p(split), _p(clone), _p(tau), C.byref(po), arr,
                                 len(extra), C.byref(pv) if pv is not None else None, int(capacity), _p(new_n),
                                 _p(err), _p(ws), ws.numel(), _stream(stream)), "gs_densify_apply")
    return out, ex_out, new_n, err


def raster_bwd_splat(proj: Projected, bins: Bins, frame: Frame, image, d_image, stop, ckpt,
                     grads: Optional[RecGrads] = None, stream=None) -> RecGrads:
    """Per-splat backward from raster_fwd_ckpt's image, stop indices and checkpoints."""
    grads = RecGrads.zeros(proj.mean2d.shape[0], frame.device) if grads is None else grads
    check(lib().gs_raster_bwd_splat(C.byref(proj.struct()), C.byref(bins.struct()), C.byref(frame.frame),
                                    _p(image), _p(_need(d_image, torch.float32, "d_image")), _p(stop), _p(ckpt),
                                    ckpt.numel() * ckpt.element_size(), C.byref(grads.struct()),
                                    _stream(stream)), "gs_raster_bwd_splat")
    return grads
