"""ctypes declarations mirroring include/gs.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

c_float_p = C.POINTER(C.c_float)
vp = C.c_void_p


class GsCamera(C.Structure):
    _fields_ = [("R", C.c_float * 9), ("t", C.c_float * 3), ("fx", C.c_float), ("fy", C.c_float),
                ("cx", C.c_float), ("cy", C.c_float), ("width", C.c_int32), ("height", C.c_int32),
                ("near_plane", C.c_float), ("grid_x", C.c_int32), ("grid_y", C.c_int32),
                ("tile_offset", C.c_int32), ("pixel_offset", C.c_int64)]


class GsFrame(C.Structure):
    _fields_ = [("cams_dev", vp), ("n_views", C.c_int32), ("tile_w", C.c_int32), ("tile_h", C.c_int32),
                ("n_tiles", C.c_int32), ("n_pixels", C.c_int64), ("max_width", C.c_int32),
                ("max_height", C.c_int32), ("sort_fused_bits", C.c_int32)]


class GsParams(C.Structure):
    _fields_ = [("means", vp), ("log_scales", vp), ("quats", vp), ("opacity_logits", vp), ("sh", vp),
                ("n", C.c_int64), ("sh_degree", C.c_int32), ("sh_stride", C.c_int32)]


class GsProj(C.Structure):
    _fields_ = [("mean2d", vp), ("conic_opacity", vp), ("rgb", vp), ("depth", vp), ("radius", vp),
                ("rect", vp), ("clamped", vp), ("n_records", C.c_int64)]


class GsBins(C.Structure):
    _fields_ = [("vals", vp), ("keys", vp), ("ranges", vp), ("d_count", vp), ("capacity", C.c_int64)]


class GsRasterCfg(C.Structure):
    _fields_ = [("bg", C.c_float * 3), ("store_stop", C.c_int32), ("stage_depth", C.c_int32),
                ("d_queue", vp)]


class GsRecGrads(C.Structure):
    _fields_ = [("d_mean2d", vp), ("d_conic_opacity", vp), ("d_rgb", vp)]


class GsParamGrads(C.Structure):
    _fields_ = [("d_means", vp), ("d_log_scales", vp), ("d_quats", vp), ("d_opacity_logits", vp),
                ("d_sh", vp)]


class GsDensifyCfg(C.Structure):
    _fields_ = [("mode", C.c_int32), ("grad_threshold", C.c_float), ("log_scale_threshold", C.c_float),
                ("prune_adaptive", C.c_int32), ("prune_logit", C.c_float),
                ("prune_upper_logit", C.c_float), ("prune_ratio", C.c_double), ("seed", C.c_uint64),
                ("event", C.c_uint32)]


class GsExtraArray(C.Structure):
    _fields_ = [("src", vp), ("dst", vp), ("width", C.c_int32)]


class GsProvenance(C.Structure):
    _fields_ = [("origin_in", vp), ("splits_in", vp), ("clones_in", vp), ("origin_out", vp), ("splits_out", vp),
                ("clones_out", vp)]


class GsParamsOut(C.Structure):
    _fields_ = [("means", vp), ("log_scales", vp), ("quats", vp), ("opacity_logits", vp), ("sh", vp)]


class GsAdamState(C.Structure):
    _fields_ = [("m", vp * 5), ("v", vp * 5)]


class GsAdamCfg(C.Structure):
    _fields_ = [("lr", C.c_float * 5), ("eps", C.c_float), ("beta1", C.c_double), ("beta2", C.c_double),
                ("step", C.c_int32)]


P = C.POINTER
SIGNATURES = {
    "gs_status_str": (C.c_char_p, [C.c_int]),
    "gs_version": (C.c_char_p, []),
    "gs_launch_count": (C.c_uint64, []),
    "gs_tile_supported": (C.c_int32, [C.c_int32, C.c_int32]),
    "gs_frame_init": (C.c_int, [P(GsCamera), C.c_int32, C.c_int32, C.c_int32, P(GsFrame)]),
    "gs_bin_sort_workspace_size": (C.c_size_t, [C.c_int64, C.c_int64, P(GsFrame)]),
    "gs_project": (C.c_int, [P(GsParams), P(GsFrame), P(GsProj), vp]),
    "gs_bin_sort": (C.c_int, [P(GsProj), P(GsFrame), P(GsBins), vp, C.c_size_t, vp, vp]),
    "gs_raster_fwd": (C.c_int, [P(GsProj), P(GsBins), P(GsFrame), P(GsRasterCfg), vp, vp, vp, vp]),
    "gs_raster_count": (C.c_int, [P(GsProj), P(GsBins), P(GsFrame), vp, vp]),
    "gs_l1_loss_grad": (C.c_int, [P(GsFrame), vp, vp, vp, vp, vp]),
    "gs_raster_bwd": (C.c_int, [P(GsProj), P(GsBins), P(GsFrame), P(GsRasterCfg), vp, vp, vp, P(GsRecGrads), vp]),
    "gs_raster_ckpt_size": (C.c_size_t, [P(GsFrame), C.c_int64, C.c_int64]),
    "gs_raster_ckpt_usage": (C.c_int, [P(GsFrame), C.c_int64, vp, C.c_size_t, vp, vp]),
    "gs_raster_fwd_ckpt": (C.c_int, [P(GsProj), P(GsBins), P(GsFrame), P(GsRasterCfg), vp, vp, vp, vp, C.c_size_t,
                                     vp]),
    "gs_raster_bwd_splat": (C.c_int, [P(GsProj), P(GsBins), P(GsFrame), vp, vp, vp, vp, C.c_size_t,
                                      P(GsRecGrads), vp]),
    "gs_project_bwd": (C.c_int, [P(GsParams), P(GsFrame), P(GsProj), P(GsRecGrads), P(GsParamGrads), vp,
                                 vp, vp]),
    "gs_densify_accum": (C.c_int, [vp, vp, P(GsFrame), C.c_int64, vp, vp, vp]),
    "gs_densify_workspace_size": (C.c_size_t, [C.c_int64]),
    "gs_densify_select": (C.c_int, [P(GsDensifyCfg), vp, vp, vp, vp, C.c_int64, vp, vp, vp, vp, vp,
                                    C.c_size_t, vp]),
    "gs_densify_select_static": (C.c_int, [P(GsDensifyCfg), vp, vp, vp, vp, C.c_int64, vp, vp, vp, vp, vp]),
    "gs_densify_apply": (C.c_int, [P(GsDensifyCfg), P(GsParams), vp, vp, vp, P(GsParamsOut),
                                   P(GsExtraArray), C.c_int32, P(GsProvenance), C.c_int64, vp, vp, vp,
                                   C.c_size_t, vp]),
    "gs_photometric_workspace_size": (C.c_size_t, [P(GsFrame)]),
    "gs_photometric_loss_grad": (C.c_int, [P(GsFrame), vp, vp, C.c_float, vp, vp, vp, C.c_size_t, vp]),
    "gs_adam_step": (C.c_int, [P(GsAdamCfg), P(GsParamsOut), C.c_int64, C.c_int32, P(GsParamGrads),
                               P(GsAdamState), vp, C.c_int32, vp]),
    "gs_opacity_reset": (C.c_int, [vp, vp, vp, C.c_int64, C.c_float, vp]),
    "gs_downscaled_size": (C.c_int32, [C.c_int32, C.c_int32]),
    "gs_downscale": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32, C.c_int32, vp, vp]),
    "gs_spectrum_workspace_size": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32]),
    "gs_spectrum_l1": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int32, vp, vp, C.c_size_t, vp]),
    "gs_debug_status": (C.c_int, [P(C.c_uint64)]),
}

_lib = None


def load(path: str | None = None):
    """Load libgs.so (built in-tree) and declare every entry point; raise if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB
    if not os.path.exists(p):
        raise RuntimeError(f"libgs is not built ({p} missing): run paper_2507_20239_gb300.build.build()")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


STATUS = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CAPACITY", 3: "GS_ERR_CUDA",
          4: "GS_ERR_TIMEOUT", 5: "GS_ERR_UNSUPPORTED"}


class GsError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"{where}: {STATUS.get(code, code)}")
        self.code = code


def check(code, where):
    if code != 0:
        raise GsError(code, where)
