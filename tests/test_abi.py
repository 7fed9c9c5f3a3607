"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry
point include/gs.h declares; the ctypes mirror has the C layout; host-only entry
points and host-side argument checks work on the CPU (no device call is made)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

from paper_2507_20239_gb300 import build as gbuild
from paper_2507_20239_gb300 import _abi

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gs.h")


@pytest.fixture(scope="module")
def lib():
    gbuild.build()
    return _abi.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_expected_entry_points():
    names = declared_functions()
    for want in ("gs_project", "gs_bin_sort", "gs_raster_fwd", "gs_raster_bwd", "gs_project_bwd",
                 "gs_densify_accum", "gs_densify_select", "gs_densify_apply", "gs_l1_loss_grad"):
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared_functions()) <= set(_abi.SIGNATURES)


STRUCTS = {
    "gs_camera_t": (_abi.GsCamera, ["R", "t", "fx", "width", "near_plane", "grid_x", "tile_offset", "pixel_offset"]),
    "gs_frame_t": (_abi.GsFrame, ["cams_dev", "n_views", "n_tiles", "n_pixels", "max_height"]),
    "gs_params_t": (_abi.GsParams, ["means", "sh", "n", "sh_degree", "sh_stride"]),
    "gs_proj_t": (_abi.GsProj, ["mean2d", "clamped", "n_records"]),
    "gs_bins_t": (_abi.GsBins, ["vals", "keys", "ranges", "d_count", "capacity"]),
    "gs_raster_cfg_t": (_abi.GsRasterCfg, ["bg", "store_stop", "stage_depth", "d_queue"]),
    "gs_rec_grads_t": (_abi.GsRecGrads, ["d_mean2d", "d_rgb"]),
    "gs_param_grads_t": (_abi.GsParamGrads, ["d_means", "d_sh"]),
    "gs_densify_cfg_t": (_abi.GsDensifyCfg, ["mode", "prune_upper_logit", "prune_ratio", "seed", "event"]),
    "gs_extra_array_t": (_abi.GsExtraArray, ["src", "dst", "width"]),
    "gs_params_out_t": (_abi.GsParamsOut, ["means", "sh"]),
    "gs_provenance_t": (_abi.GsProvenance, ["origin_in", "clones_in", "origin_out", "clones_out"]),
}


def test_ctypes_layout_matches_c_compiler():
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "gs.h"', "int main(void) {"]
    for name, (_, fields) in STRUCTS.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for f in fields:
            lines.append(f'printf("{name} {f} %zu\\n", offsetof({name}, {f}));')
    lines.append("return 0; }")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(src, "w").write("\n".join(lines))
        subprocess.run(["gcc", "-I", os.path.dirname(HEADER), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    for line in out.splitlines():
        parts = line.split()
        cls = STRUCTS[parts[0]][0]
        if parts[1] == "size":
            assert C.sizeof(cls) == int(parts[2]), line
        else:
            assert getattr(cls, parts[1]).offset == int(parts[2]), line


def test_host_only_entry_points(lib):
    assert lib.gs_status_str(0) == b"ok"
    assert b"sm_103a" in lib.gs_version()
    assert lib.gs_tile_supported(16, 16) and lib.gs_tile_supported(8, 8) and lib.gs_tile_supported(16, 32)
    assert not lib.gs_tile_supported(12, 12)
    cams = (_abi.GsCamera * 3)()
    for i, (w, h) in enumerate([(312, 207), (623, 413), (1246, 826)]):
        cams[i].width, cams[i].height = w, h
        cams[i].fx = cams[i].fy = 100.0
        cams[i].near_plane = 0.2
    fr = _abi.GsFrame()
    assert lib.gs_frame_init(cams, 3, 16, 16, C.byref(fr)) == 0
    assert [cams[i].grid_x for i in range(3)] == [20, 39, 78]
    assert [cams[i].grid_y for i in range(3)] == [13, 26, 52]
    assert [cams[i].tile_offset for i in range(3)] == [0, 260, 260 + 1014]
    assert fr.n_tiles == 260 + 1014 + 4056
    assert fr.n_pixels == 312 * 207 + 623 * 413 + 1246 * 826
    assert [cams[i].pixel_offset for i in range(3)] == [0, 312 * 207, 312 * 207 + 623 * 413]
    assert lib.gs_frame_init(cams, 3, 12, 12, C.byref(fr)) == 1
    assert lib.gs_bin_sort_workspace_size(1000, 5000, C.byref(fr)) > 4 * 5000 * 3
    assert lib.gs_densify_workspace_size(1000) > 0


def test_host_argument_checks_return_invalid_arg(lib):
    fr = _abi.GsFrame()
    assert lib.gs_project(None, C.byref(fr), None, None) == 1
    assert lib.gs_bin_sort(None, None, None, None, 0, None, None) == 1
    assert lib.gs_raster_fwd(None, None, None, None, None, None, None, None) == 1
    assert lib.gs_raster_bwd(None, None, None, None, None, None, None, None, None) == 1
    assert lib.gs_project_bwd(None, None, None, None, None, None, None, None) == 1
    assert lib.gs_densify_accum(None, None, None, 0, None, None, None) == 1
    assert lib.gs_l1_loss_grad(None, None, None, None, None, None) == 1
    p = _abi.GsParams()
    p.n, p.sh_degree, p.sh_stride = 10, 4, 25       # degree 4 is not supported
    assert lib.gs_project(C.byref(p), C.byref(fr), None, None) == 1


def _a256(x):
    return (x + 255) // 256 * 256


def test_checkpoint_size_and_bucket_layout(lib):
    """gs_raster_ckpt_size's formula (256 pool counters, a 4-byte table entry per
    (bucket, 8x8 block), 1 KB per slot; n_slots < 0: a slot per table entry), and the
    bucket numbering it relies on: tile t's 32-entry buckets b are floor(s_t / 32) +
    t + b for a list starting at s_t, which never overlap between tiles and stay below
    ceil(M / 32) + n_tiles."""
    import numpy as np
    cams = (_abi.GsCamera * 2)()
    for i, (w, h) in enumerate([(623, 413), (1246, 826)]):
        cams[i].width, cams[i].height = w, h
        cams[i].fx = cams[i].fy = 100.0
        cams[i].near_plane = 0.2
    for tw, th in ((16, 16), (8, 8), (16, 32)):
        fr = _abi.GsFrame()
        assert lib.gs_frame_init(cams, 2, tw, th, C.byref(fr)) == 0
        for cap in (0, 1, 31, 32, 33, 1_000_003):
            entries = ((cap + 31) // 32 + fr.n_tiles) * (tw * th // 64)
            head = 1024 + _a256(4 * entries)
            assert lib.gs_raster_ckpt_size(C.byref(fr), cap, 0) == head
            assert lib.gs_raster_ckpt_size(C.byref(fr), cap, 1000) == head + 1000 * 1024
            assert lib.gs_raster_ckpt_size(C.byref(fr), cap, -1) == head + entries * 1024
        assert lib.gs_raster_ckpt_size(C.byref(fr), -1, 0) == 0
    assert lib.gs_raster_ckpt_size(None, 10, 0) == 0
    assert lib.gs_raster_ckpt_usage(None, 0, None, 0, None, None) == 1
    assert lib.gs_raster_fwd_ckpt(None, None, None, None, None, None, None, None, 0, None) == 1
    assert lib.gs_raster_bwd_splat(None, None, None, None, None, None, None, 0, None, None) == 1
    rng = np.random.default_rng(0)
    for trial in range(200):
        n_tiles = int(rng.integers(1, 60))
        lens = rng.choice([0, 1, 31, 32, 33, 64, 100], n_tiles) * (rng.random(n_tiles) < 0.8)
        starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
        M = int(lens.sum())
        used = set()
        for t in range(n_tiles):
            for b in range((int(lens[t]) + 31) // 32):
                k = int(starts[t]) // 32 + t + b
                assert k not in used and k < (M + 31) // 32 + n_tiles, (trial, t, b)
                used.add(k)


def test_debug_status_entry_point(lib):
    # the release library has no bounds checks compiled in and says so; the debug
    # library (-DGS_DEBUG) builds and exports the same entry points
    import ctypes as C
    w = C.c_uint64(5)
    assert lib.gs_debug_status(C.byref(w)) == 5 and w.value == 0      # GS_ERR_UNSUPPORTED
    assert lib.gs_debug_status(None) == 1
    dbg = _abi.load(gbuild.build(debug=True))
    missing = [n for n in declared_functions() if not hasattr(dbg, n)]
    assert not missing, missing
