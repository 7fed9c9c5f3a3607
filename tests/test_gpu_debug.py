"""The debug library (libgs_debug.so, the hot path with its bounds checks compiled
in): the same results as the release library with a clean status, and a record id
beyond the records, planted in a tile's list, reported by the forward's own check
(code 1 and the id) instead of being dereferenced."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2507_20239_gb300 import _abi, build as gbuild
from paper_2507_20239_gb300 import rasterizer as R
from tests.gs_fixtures import dev_params, rel_l2, scene

pytestmark = pytest.mark.gpu


@pytest.fixture
def debug_lib():
    path = gbuild.build(debug=True)
    lib = _abi.load(path)
    saved = _abi._lib
    _abi._lib = lib
    try:
        yield lib
    finally:
        _abi._lib = saved


def _status(lib):
    w = C.c_uint64(0)
    assert lib.gs_debug_status(C.byref(w)) == 0
    return w.value


def _run_all(sc, frame):
    P = dev_params(sc)
    proj = R.project(P, sc.sh_degree, frame)
    bins = R.bin_sort(proj, frame)
    img, T, stop = R.raster_fwd(proj, bins, frame, store_stop=True)
    counts = R.raster_count(proj, bins, frame)
    ck = R.alloc_ckpt(frame, bins)
    R.raster_fwd_ckpt(proj, bins, frame, ck)
    dg = torch.as_tensor(np.random.default_rng(1).normal(0, 1, img.numel()).astype(np.float32)).cuda()
    gs_ = R.raster_bwd_splat(proj, bins, frame, img, dg, stop, ck)
    gp = R.raster_bwd(proj, bins, frame, img, dg, stop=stop)
    torch.cuda.synchronize()
    return img, stop, counts, gs_, gp


def test_debug_build_matches_release(debug_lib):
    sc = scene("orbit_small")
    frame = R.Frame(sc.cameras)
    _status(debug_lib)                                    # clear
    dbg = _run_all(sc, frame)
    assert _status(debug_lib) == 0
    _abi._lib = _abi.load()
    rel = _run_all(sc, frame)
    _abi._lib = debug_lib
    for a, b in zip(dbg[:3], rel[:3]):
        assert torch.equal(a, b)                          # the checks change no arithmetic
    for a, b in zip(dbg[3:], rel[3:]):           # atomically summed: equal up to summation order
        for x, y in ((a.d_mean2d, b.d_mean2d), (a.d_conic_opacity, b.d_conic_opacity), (a.d_rgb, b.d_rgb)):
            assert rel_l2(x.cpu().numpy(), y.cpu().numpy()) < 1e-5


def test_debug_build_reports_a_bad_record_id(debug_lib):
    sc = scene("small")
    frame = R.Frame(sc.cameras)
    P = dev_params(sc)
    proj = R.project(P, sc.sh_degree, frame)
    bins = R.bin_sort(proj, frame)
    torch.cuda.synchronize()
    ranges = bins.ranges.cpu().numpy().view(np.uint32)
    t = int(np.argmax(ranges[:, 1] - ranges[:, 0]))
    assert ranges[t, 1] > ranges[t, 0]
    bad = proj.mean2d.shape[0] + 7
    bins.vals[int(ranges[t, 0])] = bad                    # first entry of the longest list
    _status(debug_lib)
    R.raster_fwd(proj, bins, frame, store_stop=True)      # every gather by a record id is checked
    assert _status(debug_lib) == (1 << 48) | bad
    assert _status(debug_lib) == 0                        # read and cleared
