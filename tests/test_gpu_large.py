"""The large-scene workload (5M Gaussians, SH degree 3, 4 views at 1600x1060,
stop indices recomputed by the backward) on sampled outputs: the batched
projection against the FP64 oracle on 20,000 sampled Gaussians per view, and
view 0's compositing and gradient on sampled tiles."""
import numpy as np
import pytest
import torch

from paper_2507_20239_gb300 import rasterizer as R
from paper_2507_20239_gb300 import synth
from tests.gs_fixtures import bins_pairs, exact_list_check, oracle_records_fp32, rel_l2
from tests.test_gpu_project import _compare_projection
from tests.test_gpu_raster import GRAD_TOL, _compare_fwd, _gpu, _oracle_fwd, _tile_mask

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def large():
    return synth.large_scene(4)


def test_large_projection_sampled(large):
    rng = np.random.default_rng(40)
    sample = np.sort(rng.choice(large.n, 20000, replace=False))
    _compare_projection(large, large.cameras, sample=sample)


def test_large_lists_hold_every_exact_fp64_pair(large):
    """The four-view frame of the large scene binned in one launch (the benchmark's
    configuration), views 0 and 3 against the exact FP64 footprint geometry of the
    GPU's own records (see tests/gs_fixtures.exact_list_check)."""
    frame = R.Frame(large.cameras)
    P = R.to_device_params(large.params(), "cuda")
    proj = R.project(P, large.sh_degree, frame)
    bins = R.bin_sort(proj, frame)
    torch.cuda.synchronize()
    tiles, recs = bins_pairs(bins, frame.n_tiles)
    del bins
    n = large.n
    for v in (0, 3):
        W, H, _, toff, gx = frame.views[v][:5]
        nt = gx * ((H + 15) // 16)
        sel = (tiles >= toff) & (tiles < toff + nt)
        sl = slice(v * n, (v + 1) * n)
        co = proj.conic_opacity[sl].cpu().numpy()
        listed, must, between = exact_list_check(
            proj.mean2d[sl].cpu().numpy(), co[:, :3], proj.rgb[sl, 3].cpu().numpy(), proj.radius[sl].cpu().numpy(),
            W, H, (16, 16), tiles[sel] - toff, recs[sel] - v * n)
        print(f"view {v}: listed {listed}, exact-with-margin {must}, within the margin {between}")
        assert listed > 1_000_000 and between < 1e-3 * listed


def test_large_view_raster_recomputed_stop_sampled_tiles(large):
    cam = large.cameras[0]
    tile = (16, 16)
    rec = oracle_records_fp32(large.params(), large.sh_degree, cam, tile)
    frame, proj, bins, img, T, stop = _gpu([rec], [cam], tile, (0, 0, 0))
    ranges = bins.ranges.cpu().numpy()
    lens = ranges[:, 1] - ranges[:, 0]
    rng = np.random.default_rng(41)
    busy = np.nonzero(lens > 0)[0]
    tiles = sorted(set(rng.choice(busy, 16, replace=False).tolist()) | set(np.argsort(lens)[-2:].tolist()))
    mask = _tile_mask(cam, tile, tiles)
    d_image = np.where(mask[None], rng.normal(0, 1, (3, cam.height, cam.width)), 0).astype(np.float32)
    o, g = _oracle_fwd(rec, cam, tile, (0, 0, 0), tiles=tiles, d_image=d_image)
    counts = R.raster_count(proj, bins, frame).cpu().numpy().reshape(cam.height, cam.width, 2)
    _compare_fwd(o, frame.view_image(img, 0).cpu().numpy(), frame.view_pixels(T, 0).cpu().numpy(),
                 frame.view_pixels(stop, 0).cpu().numpy(), mask=mask, counts=counts, max_flag_frac=5e-3)
    rg = R.raster_bwd(proj, bins, frame, img, torch.as_tensor(d_image.reshape(-1)).cuda(), stop=None)
    torch.cuda.synchronize()
    got = dict(d_mean2d=rg.d_mean2d.cpu().numpy(), d_conic=rg.d_conic_opacity[:, :3].cpu().numpy(),
               d_opacity=rg.d_conic_opacity[:, 3].cpu().numpy(), d_rgb=rg.d_rgb[:, :3].cpu().numpy())
    for k in got:
        e = rel_l2(got[k], g[k])
        assert e < GRAD_TOL, (k, e)


def test_large_views_per_splat_backward(large):
    """The per-splat backward at the large scene's size: view 0 on sampled tiles
    against the FP64 oracle, and the four views in one training step (the
    benchmark's launch configuration) against the per-pixel step: identical images,
    gradients within summation order."""
    from paper_2507_20239_gb300.step import StepConfig, TrainStep, duplicates
    from tests.gs_fixtures import records_to_gpu
    cam = large.cameras[0]
    tile = (16, 16)
    rec = oracle_records_fp32(large.params(), large.sh_degree, cam, tile)
    frame = R.Frame([cam], tile=tile)
    proj = records_to_gpu([rec])
    bins = R.bin_sort(proj, frame)
    ckpt = R.alloc_ckpt(frame, bins)
    img, T, stop = R.raster_fwd_ckpt(proj, bins, frame, ckpt)
    ranges = bins.ranges.cpu().numpy()
    lens = ranges[:, 1] - ranges[:, 0]
    rng = np.random.default_rng(42)
    busy = np.nonzero(lens > 0)[0]
    tiles = sorted(set(rng.choice(busy, 16, replace=False).tolist()) | set(np.argsort(lens)[-2:].tolist()))
    mask = _tile_mask(cam, tile, tiles)
    d_image = np.where(mask[None], rng.normal(0, 1, (3, cam.height, cam.width)), 0).astype(np.float32)
    _, g = _oracle_fwd(rec, cam, tile, (0, 0, 0), tiles=tiles, d_image=d_image)
    rs = R.raster_bwd_splat(proj, bins, frame, img, torch.as_tensor(d_image.reshape(-1)).cuda(), stop, ckpt)
    torch.cuda.synchronize()
    got = dict(d_mean2d=rs.d_mean2d.cpu().numpy(), d_conic=rs.d_conic_opacity[:, :3].cpu().numpy(),
               d_opacity=rs.d_conic_opacity[:, 3].cpu().numpy(), d_rgb=rs.d_rgb[:, :3].cpu().numpy())
    for k in got:
        e = rel_l2(got[k], g[k])
        assert e < GRAD_TOL, (k, e)
    del proj, bins, ckpt, img, T, stop, rs

    P = R.to_device_params(large.params(), "cuda")
    M = duplicates(P, large.sh_degree, R.Frame(large.cameras))
    out = {}
    for bw in ("pixel", "splat"):
        st = TrainStep(P, large.sh_degree, large.cameras, large.targets, StepConfig(backward=bw),
                       capacity=int(M * 1.1) + 4096)
        st.run()
        torch.cuda.synchronize()
        assert st.error() == 0
        out[bw] = (st.image.clone(), st.loss.clone(), {k: v.clone() for k, v in st.pgrads.items()})
        del st
        torch.cuda.empty_cache()
    assert torch.equal(out["pixel"][0], out["splat"][0])
    assert torch.allclose(out["pixel"][1], out["splat"][1], rtol=1e-5, atol=0)   # atomic partial sums
    for k in R.PARAM_KEYS:
        e = rel_l2(out["splat"][2][k].cpu().numpy(), out["pixel"][2][k].cpu().numpy())
        assert e < 1e-4, (k, e)
