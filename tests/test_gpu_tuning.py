"""The step's tuning knobs and the autotuner that picks them (tile shape, tile-id
bits sorted during emission, the backward's staging depth, per-pixel or per-splat
backward): none changes the rendered images, and the gradients agree up to
summation order."""
import numpy as np
import pytest
import torch

from paper_2507_20239_gb300 import rasterizer as R
from paper_2507_20239_gb300.autotune import autotune, default_candidates
from paper_2507_20239_gb300.step import StepConfig, TrainStep
from tests.gs_fixtures import dev_params, rel_l2, scene

pytestmark = pytest.mark.gpu


def _run(sc, P, cfg, store_stop=True):
    st = TrainStep(P, sc.sh_degree, sc.cameras, sc.targets, cfg, store_stop=store_stop)
    st.run()
    torch.cuda.synchronize()
    assert st.error() == 0
    return st


def test_knobs_keep_images_and_gradients():
    sc = scene("batched_small")                  # six mixed-resolution views
    P = dev_params(sc)
    ref = _run(sc, P, StepConfig())
    cands = default_candidates(tiles=((16, 16), (8, 8), (16, 32)), fused_bits=(0, 2, 8), stage_depths=(0, 1))
    # 9 (tile, bits) pairs x (two staging depths + per-splat, per-tile or queued forward)
    assert len(cands) == 36
    for cfg in cands + ["recomputed"]:
        st = _run(sc, P, StepConfig(), store_stop=False) if cfg == "recomputed" else _run(sc, P, cfg)
        for v in range(len(sc.cameras)):
            assert torch.equal(st.frame.view_image(st.image, v), ref.frame.view_image(ref.image, v)), cfg
        # the per-view loss sums block partials atomically: equal up to summation order
        assert torch.allclose(st.loss, ref.loss, rtol=1e-5, atol=0), cfg
        for k in R.PARAM_KEYS:
            e = rel_l2(st.pgrads[k].cpu().numpy(), ref.pgrads[k].cpu().numpy())
            assert e < 1e-4, (cfg, k, e)
        # visibility (radius > 0) needs a non-empty tile rectangle, so a record whose
        # box only meets the padding of a partial edge tile counts for one tile shape
        # and not another; it never touches a pixel and gets a zero gradient
        if st.config.tile == ref.config.tile:
            assert torch.equal(st.stats.count, ref.stats.count), cfg
        # the statistic is a per-Gaussian norm of a sum of per-pixel terms that can
        # cancel; summed in another order (the per-splat backward also starts each
        # 32-entry bucket from the forward's checkpoint) a small one moves by more
        # than 1e-4 of itself, so it is held like the gradients: relative L2, and
        # element-wise against the largest value
        a, b = st.stats.accum.double(), ref.stats.accum.double()
        assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) < 1e-4, cfg
        assert torch.all((a - b).abs() <= 1e-4 * b.abs() + 1e-5 * b.abs().max()), cfg


def test_autotune_picks_a_measured_candidate():
    sc = scene("batched_small")
    P = dev_params(sc)
    cands = [StepConfig((16, 16)), StepConfig((8, 8), 0, 1), StepConfig((16, 32), 8, 0)]
    res = autotune(P, sc.sh_degree, sc.cameras, sc.targets, candidates=cands, reps=2)
    assert res.best in cands
    assert res.images_identical
    timed = [ms for _, ms, _ in res.table if ms is not None]
    assert len(timed) == 3 and res.best_ms == min(timed) and all(np.isfinite(timed))
    # cached for the same scene size, views and candidates
    assert autotune(P, sc.sh_degree, sc.cameras, sc.targets, candidates=cands, reps=2) is res


def test_invalid_stage_depth_is_rejected():
    sc = scene("small")
    P = dev_params(sc)
    st = _run(sc, P, StepConfig())
    with pytest.raises(RuntimeError):
        R.raster_bwd(st.proj, st.bins, st.frame, st.image, st.d_image, stage_depth=3)


@pytest.mark.parametrize("name,tile", [("orbit_small", (16, 16)), ("batched_small", (8, 8)),
                                       ("batched_small", (16, 32))])
def test_queued_forward_is_identical(name, tile):
    """The forward as a persistent grid of warps claiming (tile, 8x8 block) units:
    the image, transmittance and stop indices of the one-CTA-per-tile forward, bit for
    bit, with and without checkpoints; the per-splat backward from the queued
    forward's checkpoints gives the same gradients."""
    sc = scene(name)
    frame = R.Frame(sc.cameras, tile=tile)
    proj = R.project(dev_params(sc), sc.sh_degree, frame)
    bins = R.bin_sort(proj, frame)
    q = torch.zeros(1, dtype=torch.int32, device="cuda")
    a = R.raster_fwd(proj, bins, frame, store_stop=True)
    b = R.raster_fwd(proj, bins, frame, store_stop=True, queue=q)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    assert int(q.item()) >= frame.n_tiles * tile[0] * tile[1] // 64      # every unit was claimed
    ck_a, ck_b = R.alloc_ckpt(frame, bins), R.alloc_ckpt(frame, bins)
    fa = R.raster_fwd_ckpt(proj, bins, frame, ck_a)
    fb = R.raster_fwd_ckpt(proj, bins, frame, ck_b, queue=q)
    for x, y in zip(fa, fb):
        assert torch.equal(x, y)
    dg = torch.as_tensor(np.random.default_rng(4).normal(0, 1, fa[0].numel()).astype(np.float32)).cuda()
    ga = R.raster_bwd_splat(proj, bins, frame, fa[0], dg, fa[2], ck_a)
    gb = R.raster_bwd_splat(proj, bins, frame, fb[0], dg, fb[2], ck_b)
    torch.cuda.synchronize()
    for x, y in ((ga.d_mean2d, gb.d_mean2d), (ga.d_conic_opacity, gb.d_conic_opacity), (ga.d_rgb, gb.d_rgb)):
        assert rel_l2(x.cpu().numpy(), y.cpu().numpy()) < 1e-6
