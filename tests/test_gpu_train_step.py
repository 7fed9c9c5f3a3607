"""The training step's loss (L1 + D-SSIM, gs_photometric_loss_grad), Adam
(gs_adam_step, dense and sparse) and opacity reset (gs_opacity_reset) against the
FP64 oracles on the same FP32 inputs."""
import math

import numpy as np
import pytest
import torch

from oracle import loss as oloss
from oracle import optim as oopt
from paper_2507_20239_gb300 import optim as O
from paper_2507_20239_gb300 import rasterizer as R
from paper_2507_20239_gb300 import synth
from tests.gs_fixtures import rel_l2

pytestmark = pytest.mark.gpu


def _cam(w, h):
    return synth.Camera(np.eye(3, dtype=np.float32), np.array([0, 0, 4], np.float32), float(w), float(w),
                        w / 2, h / 2, w, h)


@pytest.mark.parametrize("sizes", [[(80, 64)], [(53, 37), (120, 90), (7, 5)]])
def test_photometric_loss_and_gradient_match_oracle(sizes):
    rng = np.random.default_rng(len(sizes))
    cams = [_cam(w, h) for w, h in sizes]
    frame = R.Frame(cams)
    imgs = [rng.uniform(size=(3, h, w)).astype(np.float32) for w, h in sizes]
    tgts = [np.clip(im + rng.normal(0, 0.1, im.shape), 0, 1).astype(np.float32) for im in imgs]
    d_img, loss = O.photometric_loss_grad(frame, frame.pack_images(imgs), frame.pack_images(tgts), 0.2)
    torch.cuda.synchronize()
    for v, (im, tg) in enumerate(zip(imgs, tgts)):
        want_l, want_g = oloss.photometric_loss_grad(im, tg, 0.2)
        assert abs(float(loss[v]) - want_l) <= 1e-5 * want_l
        got = frame.view_image(d_img, v).cpu().numpy()
        assert rel_l2(got, want_g) < 1e-4


def test_photometric_loss_of_identical_images_is_zero():
    frame = R.Frame([_cam(40, 30)])
    img = frame.pack_images([np.random.default_rng(3).uniform(size=(3, 30, 40)).astype(np.float32)])
    d_img, loss = O.photometric_loss_grad(frame, img, img.clone(), 0.2)
    assert abs(float(loss[0])) < 1e-6 and float(d_img.abs().max()) < 1e-9


def _params(rng, n, K=16):
    return {"means": rng.normal(size=(n, 3)), "log_scales": rng.normal(-4, 0.5, (n, 3)),
            "quats": rng.normal(size=(n, 4)), "opacity_logits": rng.normal(size=n),
            "sh": rng.normal(0, 0.1, (n, K, 3))}


@pytest.mark.parametrize("sparse", [False, True])
def test_adam_step_matches_oracle(sparse):
    rng = np.random.default_rng(7)
    n = 5000
    p = {k: v.astype(np.float32) for k, v in _params(rng, n).items()}
    g = {k: (rng.normal(size=v.shape) * 10.0 ** rng.integers(-6, 0, v.shape)).astype(np.float32) for k, v in p.items()}
    m = {k: rng.normal(0, 1e-3, v.shape).astype(np.float32) for k, v in p.items()}
    vv = {k: np.abs(rng.normal(0, 1e-6, v.shape)).astype(np.float32) for k, v in p.items()}
    lrs = {"means": 7e-4, "log_scales": 5e-3, "quats": 1e-3, "opacity_logits": 5e-2, "sh": 2.5e-3}
    radius = np.where(rng.uniform(size=2 * n) < 0.4, rng.integers(1, 9, 2 * n), 0).astype(np.int32)
    vis = (radius.reshape(2, n) > 0).any(0)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda()
    P = {k: dev(v) for k, v in p.items()}
    opt = O.Adam(P, lrs)
    opt.m = {k: dev(v) for k, v in m.items()}
    opt.v = {k: dev(v) for k, v in vv.items()}
    opt.t = 2
    opt.step(P, {k: dev(v) for k, v in g.items()}, radius=dev(radius) if sparse else None, n_views=2)
    torch.cuda.synchronize()
    for k in p:
        wp, wm, wv = oopt.adam_step(p[k], g[k], m[k], vv[k], lrs[k], 3, visible=vis if sparse else None)
        gp, gm, gv = P[k].cpu().numpy(), opt.m[k].cpu().numpy(), opt.v[k].cpu().numpy()
        # the parameter step from the kernel's own moments (m may cancel in FP32, and
        # that rounding is checked just below): p - lr / bc1 m / (sqrt(v) / sqrt(bc2) + eps)
        bc1, bc2 = 1 - 0.9 ** 3, 1 - 0.999 ** 3
        step = lrs[k] / bc1 * gm.astype(np.float64) / (np.sqrt(gv.astype(np.float64)) / math.sqrt(bc2) + 1e-15)
        if sparse:
            step = np.where(vis.reshape((-1,) + (1,) * (p[k].ndim - 1)), step, 0.0)
        assert np.all(np.abs(gp - (p[k] - step)) <= 1e-6 * (np.abs(p[k]) + np.abs(step)) + 1e-12), k
        # FP32 rounding of beta m + (1 - beta) g, relative to the terms (they may cancel)
        assert np.all(np.abs(gm - wm) <= 1e-6 * (np.abs(m[k]) + np.abs(g[k])) + 1e-30), k
        assert np.all(np.abs(gv - wv) <= 1e-6 * (np.abs(vv[k]) + g[k].astype(np.float64) ** 2) + 1e-30), k
        if sparse:
            rows = ~vis
            assert np.array_equal(gp[rows], p[k][rows]) and np.array_equal(gm[rows], m[k][rows]), k


def test_opacity_reset_matches_oracle():
    rng = np.random.default_rng(8)
    lg = rng.normal(-2, 3, 10000).astype(np.float32)
    P = {"opacity_logits": torch.as_tensor(lg).cuda()}
    opt = O.Adam({k: torch.zeros(10000, 3, device="cuda") if k != "opacity_logits" else P[k] for k in R.PARAM_KEYS},
                 {k: 1e-3 for k in R.PARAM_KEYS})
    opt.m["opacity_logits"].fill_(0.5)
    O.opacity_reset(P, opt, 0.01)
    torch.cuda.synchronize()
    want = np.minimum(lg, np.float32(math.log(0.01 / 0.99)))
    assert np.array_equal(P["opacity_logits"].cpu().numpy(), want)
    assert np.allclose(want, oopt.opacity_reset(lg), atol=1e-7)
    assert float(opt.m["opacity_logits"].abs().max()) == 0.0
