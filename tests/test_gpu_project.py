"""gs_project (EWA projection + SH colour) and gs_project_bwd against the FP64 oracle."""
import numpy as np
import pytest
import torch

from oracle import pipeline as opipe
from oracle import project as oproj
from paper_2507_20239_gb300 import rasterizer as R
from paper_2507_20239_gb300 import synth
from tests.gs_fixtures import dev_params, rel_l2, scene

pytestmark = pytest.mark.gpu


def _straddle_ok(pr, tile=16, tol=1e-4):
    """Records whose integer outputs (radius, rect, visibility) sit within rounding
    distance of a decision boundary in the FP64 oracle."""
    half = np.where(pr["half"] > 0, pr["half"], 0.0)
    hmax = half.max(1)
    near_int = np.abs(hmax - np.round(hmax)) < tol * np.maximum(hmax, 1)
    u, v = pr["mean2d"][:, 0], pr["mean2d"][:, 1]
    edges = np.stack([(u - half[:, 0]) / tile, (v - half[:, 1]) / tile, (u + half[:, 0]) / tile,
                      (v + half[:, 1]) / tile], 1)
    near_edge = (np.abs(edges - np.round(edges)) < tol).any(1)
    o = pr["opacity"]
    near_o = np.abs(o * 255 - 1) < 1e-5
    return near_int | near_edge | near_o


def _compare_projection(sc, cams, tile=(16, 16), sample=None):
    frame = R.Frame(cams, tile=tile)
    P = dev_params(sc)
    proj = R.project(P, sc.sh_degree, frame)
    torch.cuda.synchronize()
    n = sc.n
    idx = np.arange(n) if sample is None else sample
    sub = {k: v[idx] for k, v in sc.params().items()}
    for v, cam in enumerate(cams):
        pr = oproj.project_np(sub, sc.sh_degree, cam, tile[0], tile[1])
        rows = v * n + idx
        rad = proj.radius.cpu().numpy()[rows]
        rect = proj.rect_np()[rows]
        ok = _straddle_ok(pr, tile[0])
        vis_o = pr["visible"]
        vis_g = rad > 0
        bad = (vis_o != vis_g) & ~ok
        assert bad.sum() == 0, f"visibility differs on {bad.sum()} non-straddling records"
        both = vis_o & vis_g & ~ok
        assert np.array_equal(rad[both], pr["radius"][both])
        assert np.array_equal(rect[both], pr["rect"][both])
        assert both.sum() > 0.5 * vis_o.sum()
        vis = vis_o & vis_g
        m2 = proj.mean2d.cpu().numpy()[rows][vis]
        assert np.abs(m2 - pr["mean2d"][vis]).max() < 2e-3
        co = proj.conic_opacity.cpu().numpy()[rows][vis]
        cf = pr["conic_f"][vis]
        # the conic (A B; B C) = (A, A beta; A beta, gamma + A beta^2) implied by the
        # factored form, per record to a relative 1e-5 of its largest entry
        def mat(f):
            f = f.astype(np.float64)
            return np.stack([f[:, 0], f[:, 0] * f[:, 1], f[:, 2] + f[:, 0] * f[:, 1] ** 2], 1)
        mg, mo = mat(co[:, :3]), mat(cf)
        rel = np.abs(mg - mo).max(1) / np.abs(mo).max(1)
        assert rel.max() < 1e-5, rel.max()
        assert np.abs(co[:, 3] - pr["opacity"][vis]).max() < 1e-6
        dep = proj.depth.cpu().numpy()[rows][vis]
        assert np.abs(dep - pr["depth"][vis]).max() < 1e-5 * np.abs(pr["depth"][vis]).max()
        rgb = proj.rgb.cpu().numpy()[rows][vis]
        assert np.abs(rgb[:, :3] - pr["rgb"][vis]).max() < 2e-6
        assert np.abs(rgb[:, 3] - pr["q_max"][vis]).max() < 2e-5          # q_max = 2 ln(255 o)
        cl = proj.clamped.cpu().numpy()[rows][vis]
        want = (pr["clamped"][vis] * np.array([1, 2, 4])).sum(1)
        near0 = (np.abs(pr["rgb"][vis] - 0) < 1e-6).any(1)
        assert np.array_equal(cl[~near0], want[~near0])
        # culled rows are all zero
        cul = ~vis_g
        assert np.all(proj.conic_opacity.cpu().numpy()[rows][cul] == 0)


def test_project_small_scene():
    sc = scene("small")
    _compare_projection(sc, sc.cameras)


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (16, 32)])
def test_project_orbit_sh3_tiles(tile):
    sc = scene("orbit_small")
    _compare_projection(sc, sc.cameras, tile)


def test_project_multiview_mixed_resolution():
    sc = scene("batched_small")
    _compare_projection(sc, sc.cameras)


def test_project_full_size_sampled():
    sc = scene("orbit")                       # 1.5M Gaussians, SH degree 3, 1246x826
    rng = np.random.default_rng(0)
    sample = np.sort(rng.choice(sc.n, 20000, replace=False))
    _compare_projection(sc, sc.cameras, sample=sample)


def _rand_rec_grads(rng, R_, scale=1.0):
    return dict(d_mean2d=rng.normal(0, scale, (R_, 2)), d_conic=rng.normal(0, scale, (R_, 3)),
                d_opacity=rng.normal(0, scale, R_), d_rgb=rng.normal(0, scale, (R_, 3)))


def _rec_grads_gpu(gs):
    n = gs[0]["d_mean2d"].shape[0]
    V = len(gs)
    co = np.zeros((V * n, 4), np.float32)
    co[:, :3] = np.concatenate([g["d_conic"] for g in gs])
    co[:, 3] = np.concatenate([g["d_opacity"] for g in gs])
    rgb = np.zeros((V * n, 4), np.float32)
    rgb[:, :3] = np.concatenate([g["d_rgb"] for g in gs])
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda()
    return R.RecGrads(t(np.concatenate([g["d_mean2d"] for g in gs])), t(co), t(rgb))


@pytest.mark.parametrize("name", ["small", "orbit_small", "batched_small"])
def test_project_vjp_matches_oracle(name):
    sc = scene(name)
    cams = sc.cameras
    n = min(sc.n, 4000)
    sub = {k: v[:n] for k, v in sc.params().items()}
    frame = R.Frame(cams)
    P = {k: torch.as_tensor(np.ascontiguousarray(v)).cuda() for k, v in sub.items()}
    proj = R.project(P, sc.sh_degree, frame)
    rng = np.random.default_rng(1)
    gs = [{k: v.astype(np.float32) for k, v in _rand_rec_grads(rng, n).items()} for _ in cams]
    rad = proj.radius.cpu().numpy().reshape(len(cams), n)
    # the oracle's gradient is zero for culled records; agree on visibility first
    vis = [oproj.project_np(sub, sc.sh_degree, c)["visible"] for c in cams]
    for v in range(len(cams)):
        assert np.array_equal(vis[v], rad[v] > 0)
    out = R.project_bwd(P, sc.sh_degree, frame, proj, _rec_grads_gpu(gs))
    torch.cuda.synchronize()
    want = opipe.project_vjp(sub, sc.sh_degree, cams, gs)
    for k in R.PARAM_KEYS:
        got = out[k].cpu().numpy()
        assert rel_l2(got, want[k]) < 1e-4, (k, rel_l2(got, want[k]))


def test_project_vjp_clamped_colour_and_fov_clamp():
    # a Gaussian far off to the side (J clamp active) and one with a clamped channel
    cam = synth.Camera(R=np.eye(3, dtype=np.float32), t=np.array([0, 0, 2], np.float32), fx=60.0, fy=60.0,
                       cx=32.0, cy=32.0, width=64, height=64)
    p = dict(means=np.array([[1.2, 0.0, 0.0], [0.05, 0.1, 0.3]], np.float32),
             log_scales=np.array([[-0.5, -0.8, -0.6], [-2.0, -2.2, -1.9]], np.float32),
             quats=np.array([[0.9, 0.1, 0.2, 0.3], [0.5, -0.5, 0.5, 0.5]], np.float32),
             opacity_logits=np.array([0.3, -0.2], np.float32),
             sh=np.array([[[0.2, -3.0, 0.5]], [[-4.0, 0.1, 0.9]]], np.float32))
    frame = R.Frame([cam])
    P = {k: torch.as_tensor(v).cuda() for k, v in p.items()}
    proj = R.project(P, 0, frame)
    assert (proj.radius.cpu().numpy() > 0).all()
    assert list(proj.clamped.cpu().numpy()) == [2, 1]
    rng = np.random.default_rng(3)
    g = {k: v.astype(np.float32) for k, v in _rand_rec_grads(rng, 2).items()}
    out = R.project_bwd(P, 0, frame, proj, _rec_grads_gpu([g]))
    want = opipe.project_vjp(p, 0, [cam], [g])
    for k in R.PARAM_KEYS:
        assert rel_l2(out[k].cpu().numpy(), want[k]) < 1e-4, k
