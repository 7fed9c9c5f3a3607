"""gs_raster_fwd_ckpt / gs_raster_bwd_splat (the per-splat backward) against the
FP64 oracle and against the per-pixel gs_raster_bwd.

Both sides consume the same FP32 records (the oracle's FP64 projection rounded);
the oracle's gradient is that of Eq. 2 evaluated in FP64 (the same one the
per-pixel backward is held to). The forward that stores checkpoints must render
exactly what gs_raster_fwd renders.
"""
import numpy as np
import pytest
import torch

from oracle import raster as oras
from paper_2507_20239_gb300 import rasterizer as R
from paper_2507_20239_gb300 import synth
from paper_2507_20239_gb300._abi import GsError
from tests.gs_fixtures import oracle_lists, oracle_records_fp32, records_to_gpu, rel_l2, scene

pytestmark = pytest.mark.gpu
GRAD_TOL = 1e-3          # against the FP64 oracle (as for gs_raster_bwd)
SAME_TOL = 1e-4          # against gs_raster_bwd: FP32 on both sides, summation order differs


def _fwd_both(recs, cams, tile, bg):
    frame = R.Frame(cams, tile=tile)
    proj = records_to_gpu(recs)
    bins = R.bin_sort(proj, frame)
    ckpt = R.alloc_ckpt(frame, bins)
    img, T, stop = R.raster_fwd_ckpt(proj, bins, frame, ckpt, bg)
    img0, T0, stop0 = R.raster_fwd(proj, bins, frame, bg, store_stop=True)
    torch.cuda.synchronize()
    assert torch.equal(img, img0) and torch.equal(T, T0) and torch.equal(stop, stop0)
    return frame, proj, bins, img, stop, ckpt


def _grads(rg):
    return dict(d_mean2d=rg.d_mean2d.cpu().numpy(), d_conic=rg.d_conic_opacity[:, :3].cpu().numpy(),
                d_opacity=rg.d_conic_opacity[:, 3].cpu().numpy(), d_rgb=rg.d_rgb[:, :3].cpu().numpy())


def _oracle_vjp(rec, cam, tile, bg, d_image, tiles=None):
    return oras.raster_vjp(rec["mean2d"], rec["conic_f"], rec["opacity"], rec["rgb"], oracle_lists(rec),
                           cam.width, cam.height, d_image, tile[0], tile[1], bg, tiles)


@pytest.mark.parametrize("name,tile,bg", [("small", (16, 16), (0, 0, 0)), ("small", (8, 8), (0.2, 0.5, 1.0)),
                                          ("orbit_small", (16, 16), (0.1, 0.2, 0.3)),
                                          ("orbit_small", (8, 8), (0, 0, 0)),
                                          ("orbit_small", (16, 32), (0, 0, 0)),
                                          ("orbit_small", (32, 16), (0.3, 0.3, 0.3))])
def test_splat_bwd_matches_oracle(name, tile, bg):
    sc = scene(name)
    cam = sc.cameras[0]
    rec = oracle_records_fp32(sc.params(), sc.sh_degree, cam, tile)
    frame, proj, bins, img, stop, ckpt = _fwd_both([rec], [cam], tile, bg)
    rng = np.random.default_rng(7)
    d_image = rng.normal(0, 1, (3, cam.height, cam.width)).astype(np.float32)
    o, g = _oracle_vjp(rec, cam, tile, bg, d_image)
    assert o["flag"].sum() <= max(2, 2e-3 * o["flag"].size)
    dg = torch.as_tensor(d_image.reshape(-1)).cuda()
    rs = R.raster_bwd_splat(proj, bins, frame, img, dg, stop, ckpt)
    rp = R.raster_bwd(proj, bins, frame, img, dg, bg, stop=stop)
    torch.cuda.synchronize()
    got, pix = _grads(rs), _grads(rp)
    assert np.all(rs.d_rgb[:, 3].cpu().numpy() == 0)
    for k in got:
        e = rel_l2(got[k], g[k])
        assert e < GRAD_TOL, (k, e)
        e2 = rel_l2(got[k], pix[k])
        assert e2 < SAME_TOL, (k, e2)
    cul = rec["radius"] == 0
    assert np.all(got["d_mean2d"][cul] == 0) and np.all(got["d_rgb"][cul] == 0)


def test_splat_full_size_view_sampled_tiles():
    """1.5M Gaussians at 1246x826 (the benchmark's view): the oracle back-propagates
    a d_image that is non-zero on 24 sampled tiles and the 4 longest lists; the
    whole-image gradient is compared with the per-pixel backward."""
    sc = scene("orbit")
    cam = sc.cameras[0]
    tile = (16, 16)
    rec = oracle_records_fp32(sc.params(), sc.sh_degree, cam, tile)
    frame, proj, bins, img, stop, ckpt = _fwd_both([rec], [cam], tile, (0, 0, 0))
    ranges = bins.ranges.cpu().numpy()
    lens = ranges[:, 1] - ranges[:, 0]
    rng = np.random.default_rng(11)
    busy = np.nonzero(lens > 0)[0]
    tiles = sorted(set(rng.choice(busy, 24, replace=False).tolist()) | set(np.argsort(lens)[-4:].tolist()))
    gx = (cam.width + tile[0] - 1) // tile[0]
    mask = np.zeros((cam.height, cam.width), bool)
    for t in tiles:
        tx, ty = t % gx, t // gx
        mask[ty * tile[1]:(ty + 1) * tile[1], tx * tile[0]:(tx + 1) * tile[0]] = True
    d_image = np.where(mask[None], rng.normal(0, 1, (3, cam.height, cam.width)), 0).astype(np.float32)
    _, g = _oracle_vjp(rec, cam, tile, (0, 0, 0), d_image, tiles=tiles)
    rs = R.raster_bwd_splat(proj, bins, frame, img, torch.as_tensor(d_image.reshape(-1)).cuda(), stop, ckpt)
    torch.cuda.synchronize()
    got = _grads(rs)
    for k in got:
        e = rel_l2(got[k], g[k])
        assert e < GRAD_TOL, (k, e)
    # the whole view, a dense d_image: per-splat against per-pixel
    dg = torch.as_tensor(rng.normal(0, 1, 3 * cam.height * cam.width).astype(np.float32)).cuda()
    rs = R.raster_bwd_splat(proj, bins, frame, img, dg, stop, ckpt)
    rp = R.raster_bwd(proj, bins, frame, img, dg, stop=stop)
    torch.cuda.synchronize()
    got, pix = _grads(rs), _grads(rp)
    for k in got:
        e = rel_l2(got[k], pix[k])
        assert e < SAME_TOL, (k, e)


def test_splat_batched_mixed_resolution_views():
    sc = scene("batched_small")
    recs = [oracle_records_fp32(sc.params(), sc.sh_degree, c) for c in sc.cameras]
    frame, proj, bins, img, stop, ckpt = _fwd_both(recs, sc.cameras, (16, 16), (0, 0, 0))
    dg = torch.as_tensor(np.random.default_rng(3).normal(0, 1, img.numel()).astype(np.float32)).cuda()
    rs = R.raster_bwd_splat(proj, bins, frame, img, dg, stop, ckpt)
    rp = R.raster_bwd(proj, bins, frame, img, dg, stop=stop)
    torch.cuda.synchronize()
    got, pix = _grads(rs), _grads(rp)
    for k in got:
        e = rel_l2(got[k], pix[k])
        assert e < SAME_TOL, (k, e)
    # every view's share against the oracle on that view alone
    n = sc.params()["means"].shape[0]
    for v in (0, len(sc.cameras) - 1):
        cam = sc.cameras[v]
        d_v = frame.view_image(dg, v).cpu().numpy().reshape(3, cam.height, cam.width)
        _, g = _oracle_vjp(recs[v], cam, (16, 16), (0, 0, 0), d_v)
        sl = slice(v * n, (v + 1) * n)
        for k in got:
            e = rel_l2(got[k][sl], g[k])
            assert e < GRAD_TOL, (v, k, e)


def test_splat_ragged_image_and_empty_tiles():
    # a 37x23 image (ragged last tile row and column) where most tiles are empty
    sc = synth.small_scene(3, n=40, width=37, height=23)
    cam = sc.cameras[0]
    rec = oracle_records_fp32(sc.params(), 0, cam)
    frame, proj, bins, img, stop, ckpt = _fwd_both([rec], [cam], (16, 16), (0.1, 0.1, 0.1))
    d_image = np.random.default_rng(5).normal(0, 1, (3, cam.height, cam.width)).astype(np.float32)
    _, g = _oracle_vjp(rec, cam, (16, 16), (0.1, 0.1, 0.1), d_image)
    rs = R.raster_bwd_splat(proj, bins, frame, img, torch.as_tensor(d_image.reshape(-1)).cuda(), stop, ckpt)
    torch.cuda.synchronize()
    got = _grads(rs)
    for k in got:
        e = rel_l2(got[k], g[k])
        assert e < GRAD_TOL, (k, e)


def test_splat_nothing_visible():
    # every Gaussian behind the camera: empty lists, zero gradients (the buffers are
    # overwritten, not accumulated into)
    sc = synth.small_scene(4, n=64, width=40, height=30)
    cam = sc.cameras[0]
    rec = oracle_records_fp32(sc.params(), 0, cam)
    for k in ("radius",):
        rec[k] = np.zeros_like(rec[k])
    rec["rect"][:] = 0
    frame, proj, bins, img, stop, ckpt = _fwd_both([rec], [cam], (16, 16), (0.5, 0.5, 0.5))
    assert int(bins.count.item()) == 0
    grads = R.RecGrads.zeros(proj.mean2d.shape[0], frame.device)
    for t in (grads.d_mean2d, grads.d_conic_opacity, grads.d_rgb):
        t.fill_(7.0)
    dg = torch.ones(img.numel(), device="cuda")
    R.raster_bwd_splat(proj, bins, frame, img, dg, stop, ckpt, grads=grads)
    torch.cuda.synchronize()
    for t in (grads.d_mean2d, grads.d_conic_opacity, grads.d_rgb):
        assert torch.count_nonzero(t) == 0
    assert torch.all(img == 0.5)


def test_ckpt_size_and_argument_errors():
    sc = scene("small")
    cam = sc.cameras[0]
    rec = oracle_records_fp32(sc.params(), sc.sh_degree, cam)
    frame, proj, bins, img, stop, ckpt = _fwd_both([rec], [cam], (16, 16), (0, 0, 0))
    cap = bins.capacity
    entries = ((cap + 31) // 32 + frame.n_tiles) * 4
    head = 1024 + (4 * entries + 255) // 256 * 256
    assert R.ckpt_bytes(frame, cap) == head + entries * 1024
    assert ckpt.numel() == R.ckpt_bytes(frame, cap)
    short = ckpt[:head - 16]                       # not even the pool counters and table
    with pytest.raises(GsError):
        R.raster_fwd_ckpt(proj, bins, frame, short)
    dg = torch.zeros_like(img)
    with pytest.raises(GsError):
        R.raster_bwd_splat(proj, bins, frame, img, dg, stop, short)
    with pytest.raises(GsError):
        R.raster_bwd_splat(proj, bins, frame, img, dg, stop, ckpt[8:])      # not 16-byte aligned
    with pytest.raises(GsError):
        R.ckpt_bytes(frame, -1)


@pytest.mark.parametrize("name,tile", [("orbit_small", (16, 16)), ("orbit_small", (32, 16)), ("orbit", (16, 16))])
def test_measured_checkpoint_slots(name, tile):
    """A buffer sized from the measured slot count (a forward into a buffer without
    slots reports it) gives the gradients of the buffer with a slot for every
    (bucket, block) pair; a buffer with too few slots reports it and runs without
    fault."""
    sc = scene(name)
    cam = sc.cameras[0]
    frame = R.Frame([cam], tile=tile)
    proj = R.project({k: torch.as_tensor(v).cuda() for k, v in sc.params().items()}, sc.sh_degree, frame)
    bins = R.bin_sort(proj, frame)
    probe = R.alloc_ckpt(frame, bins, 0)
    R.raster_fwd_ckpt(proj, bins, frame, probe)
    use = R.ckpt_usage(frame, bins, probe).cpu().numpy()
    need = int(use[0])
    assert need > 0 and use[1] == 1
    full = R.alloc_ckpt(frame, bins)
    fit = R.alloc_ckpt(frame, bins, need)
    dg = torch.as_tensor(np.random.default_rng(2).normal(0, 1, 3 * frame.n_pixels).astype(np.float32)).cuda()
    grads = {}
    for label, ck in (("full", full), ("fit", fit)):
        img, T, stop = R.raster_fwd_ckpt(proj, bins, frame, ck)
        assert int(R.ckpt_usage(frame, bins, ck)[1].item()) == 0
        grads[label] = _grads(R.raster_bwd_splat(proj, bins, frame, img, dg, stop, ck))
    for k in grads["full"]:
        assert rel_l2(grads["fit"][k], grads["full"][k]) < 1e-5, k
    print(f"{name} {tile}: {need} slots, {fit.numel() / 1e6:.1f} MB against {full.numel() / 1e6:.1f} MB")
    assert fit.numel() < (0.2 if name == "orbit" else 0.8) * full.numel()
    small = R.alloc_ckpt(frame, bins, need // 2)
    img, T, stop = R.raster_fwd_ckpt(proj, bins, frame, small)
    assert int(R.ckpt_usage(frame, bins, small)[1].item()) == 1
    g = _grads(R.raster_bwd_splat(proj, bins, frame, img, dg, stop, small))
    torch.cuda.synchronize()
    assert all(np.isfinite(v).all() for v in g.values())


def test_autograd_splat_backward_matches_pixel_backward():
    """autograd.rasterize(backward="splat") against the per-pixel wrapper: the same
    image, parameter gradients within summation order, the same densification counts."""
    from paper_2507_20239_gb300.autograd import DensifyStats, rasterize
    from tests.gs_fixtures import dev_params
    sc = scene("batched_small")
    frame = R.Frame(sc.cameras)
    tgt = frame.pack_images(sc.targets)
    out = {}
    for bw in ("pixel", "splat"):
        P = {k: v.clone().requires_grad_(True) for k, v in dev_params(sc).items()}
        stats = DensifyStats.zeros(sc.n)
        img, _ = rasterize(P, sc.sh_degree, frame, stats=stats, backward=bw)
        (img - tgt).abs().mean().backward()
        torch.cuda.synchronize()
        out[bw] = (img.detach(), {k: P[k].grad for k in R.PARAM_KEYS}, stats)
    assert torch.equal(out["pixel"][0], out["splat"][0])
    for k in R.PARAM_KEYS:
        e = rel_l2(out["splat"][1][k].cpu().numpy(), out["pixel"][1][k].cpu().numpy())
        assert e < SAME_TOL, (k, e)
    assert torch.equal(out["pixel"][2].count, out["splat"][2].count)
    assert rel_l2(out["splat"][2].accum.cpu().numpy(), out["pixel"][2].accum.cpu().numpy()) < SAME_TOL
    with pytest.raises(ValueError):
        rasterize({k: v for k, v in dev_params(sc).items()}, sc.sh_degree, frame, backward="tile")


def test_training_steps_with_the_splat_backward():
    """A few hundred steps of the trainer on the per-splat backward: the loss falls
    and the densification events run (the arithmetic of each event is pinned by the
    per-pixel training test)."""
    from paper_2507_20239_gb300 import train as T
    gt = synth.surface_scene(13, 60_000, 3)
    cams = T.orbit_views(4, 320, 212, 320.0)
    views = {r: (c, T.render_targets(gt.params(), 3, c)) for r, c in cams.items()}
    init = synth.surface_scene(3, 8_000, 3).params()
    sched = T.Schedule(stages=[(0, 4, R.DENSIFY_SPLIT_ONLY), (100, 2, R.DENSIFY_SPLIT_ONLY),
                               (200, 1, R.DENSIFY_ADAPTIVE)], total=300, densify_from=50,
                       densify_until=250, densify_every=50, sh_every=75, backward="splat")
    tr = T.Trainer(init, views, sched, extent=1.1 * 4.0)
    hist = tr.run(log_every=50)                     # (step, N, L1 + D-SSIM loss)
    assert hist[-1][2] < hist[0][2], hist
    assert [e[0] for e in tr.events] == [50, 100, 150, 200, 250]
