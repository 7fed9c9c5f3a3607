"""Central finite differences on 64 random parameters of the full-size training view
(1.5M Gaussians, SH degree 3, 1246x826, L1 loss) against the GPU's analytic
gradient.

The GPU step (TrainStep, the benchmark's launch sequence) gives every parameter
gradient in FP32. For each sampled scalar the FP64 oracle re-renders only the tiles
the perturbed Gaussian is listed in (before or after the step of +-h), with every
other record at its FP64 projection, and differences the L1 loss (mean over
3*H*W). A sample is rejected when the +-h renders differ in a discrete decision
(a pixel's composited count or stop position, or an L1 sign), since the loss is
not differentiable there.
"""
import numpy as np
import pytest
import torch

from oracle import pipeline as opipe
from oracle import project as oproj
from oracle import raster as oras
from paper_2507_20239_gb300.step import StepConfig, TrainStep
from tests.gs_fixtures import dev_params, scene

pytestmark = pytest.mark.gpu
TILE = 16


def _record_tiles(pr1, cam):
    lists = oras.tile_lists(opipe.proj_record_arrays(pr1), cam.width, cam.height, TILE, TILE)
    return {t for t, ids in lists.items() if ids.size}


class _TileRenderer:
    """FP64 loss of a set of tiles with one Gaussian's record replaced."""

    def __init__(self, params, sh_degree, cam, target):
        self.params, self.sh, self.cam = params, sh_degree, cam
        self.target = np.asarray(target, np.float64)
        pr = oproj.project_np(params, sh_degree, cam, TILE, TILE)
        self.pr = pr
        self.lists = oras.tile_lists(opipe.proj_record_arrays(pr), cam.width, cam.height, TILE, TILE)
        self.key = pr["depth"].astype(np.float32).view(np.uint32)
        self.gx = (cam.width + TILE - 1) // TILE
        self.n_pix = 3 * cam.width * cam.height

    def tiles_of(self, g):
        return {t for t, ids in self.lists.items() if ids.size and (ids == g).any()}

    def project_one(self, g, mutate):
        sub = {k: np.array(v[g:g + 1], copy=True) for k, v in self.params.items()}
        mutate(sub)
        return oproj.project_np(sub, self.sh, self.cam, TILE, TILE)

    def tile_loss(self, t, g, pr1):
        """L1 numerator over tile t with record g replaced by pr1 (1-record arrays)."""
        ids = self.lists.get(t, np.zeros(0, np.int64))
        ids = ids[ids != g]
        hit = t in _record_tiles(pr1, self.cam) if pr1["visible"][0] else False
        xy, cf = self.pr["mean2d"][ids], self.pr["conic_f"][ids]
        op, rgb = self.pr["opacity"][ids], self.pr["rgb"][ids]
        if hit:
            kg = np.float32(pr1["depth"][0]).view(np.uint32)
            keys = self.key[ids]
            full = (keys.astype(np.uint64) << np.uint64(32)) | ids.astype(np.uint64)
            pos = int(np.searchsorted(full, (np.uint64(kg) << np.uint64(32)) | np.uint64(g)))
            ins = lambda a, b: np.concatenate([a[:pos], b, a[pos:]])
            xy, cf = ins(xy, pr1["mean2d"]), ins(cf, pr1["conic_f"])
            op, rgb = ins(op, pr1["opacity"]), ins(rgb, pr1["rgb"])
        X, Y = oras.tile_pixels(t, self.gx, TILE, TILE, self.cam.width, self.cam.height)
        rec = oras.records_to_torch(xy, cf, op, rgb)
        with torch.no_grad():
            out, _, st, _, nc, fl = oras.composite(X + 0.5, Y + 0.5, rec["mean2d"], rec["conic_f"],
                                                    rec["opacity"], rec["rgb"], (0.0, 0.0, 0.0))
        diff = out.numpy().T - self.target[:, Y, X]
        return np.abs(diff).sum(), (np.asarray(st), np.asarray(nc), np.sign(diff), np.asarray(fl))


def _mutator(key, idx, delta):
    def f(sub):
        a = sub[key].reshape(-1)
        a[idx] = a[idx] + delta
    return f


def test_central_differences_on_64_parameters_full_view():
    sc = scene("orbit")
    cam = sc.cameras[0]
    params = sc.params()
    P = dev_params(sc)
    step = TrainStep(P, sc.sh_degree, [cam], sc.targets, StepConfig((TILE, TILE)))
    step.run()
    torch.cuda.synchronize()
    assert step.error() == 0
    g_gpu = {k: v.cpu().numpy() for k, v in step.pgrads.items()}

    tr = _TileRenderer({k: np.asarray(v, np.float64) for k, v in params.items()}, sc.sh_degree, cam,
                       sc.targets[0])
    # candidates: visible Gaussians listed in 1..4 tiles with a non-negligible gradient
    rng = np.random.default_rng(64)
    vis = np.nonzero(tr.pr["visible"])[0]
    rect = tr.pr["rect"][vis]
    small = vis[((rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1])) <= 4]
    gnorm = np.abs(g_gpu["opacity_logits"][small])
    pool = small[gnorm > np.percentile(gnorm, 50)]
    groups = [("means", 3)] * 13 + [("log_scales", 3)] * 13 + [("quats", 4)] * 12 + \
             [("opacity_logits", 1)] * 12 + [("sh_dc", 3)] * 7 + [("sh_rest", 45)] * 7
    fd, an, rejected = [], [], 0
    for grp, width in groups:
        g = int(rng.choice(pool))
        comp = int(rng.integers(width))
        if grp == "sh_dc":
            key, idx = "sh", comp
        elif grp == "sh_rest":
            key, idx = "sh", 3 + comp
        else:
            key, idx = grp, comp
        theta = float(np.asarray(params[key][g]).reshape(-1)[idx])
        h = 1e-6 * max(1.0, abs(theta))
        prp = tr.project_one(g, _mutator(key, idx, +h))
        prm = tr.project_one(g, _mutator(key, idx, -h))
        tiles = tr.tiles_of(g) | (_record_tiles(prp, cam) if prp["visible"][0] else set()) | \
            (_record_tiles(prm, cam) if prm["visible"][0] else set())
        lp = lm = 0.0
        flip = False
        for t in tiles:
            a, sa = tr.tile_loss(t, g, prp)
            b, sb = tr.tile_loss(t, g, prm)
            lp += a
            lm += b
            flip |= any(not np.array_equal(x, y) for x, y in zip(sa[:3], sb[:3]))
        if flip or prp["visible"][0] != prm["visible"][0]:
            rejected += 1
            continue
        fd.append((lp - lm) / (2 * h) / tr.n_pix)
        an.append(float(g_gpu[key][g].reshape(-1)[idx]))
    fd, an = np.array(fd), np.array(an)
    assert len(fd) >= 48, (len(fd), rejected)
    err = np.linalg.norm(an - fd) / np.linalg.norm(fd)
    assert err < 1e-3, (err, len(fd), rejected)
    assert np.count_nonzero(fd) > 0.75 * len(fd)
