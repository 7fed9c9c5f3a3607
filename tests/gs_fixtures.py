"""Shared helpers for the GPU parity tests: seeded scenes, oracle projections
rounded to FP32 (the records both sides then consume), and packing of those
records into the CUDA path's device layout."""
from __future__ import annotations

import functools

import numpy as np
import torch

from oracle import project as oproj
from oracle import raster as oras
from paper_2507_20239_gb300 import synth

DEV = "cuda"


def dev_params(scene) -> dict:
    return {k: torch.as_tensor(np.ascontiguousarray(v)).to(DEV) for k, v in scene.params().items()}


def oracle_records_fp32(params: dict, sh_degree: int, cam, tile=(16, 16)) -> dict:
    """FP64 oracle projection, rounded to FP32 records; rect decided in FP32 on them."""
    pr = oproj.project_np(params, sh_degree, cam, tile[0], tile[1])
    mean2d = pr["mean2d"].astype(np.float32)
    gx, gy = pr["grid"]
    half = pr["half"].astype(np.float32)
    rect = oproj.tile_rect(mean2d, half, tile[0], tile[1], gx, gy)
    area = (rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1])
    vis = pr["visible"] & (area > 0)
    rect[~vis] = 0
    radius = np.where(vis, pr["radius"], 0).astype(np.int32)
    return dict(mean2d=mean2d, conic_f=pr["conic_f"].astype(np.float32), opacity=pr["opacity"].astype(np.float32),
                rgb=pr["rgb"].astype(np.float32), q_max=pr["q_max"].astype(np.float32),
                depth=np.where(vis, pr["depth"], 0).astype(np.float32), radius=radius, rect=rect,
                grid=(gx, gy), width=cam.width, height=cam.height, tile=tuple(tile), proj64=pr)


def records_to_gpu(recs: list):
    """Concatenate per-view FP32 records into a Projected on the GPU."""
    from paper_2507_20239_gb300 import rasterizer as R
    cat = lambda k: np.concatenate([r[k] for r in recs], 0)
    n = sum(r["mean2d"].shape[0] for r in recs)
    co = np.zeros((n, 4), np.float32)
    co[:, :3] = cat("conic_f")
    co[:, 3] = cat("opacity")
    rgb = np.zeros((n, 4), np.float32)
    rgb[:, :3] = cat("rgb")
    rgb[:, 3] = cat("q_max")
    rect = cat("rect").astype(np.uint16).view(np.int16)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(DEV)
    return R.Projected(t(cat("mean2d")), t(co), t(rgb), t(cat("depth")), t(cat("radius").astype(np.int32)),
                       t(rect), torch.zeros(n, dtype=torch.uint8, device=DEV))


def oracle_lists(rec: dict):
    return oras.tile_lists(rec, rec["width"], rec["height"], *rec["tile"])


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


@functools.lru_cache(maxsize=None)
def scene(name: str):
    if name == "small":
        return synth.small_scene(0)
    if name == "orbit":
        return synth.orbit_scene(1)
    if name == "orbit_small":
        return synth.orbit_scene(1, n=60_000, width=320, height=212, f=320.0)
    if name == "batched_small":
        sc = synth.surface_scene(2, 40_000, 3)
        cams, tg = synth.mixed_resolution_cameras(6, seed=2)
        cams = [synth.orbit_camera(4.0, c_az, 15.0, c.width // 4, c.height // 4, c.fx / 4)
                for c, c_az in zip(cams, np.linspace(0, 2 * np.pi, 6, endpoint=False))]
        sc.cameras = cams
        rng = np.random.default_rng(5)
        sc.targets = [rng.uniform(0, 1, (3, c.height, c.width)).astype(np.float32) for c in cams]
        return sc
    raise KeyError(name)


def exact_list_check(mean2d, conic_f, q_max, radius, width, height, tile, list_tiles, list_recs,
                     chunk=200_000):
    """The FP32 tile lists of one view against the exact FP64 footprint geometry.

    For every visible record, the candidate tiles are those under its FP64 footprint
    box (half-extents from the conic, grown by a pixel), and each (tile, record) pair
    is decided by the exact box-minimum test (oracle.project.tile_hit, FP64) with the
    FP32 decision's derived margin (oracle.project.band_margin):
      must = the pair is kept with the box shrunk by delta and bound qb (1 - eps);
      may  = the pair is kept with the box grown by delta and bound qb (1 + eps).
    Asserts that every `must` pair is in the lists and every listed pair is `may`.
    list_tiles / list_recs: the listed pairs (view-local tile index, record index).
    Returns (listed, must, between) pair counts.
    """
    from oracle import project as oproj
    tw, th = tile
    gx, gy = oproj.tile_grid(width, height, tw, th)
    n = mean2d.shape[0]
    listed = np.unique(np.asarray(list_tiles, np.int64) * n + np.asarray(list_recs, np.int64))
    vis = np.nonzero(np.asarray(radius) > 0)[0]
    n_must = n_between = 0
    may_keys = []
    for c0 in range(0, vis.size, chunk):
        r = vis[c0:c0 + chunk]
        u = mean2d[r, 0].astype(np.float64)
        v = mean2d[r, 1].astype(np.float64)
        A, beta, gamma = (conic_f[r, k].astype(np.float64) for k in range(3))
        qb = q_max[r].astype(np.float64) * oproj.BIN_MARGIN
        hx = np.sqrt(qb * (1.0 / A + beta * beta / gamma))
        hy = np.sqrt(qb / gamma)
        x0 = np.clip(np.floor((u - hx - 1.0) / tw), 0, gx).astype(np.int64)
        x1 = np.clip(np.floor((u + hx + 1.0) / tw) + 1, 0, gx).astype(np.int64)
        y0 = np.clip(np.floor((v - hy - 1.0) / th), 0, gy).astype(np.int64)
        y1 = np.clip(np.floor((v + hy + 1.0) / th) + 1, 0, gy).astype(np.int64)
        w = np.maximum(x1 - x0, 0)
        cnt = w * np.maximum(y1 - y0, 0)
        j = np.repeat(np.arange(r.size), cnt)
        local = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        tx = x0[j] + local % w[j]
        ty = y0[j] + local // w[j]
        X0 = tx * tw + 0.5
        X1 = np.minimum((tx + 1) * tw, width) - 0.5
        Y0 = ty * th + 0.5
        Y1 = np.minimum((ty + 1) * th, height) - 0.5
        delta, eps = oproj.band_margin(u[j], v[j], beta[j], hx[j], hy[j], width, height)
        args = (u[j], v[j], A[j], beta[j], gamma[j])
        must = oproj.tile_hit(*args, qb[j] * (1 - eps), X0 + delta, X1 - delta, Y0 + delta, Y1 - delta)
        may = oproj.tile_hit(*args, qb[j] * (1 + eps), X0 - delta, X1 + delta, Y0 - delta, Y1 + delta)
        key = (ty * gx + tx) * n + r[j]
        mk = key[must]
        pos = np.searchsorted(listed, mk)
        found = (pos < listed.size) & (listed[np.minimum(pos, listed.size - 1)] == mk)
        assert found.all(), f"{(~found).sum()} pairs the exact test keeps are missing, e.g. " \
                            f"(tile, record) {[(int(k // n), int(k % n)) for k in mk[~found][:4]]}"
        n_must += int(must.sum())
        n_between += int((may & ~must).sum())
        may_keys.append(key[may])
    may_keys = np.unique(np.concatenate(may_keys)) if may_keys else np.zeros(0, np.int64)
    pos = np.searchsorted(may_keys, listed)
    ok = (pos < may_keys.size) & (may_keys[np.minimum(pos, max(may_keys.size - 1, 0))] == listed)
    assert ok.all(), f"{(~ok).sum()} listed pairs lie outside the exact footprint, e.g. " \
                     f"(tile, record) {[(int(k // n), int(k % n)) for k in listed[~ok][:4]]}"
    return int(listed.size), n_must, n_between


def bins_pairs(bins, n_tiles):
    """(tile, record) of every listed entry of a Bins, on the host."""
    ranges = bins.ranges.cpu().numpy().view(np.uint32).astype(np.int64)
    M = int(bins.count.item())
    vals = bins.vals[:M].cpu().numpy().view(np.uint32).astype(np.int64)
    lens = ranges[:n_tiles, 1] - ranges[:n_tiles, 0]
    tiles = np.repeat(np.arange(n_tiles, dtype=np.int64), lens)
    starts = np.repeat(ranges[:n_tiles, 0], lens)
    pos = starts + (np.arange(lens.sum()) - np.repeat(np.cumsum(lens) - lens, lens))
    return tiles, vals[pos]
