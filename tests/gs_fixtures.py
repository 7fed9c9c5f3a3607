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
