"""Autotuner of the training step's knobs for one batch of views.

For a given scene size and set of view resolutions it times the whole step
(TrainStep, graph-replayed) for every candidate StepConfig -- tile shape, the
low tile-id bits the binning sorts while emitting, the backward's staging
depth, the per-pixel or per-splat backward, and the forward as one CTA per tile or
as a persistent grid claiming (tile, block) units -- and keeps the fastest. None of the knobs changes the rendered images
(every candidate's images are compared with the first one's); the gradients agree
up to summation order. Results are cached per (device, Gaussians, SH degree, view
sizes, candidates) for the life of the process.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field
from typing import Callable, Optional, Sequence

import torch

from .rasterizer import lib
from .step import StepConfig, TrainStep

TILES = ((16, 16), (8, 8), (16, 32))


def default_candidates(tiles: Sequence = TILES, fused_bits: Sequence = (0, 8),
                       stage_depths: Sequence = (0, 1), splat: bool = True, queue: bool = True) -> list:
    """Every (tile, fused bits) pair with each staging depth of the per-pixel
    backward and, if splat, once with the per-splat backward; with queue, the
    per-splat candidates also with the forward as a persistent (tile, block) queue."""
    out = []
    for t, f in itertools.product(tiles, fused_bits):
        if not lib().gs_tile_supported(int(t[0]), int(t[1])):
            continue
        tile = (int(t[0]), int(t[1]))
        for s in stage_depths:
            out.append(StepConfig(tile=tile, sort_fused_bits=int(f), stage_depth=int(s)))
        if splat:
            out.append(StepConfig(tile=tile, sort_fused_bits=int(f), backward="splat"))
            if queue:
                out.append(StepConfig(tile=tile, sort_fused_bits=int(f), backward="splat", queue=True))
    return out


@dataclass
class TuneResult:
    best: StepConfig
    best_ms: float
    table: list = field(default_factory=list)     # [(label, ms or None, note)]
    images_identical: bool = True

    def as_dict(self) -> dict:
        return {"best": self.best.label(), "best_ms": round(self.best_ms, 4),
                "candidates": {lbl: (None if ms is None else round(ms, 4)) for lbl, ms, _ in self.table},
                "skipped": {lbl: note for lbl, ms, note in self.table if ms is None},
                "images_identical": self.images_identical}


def time_step(step: TrainStep, reps: int = 5, warmup: int = 2) -> float:
    """ms per step of the graph-replayed step (CUDA events on the current stream)."""
    g = step.capture()
    for _ in range(warmup):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _fits(cfg: StepConfig, cameras) -> bool:
    """A fused-bit override must not exceed the frame's tile-id width."""
    tw, th = cfg.tile
    n_tiles = sum(((int(c.width) + tw - 1) // tw) * ((int(c.height) + th - 1) // th) for c in cameras)
    bits = max(1, (max(n_tiles - 1, 0)).bit_length())
    return cfg.sort_fused_bits == 0 or cfg.sort_fused_bits <= bits


_cache: dict = {}


def select(candidates: Sequence[StepConfig], measure: Callable[[StepConfig], Optional[float]]) -> tuple:
    """The fastest candidate by measure(cfg) (ms, or None if the candidate cannot
    run); ties keep the earlier candidate. Returns (best, best_ms, table)."""
    best, best_ms, table = None, float("inf"), []
    for cfg in candidates:
        try:
            ms = measure(cfg)
            note = "" if ms is not None else "not applicable"
        except RuntimeError as e:          # e.g. a capacity or argument error from the library
            ms, note = None, str(e).splitlines()[0][:120]
        table.append((cfg.label(), ms, note))
        if ms is not None and ms < best_ms:
            best, best_ms = cfg, ms
    if best is None:
        raise RuntimeError("autotune: no candidate ran")
    return best, best_ms, table


def autotune(params: dict, sh_degree: int, cameras, target_images, candidates: Sequence[StepConfig] = None,
             reps: int = 5, device="cuda") -> TuneResult:
    candidates = list(candidates) if candidates is not None else default_candidates()
    key = (torch.cuda.get_device_name(torch.device(device)), int(params["means"].shape[0]), int(sh_degree),
           tuple((int(c.width), int(c.height)) for c in cameras), tuple(c.label() for c in candidates))
    if key in _cache:
        return _cache[key]
    ref_image = [None]
    identical = [True]

    def measure(cfg: StepConfig):
        if not _fits(cfg, cameras):
            return None
        step = TrainStep(params, sh_degree, cameras, target_images, cfg, device=device)
        ms = time_step(step, reps=reps)
        if step.error() != 0:
            raise RuntimeError("duplicate capacity exceeded")
        img = step.image.clone()
        if ref_image[0] is None:
            ref_image[0] = img
        elif not torch.equal(img, ref_image[0]):
            identical[0] = False
        del step
        return ms

    best, best_ms, table = select(candidates, measure)
    res = TuneResult(best, best_ms, table, identical[0])
    _cache[key] = res
    return res
