"""Energy-guided coarse-to-fine resolution schedule (Sec. "Energy-aware
multi-resolution") on the GPU.

For the training images I: E_r = ||E(D_r(I))||_1 r^2 (gs_downscale, gs_spectrum_l1),
averaged over the images, for r = 1..K; T_r = Round(E_r / E_1 T_densify) (half up),
clamped to [0, T_densify] and made non-increasing in r; training runs from the
coarsest scale r = K to r = 1, scale r over iterations [T_{r+1}, T_r) with
T_{K+1} = 0.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _abi
from ._abi import check
from .rasterizer import _p, _stream, lib


def downscaled_size(n: int, r: int) -> int:
    return int(lib().gs_downscaled_size(int(n), int(r)))


def downscale(image: torch.Tensor, r: int, stream=None) -> torch.Tensor:
    """D_r of a planar [C, H, W] FP32 device image."""
    img = image.contiguous()
    Cc, H, W = img.shape
    out = torch.empty(Cc, downscaled_size(H, r), downscaled_size(W, r), dtype=torch.float32, device=img.device)
    check(lib().gs_downscale(_p(img), Cc, H, W, int(r), _p(out), _stream(stream)), "gs_downscale")
    return out


def spectrum_l1(image: torch.Tensor, stream=None) -> float:
    """||E(I)||_1 of a planar [C, H, W] FP32 device image."""
    img = image.contiguous()
    Cc, H, W = img.shape
    n = lib().gs_spectrum_workspace_size(Cc, H, W)
    if n == 0:
        raise _abi.GsError(1, "gs_spectrum_workspace_size")
    ws = torch.empty(n, dtype=torch.uint8, device=img.device)
    out = torch.empty(1, dtype=torch.float64, device=img.device)
    check(lib().gs_spectrum_l1(_p(img), Cc, H, W, _p(out), _p(ws), ws.numel(), _stream(stream)), "gs_spectrum_l1")
    return float(out.item())


def energies(images, K: int, device="cuda") -> np.ndarray:
    """E_r for r = 1..K (index r-1), averaged over the images ([C, H, W] arrays)."""
    E = np.zeros(K)
    for im in images:
        t = torch.as_tensor(np.asarray(im, np.float32)).to(device)
        for r in range(1, K + 1):
            E[r - 1] += spectrum_l1(downscale(t, r) if r > 1 else t) * r * r
    return E / len(images)


def iterations(E, T_densify: int) -> np.ndarray:
    E = np.asarray(E, np.float64)
    T = np.array([min(max(int(math.floor(e / E[0] * T_densify + 0.5)), 0), T_densify) for e in E], np.int64)
    for i in range(1, len(T)):
        T[i] = min(T[i], T[i - 1])
    return T


def stages(T) -> list:
    """[(start, end, r)] from the coarsest scale to r = 1, empty scales dropped."""
    K = len(T)
    out = []
    for r in range(K, 0, -1):
        start = int(T[r]) if r < K else 0
        if int(T[r - 1]) > start:
            out.append((start, int(T[r - 1]), r))
    return out


def energy_schedule(images, K: int = 8, T_densify: int = 25000, device="cuda"):
    """(E, T, stages) of the training images."""
    E = energies(images, K, device)
    T = iterations(E, T_densify)
    return E, T, stages(T)
