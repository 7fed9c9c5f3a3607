"""FP64 oracle of the energy-guided coarse-to-fine resolution schedule (Sec.
"Energy-aware multi-resolution", the equations for E(I), D_r, E_r and T_r).
Test infrastructure only: imported by tests/, never by the library.

Readings (the paper leaves these open):
* D_r is bilinear downscaling with anti-aliasing, taken as the separable triangle
  filter whose support widens with the scale: an output of W_r = floor(W/r + 1/2)
  columns has scale s = W / W_r, output column j samples the input at
  c_j = (j + 1/2) s - 1/2 with weights max(0, 1 - |k - c_j| / s) over the input
  columns k inside the image, normalised to sum 1 (rows likewise).
* E(I) is the magnitude of the 2D DFT of each channel (numpy's unnormalised
  forward transform); ||E(I_r)||_1 sums it over all frequencies and channels.
* E_r = ||E(D_r(I))||_1 r^2, averaged over the training images.
* T_r = Round(E_r / E_1 T_densify) with Round half up, clamped to [0, T_densify]
  and made non-increasing in r; stage r covers iterations [T_{r+1}, T_r) with
  T_{K+1} = 0.
"""
from __future__ import annotations

import math

import numpy as np


def downscaled_size(n: int, r: int) -> int:
    return max(1, int(math.floor(n / r + 0.5)))


def aa_weights(n_in: int, n_out: int) -> np.ndarray:
    """[n_out, n_in] FP64 matrix of the anti-aliased bilinear (triangle) filter."""
    s = n_in / n_out
    k = np.arange(n_in, dtype=np.float64)
    out = np.zeros((n_out, n_in))
    for j in range(n_out):
        c = (j + 0.5) * s - 0.5
        w = np.maximum(0.0, 1.0 - np.abs(k - c) / s)
        out[j] = w / w.sum()
    return out


def downscale(img: np.ndarray, r: int) -> np.ndarray:
    """D_r of a planar [C, H, W] image (FP64)."""
    img = np.asarray(img, np.float64)
    _, H, W = img.shape
    if r == 1:
        return img.copy()
    Wy = aa_weights(H, downscaled_size(H, r))
    Wx = aa_weights(W, downscaled_size(W, r))
    return np.stack([Wy @ c @ Wx.T for c in img])


def spectrum_l1(img: np.ndarray) -> float:
    """||E(I)||_1: the sum over channels and frequencies of |DFT2(I_c)|."""
    return float(sum(np.abs(np.fft.fft2(np.asarray(c, np.float64))).sum() for c in img))


def energies(images, K: int) -> np.ndarray:
    """E_r for r = 1..K (index r-1), averaged over the images."""
    E = np.zeros(K)
    for img in images:
        for r in range(1, K + 1):
            E[r - 1] += spectrum_l1(downscale(img, r)) * r * r
    return E / len(images)


def iterations(E: np.ndarray, T_densify: int) -> np.ndarray:
    """T_r for r = 1..K (index r-1) from the energies."""
    T = np.floor(E / E[0] * T_densify + 0.5).astype(np.int64)
    T = np.clip(T, 0, T_densify)
    for i in range(1, len(T)):              # non-increasing in r
        T[i] = min(T[i], T[i - 1])
    return T


def stages(T: np.ndarray) -> list:
    """[(start, end, r)] from coarsest to finest, empty stages dropped."""
    K = len(T)
    out = []
    for r in range(K, 0, -1):
        start = int(T[r]) if r < K else 0
        end = int(T[r - 1])
        if end > start:
            out.append((start, end, r))
    return out
