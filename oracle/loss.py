"""L1 photometric loss (FP64) -- test infrastructure only.

The L1 part of Eq. 3, ||I - I_hat||_1, read as the mean over the H*W*3 values of
one view (the paper does not fix the normalisation); for several views the loss
is the sum of the per-view means. The gradient at I == I_hat is taken as 0.
"""
from __future__ import annotations

import numpy as np


def l1_loss_grad(image: np.ndarray, target: np.ndarray):
    """Return (loss, d_loss/d_image) for one view; both arrays are [3, H, W]."""
    diff = np.asarray(image, np.float64) - np.asarray(target, np.float64)
    n = diff.size
    return float(np.abs(diff).sum() / n), np.sign(diff) / n


# ----------------------------------------------------------------------------------------
# D-SSIM term of Eq. 3 (FP64). Readings (the paper names the term, not its window):
# the 3DGS lineage's SSIM -- per channel, an 11 x 11 Gaussian window (sigma 1.5,
# normalised), zero padding to the image size, C1 = 0.01^2, C2 = 0.03^2 (data range 1),
# averaged over the 3 H W values; D-SSIM = 1 - SSIM; the total loss is
# (1 - lambda) L1 + lambda D-SSIM with lambda = 0.2, the L1 part as above.
SSIM_WINDOW, SSIM_SIGMA = 11, 1.5
SSIM_C1, SSIM_C2 = 0.01 ** 2, 0.03 ** 2


def gaussian_window(size=SSIM_WINDOW, sigma=SSIM_SIGMA) -> np.ndarray:
    x = np.arange(size, dtype=np.float64) - (size - 1) / 2
    g = np.exp(-x * x / (2 * sigma * sigma))
    return g / g.sum()


def ssim_map(image, target):
    """Per-pixel SSIM [3, H, W] as a torch FP64 tensor (differentiable in image)."""
    import torch
    import torch.nn.functional as F
    x = image if isinstance(image, torch.Tensor) else torch.as_tensor(np.asarray(image, np.float64))
    y = torch.as_tensor(np.asarray(target, np.float64))
    g = torch.as_tensor(gaussian_window())
    k = (g[:, None] * g[None, :])[None, None].expand(x.shape[0], 1, SSIM_WINDOW, SSIM_WINDOW).contiguous()
    pad = SSIM_WINDOW // 2
    blur = lambda a: F.conv2d(a[None], k, padding=pad, groups=x.shape[0])[0]
    mx, my = blur(x), blur(y)
    sxx, syy, sxy = blur(x * x) - mx * mx, blur(y * y) - my * my, blur(x * y) - mx * my
    return ((2 * mx * my + SSIM_C1) * (2 * sxy + SSIM_C2)) / ((mx * mx + my * my + SSIM_C1) * (sxx + syy + SSIM_C2))


def photometric_loss_grad(image: np.ndarray, target: np.ndarray, lam: float = 0.2):
    """Return (loss, d_loss/d_image) of (1 - lam) L1 + lam (1 - SSIM) for one view."""
    import torch
    x = torch.tensor(np.asarray(image, np.float64), requires_grad=True)
    ssim = ssim_map(x, target).mean()
    (lam * (1.0 - ssim)).backward()
    l1, g1 = l1_loss_grad(image, target)
    return float((1 - lam) * l1 + lam * (1.0 - float(ssim))), (1 - lam) * g1 + x.grad.numpy()
