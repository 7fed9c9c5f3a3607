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
