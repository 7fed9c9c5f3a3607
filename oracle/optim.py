"""Optimiser steps of the training loop (FP64) -- test infrastructure only.

Adam as in the 3DGS lineage (bias-corrected moments, eps added to sqrt(v_hat));
"sparse" Adam (the accelerated lineage the paper builds on) leaves the rows of
Gaussians not visible in the step's views untouched, moments included. Opacity
reset: every logit is lowered to at most logit(0.01) and the opacity moments are
cleared.
"""
from __future__ import annotations

import math

import numpy as np


def adam_step(p, g, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-15, visible=None):
    """One step (t >= 1) on row-major arrays [N, ...]; returns new (p, m, v) in FP64."""
    p, g, m, v = (np.asarray(a, np.float64) for a in (p, g, m, v))
    m1 = beta1 * m + (1 - beta1) * g
    v1 = beta2 * v + (1 - beta2) * g * g
    mh = m1 / (1 - beta1 ** t)
    vh = v1 / (1 - beta2 ** t)
    p1 = p - lr * mh / (np.sqrt(vh) + eps)
    if visible is None:
        return p1, m1, v1
    sel = np.asarray(visible, bool).reshape((-1,) + (1,) * (p.ndim - 1))
    return np.where(sel, p1, p), np.where(sel, m1, m), np.where(sel, v1, v)


def opacity_reset(logits, max_opacity=0.01):
    cap = math.log(max_opacity / (1 - max_opacity))
    return np.minimum(np.asarray(logits, np.float64), cap)


def position_lr(step, lr_init, lr_final, full_res_start, total):
    """Constant while training at reduced resolution, then log-linear decay from
    lr_init to lr_final over [full_res_start, total]."""
    if step <= full_res_start:
        return lr_init
    t = min(1.0, (step - full_res_start) / max(1, total - full_res_start))
    return math.exp((1 - t) * math.log(lr_init) + t * math.log(lr_final))
