"""Densification bookkeeping -- test infrastructure only.

Follows the paper's densification rule (Sec. "Preliminary", last paragraph): the
norm of each Gaussian's average position gradient is compared with a threshold;
above it the Gaussian is split when its largest scale exceeds a scale threshold
and cloned otherwise. Global-to-local densification (Sec. "Global-to-local
framework") disables clone in the first phase. Adaptive opacity pruning (Sec.
"Adaptive Opacity Pruning"): tau = min(alpha_sorted[floor(N p)], tau_u).

All predicates act on the FP32 tensors they are given and are evaluated in
FP32 with one rounding per operation (numpy float32 scalar semantics), so the
selections are exact. Readings where the paper is silent:
  * statistic per view and record with radius > 0: n = sqrt(gx^2 + gy^2) with
    (gx, gy) = (dL/du * W/2, dL/dv * H/2), the mean2D gradient in NDC units;
    accum += n, count += 1, views in order;
  * avg = accum / count (0 when count = 0); "exceeds" is strict (>);
  * big = max_k log_scale_k > thr_s (thr_s = FP32 of log(0.01 * extent));
  * modes: ADAPTIVE (split if big, clone otherwise), SPLIT_ONLY (the first,
    global phase: clone disabled, big Gaussians still split), ALL_SPLIT and
    ALL_CLONE (every selected Gaussian split / cloned, the single-operation
    variants of the split-clone analysis);
  * pruning acts on the post-densification set; children and clones inherit
    the parent's opacity, so a record is kept iff its logit >= tau_logit;
    tau is applied in logit space (sigmoid is increasing): tau_logit =
    min(k-th smallest logit of the post-densification multiset, FP32 logit(tau_u)),
    k = min(floor(N' p), N' - 1), 0-based;
  * output order: survivors in original order, then clones in parent order,
    then split children in parent order (child 0 then child 1); split parents
    are removed; 2 children with log-scale s - FP32(log 1.6);
  * child mean = mu + R(q) (exp(s) * z), z ~ N(0, I) by Box-Muller from one
    Philox4x32-10 block per child (Salmon et al., SC'11), counter =
    (parent, 0, event, child), key = (seed lo, seed hi).
"""
from __future__ import annotations

import math

import numpy as np

from .project import quat_to_rotmat

ADAPTIVE, SPLIT_ONLY, ALL_SPLIT, ALL_CLONE = 0, 1, 2, 3
f32 = np.float32


def accumulate_stats(d_mean2d_views, radius_views, sizes, accum=None, count=None):
    """accum/count update from per-view record gradients.

    d_mean2d_views: list of [N,2] float32 pixel-space gradients; radius_views:
    list of [N] ints; sizes: list of (W, H). Returns updated float32 accum and
    int32 count (new arrays)."""
    n = d_mean2d_views[0].shape[0]
    acc = np.zeros(n, f32) if accum is None else np.array(accum, f32)
    cnt = np.zeros(n, np.int32) if count is None else np.array(count, np.int32)
    for g, r, (W, H) in zip(d_mean2d_views, radius_views, sizes):
        g = np.asarray(g, f32)
        gx = g[:, 0] * f32(W * 0.5)
        gy = g[:, 1] * f32(H * 0.5)
        nrm = np.sqrt(gx * gx + gy * gy)              # each op one FP32 rounding
        vis = np.asarray(r) > 0
        acc = np.where(vis, acc + nrm, acc).astype(f32)
        cnt = cnt + vis.astype(np.int32)
    return acc, cnt


def select(accum, count, log_scales, mode, grad_thr=f32(2e-4), scale_thr=None):
    """(split, clone) boolean masks."""
    accum = np.asarray(accum, f32)
    count = np.asarray(count, np.int32)
    cf = count.astype(f32)
    avg = np.where(count > 0, accum / np.where(count > 0, cf, f32(1)), f32(0)).astype(f32)
    ok = avg > f32(grad_thr)
    big = np.max(np.asarray(log_scales, f32), axis=1) > f32(scale_thr)
    if mode == ADAPTIVE:
        return ok & big, ok & ~big
    if mode == SPLIT_ONLY:
        return ok & big, np.zeros_like(ok)
    if mode == ALL_SPLIT:
        return ok, np.zeros_like(ok)
    if mode == ALL_CLONE:
        return np.zeros_like(ok), ok
    raise ValueError(mode)


def logit_threshold(tau: float) -> np.float32:
    return f32(math.log(tau / (1.0 - tau)))


def kth_smallest_weighted(values_f32, weights, k):
    """k-th smallest (0-based) of the multiset where values[i] occurs weights[i] times."""
    order = np.argsort(np.asarray(values_f32, f32), kind="stable")
    cum = np.cumsum(np.asarray(weights, np.int64)[order])
    pos = int(np.searchsorted(cum, k, side="right"))
    return f32(np.asarray(values_f32, f32)[order[pos]])


def prune_threshold(opacity_logits, split, clone, fixed_tau=None, p=None, tau_u=None):
    """tau in logit space, on the post-densification multiset (see module doc)."""
    if fixed_tau is not None:
        return logit_threshold(fixed_tau)
    mult = 1 + (np.asarray(split) | np.asarray(clone)).astype(np.int64)
    n_post = int(mult.sum())
    k = min(int(math.floor(n_post * p)), n_post - 1)
    kth = kth_smallest_weighted(opacity_logits, mult, k)
    return min(kth, logit_threshold(tau_u))


# ----------------------------------------------------------------------------------------
# Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
# SC'11): 10 rounds of two 32x32->64 multiplications, key bumped by the Weyl constants.
# ----------------------------------------------------------------------------------------
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85
MASK32 = 0xFFFFFFFF


def philox4x32_10(counter, key):
    c0, c1, c2, c3 = (int(x) & MASK32 for x in counter)
    k0, k1 = (int(x) & MASK32 for x in key)
    for r in range(10):
        if r > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def child_normals(seed: int, event: int, parent: int, child: int):
    """Three N(0,1) draws for one split child (FP64 Box-Muller)."""
    x = philox4x32_10((parent & MASK32, (parent >> 32) & MASK32, event, child),
                      (seed & MASK32, (seed >> 32) & MASK32))
    u = [((xi >> 8) + 0.5) * 2.0 ** -24 for xi in x]        # in (0, 1), exact in FP32 too
    r0 = math.sqrt(-2.0 * math.log(u[0]))
    r1 = math.sqrt(-2.0 * math.log(u[2]))
    return (r0 * math.cos(2.0 * math.pi * u[1]), r0 * math.sin(2.0 * math.pi * u[1]),
            r1 * math.cos(2.0 * math.pi * u[3]))


def apply(params: dict, split, clone, tau_logit, seed: int, event: int, extra: dict = None,
          provenance: dict = None):
    """Densify + prune. Returns (new params dict, new extra dict, index dict).

    params: means, log_scales, quats, opacity_logits, sh (float32). extra: other
    per-Gaussian float arrays (e.g. optimiser moments): survivors keep their rows,
    new rows (clones, children) are zero. Child means are FP64 here.
    provenance (optional): {origin, splits, clones} per Gaussian, for the split/clone
    analysis of Sec. "Global-to-local framework": every output row carries its
    parent's origin; the copy a clone adds counts one more clone, both children of
    a split one more split; survivors keep theirs. Returned as index["provenance"].
    """
    import torch
    split = np.asarray(split, bool)
    clone = np.asarray(clone, bool)
    logit = np.asarray(params["opacity_logits"], f32)
    keep = ~(logit < f32(tau_logit))
    surv = np.nonzero(keep & ~split)[0]
    clo = np.nonzero(keep & clone)[0]
    spl = np.nonzero(keep & split)[0]
    src = np.concatenate([surv, clo, np.repeat(spl, 2)])
    n_new = len(clo) + 2 * len(spl)
    out = {}
    for k in ("log_scales", "quats", "opacity_logits", "sh"):
        out[k] = np.asarray(params[k])[src].copy()
    means = np.asarray(params["means"], np.float64)[src].copy()
    base = len(surv) + len(clo)
    if len(spl):
        ls = np.asarray(params["log_scales"], f32)[spl]
        out["log_scales"][base:] = np.repeat(ls - f32(math.log(1.6)), 2, axis=0)
        q = torch.as_tensor(np.asarray(params["quats"], np.float64)[spl])
        Rm = quat_to_rotmat(q).numpy()
        s = np.exp(ls.astype(np.float64))
        for j, g in enumerate(spl):
            for c in range(2):
                z = np.array(child_normals(seed, event, int(g), c))
                means[base + 2 * j + c] = means[base + 2 * j + c] + Rm[j] @ (s[j] * z)
    out["means"] = means
    ex = {}
    for k, a in (extra or {}).items():
        a = np.asarray(a)
        e = a[src].copy()
        e[len(surv):] = 0
        ex[k] = e
    idx = dict(survivors=surv, clones=clo, splits=spl, source=src, n_new=n_new)
    if provenance is not None:
        pr = {k: np.asarray(provenance[k], np.int64)[src].copy() for k in ("origin", "splits", "clones")}
        pr["clones"][len(surv):len(surv) + len(clo)] += 1
        pr["splits"][len(surv) + len(clo):] += 1
        idx["provenance"] = {k: v.astype(np.int32) for k, v in pr.items()}
    return out, ex, idx
