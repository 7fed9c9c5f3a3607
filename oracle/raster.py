"""Tile binning, depth sort and Eq. 2 compositing (FP64) -- test infrastructure only.

Eq. 2 of the paper: C(p) = sum_i c_i sigma_i prod_{j<i} (1 - sigma_j), sigma_i =
alpha_i G_i'(p), over the depth-sorted Gaussians N_p visible at pixel p, with the
image split into tiles. The compositing here is that product formula written out
for all pixels of a tile at once (a cumulative product along the depth-sorted
list), with the rasterizer's cut-offs that the paper leaves implicit:

  * pixel (i, j) is sampled at (i + 0.5, j + 0.5); d = mean2D - p;
  * power P = -1/2 (A dx^2 + C dy^2) - B dx dy; an entry with P > 0 is skipped;
  * sigma = min(0.99, o exp(P)); an entry with sigma < 1/255 is skipped;
  * the walk stops before the first entry whose inclusion would make the
    transmittance T' = T (1 - sigma) fall below 1e-4 (that entry is excluded);
  * output = C + T_final * bg.

N_p for a pixel is the tile's list: every visible record whose footprint ellipse
(the region where alpha can reach the 1/255 floor, with the binning margin) meets
the tile's box of pixel centres, ordered by (FP32 depth bits, record index) --
"depth-sorted" and "tile-based" in the paper; the FP32 key is the precision of the
stored depth. Records carry the conic factored as (A, beta, gamma); the
compositing expands it to (A, B, C) = (A, A beta, gamma + A beta^2).
Gradients come from reverse-mode differentiation of this FP64 forward.
"""
from __future__ import annotations

import numpy as np
import torch

from .project import band_hit, BIN_MARGIN

ALPHA_MIN = 1.0 / 255.0
ALPHA_MAX = 0.99
T_MIN = 1e-4


# ----------------------------------------------------------------------------------------
# binning and sorting (integer work, bit-exact)
# ----------------------------------------------------------------------------------------
def emit_duplicates(rect: np.ndarray, tile_offset: np.ndarray, grid_x: np.ndarray):
    """One (global tile, record) pair per tile of each record's rectangle.

    rect [R,4] int (x0, y0, x1, y1) exclusive; tile_offset, grid_x [R] per record
    (the record's view). Returns (tile [M] int64, record [M] int64) in emission
    order: records ascending, tiles of a rectangle row-major.
    """
    w = np.maximum(rect[:, 2] - rect[:, 0], 0)
    h = np.maximum(rect[:, 3] - rect[:, 1], 0)
    cnt = (w * h).astype(np.int64)
    total = int(cnt.sum())
    rec = np.repeat(np.arange(rect.shape[0], dtype=np.int64), cnt)
    start = np.cumsum(cnt) - cnt
    local = np.arange(total, dtype=np.int64) - np.repeat(start, cnt)
    wr = w[rec]
    tx = rect[rec, 0] + local % wr
    ty = rect[rec, 1] + local // wr
    tile = tile_offset[rec] + ty * grid_x[rec] + tx
    return tile.astype(np.int64), rec


def depth_bits(depth_f32: np.ndarray) -> np.ndarray:
    """IEEE-754 bit pattern of FP32 depths (> 0, so unsigned order = numeric order)."""
    return np.ascontiguousarray(depth_f32, dtype=np.float32).view(np.uint32)


def tile_filter(tile, rec, mean2d, conic_f, q_max, tile_offset, grid_x, widths, heights, tile_w, tile_h):
    """Keep the (tile, record) candidates whose footprint ellipse meets the tile's
    pixel-centre box; evaluated in the records' dtype (see project.band_span)."""
    dt = mean2d.dtype.type
    lt = tile - tile_offset[rec]
    gx = grid_x[rec]
    tx, ty = lt % gx, lt // gx
    W, H = widths[rec], heights[rec]
    X0 = (tx * tile_w).astype(mean2d.dtype) + dt(0.5)
    X1 = np.minimum((tx + 1) * tile_w, W).astype(mean2d.dtype) - dt(0.5)
    Y0 = (ty * tile_h).astype(mean2d.dtype) + dt(0.5)
    Y1 = np.minimum((ty + 1) * tile_h, H).astype(mean2d.dtype) - dt(0.5)
    qb = (q_max.astype(mean2d.dtype) * dt(BIN_MARGIN))[rec]
    cf = conic_f.astype(mean2d.dtype)
    hit = band_hit(mean2d[rec, 0], mean2d[rec, 1], cf[rec, 0], cf[rec, 1], cf[rec, 2], qb, X0, X1, Y0, Y1)
    return tile[hit], rec[hit]


def bin_and_sort(rec_arrays: dict, tile_offset, grid_x, widths, heights, tile_w, tile_h, n_tiles):
    """Sorted duplicate list: keys = tile << 32 | depth bits, vals = record index,
    ordered by (tile, depth bits, record index); ranges[t] = [start, end) of tile
    t in the sorted list (start = end for an empty tile).

    rec_arrays: mean2d [R,2], conic_f [R,3], q_max [R], rect [R,4], depth [R] (FP32
    depth is the key); tile_offset, grid_x, widths, heights per record (its view).
    """
    tile, rec = emit_duplicates(rec_arrays["rect"], tile_offset, grid_x)
    tile, rec = tile_filter(tile, rec, rec_arrays["mean2d"], rec_arrays["conic_f"], rec_arrays["q_max"],
                            tile_offset, grid_x, widths, heights, tile_w, tile_h)
    bits = depth_bits(rec_arrays["depth"])[rec].astype(np.uint64)
    order = np.lexsort((rec, bits, tile))
    tile_s = tile[order]
    keys = (tile_s.astype(np.uint64) << np.uint64(32)) | bits[order]
    vals = rec[order].astype(np.uint32)
    counts = np.bincount(tile_s, minlength=n_tiles)[:n_tiles]
    end = np.cumsum(counts)
    ranges = np.stack([end - counts, end], 1).astype(np.uint32)
    return keys, vals, ranges


def tile_lists(rec_arrays: dict, width, height, tile_w=16, tile_h=16):
    """Per-tile record lists of one view as a dict {tile: int64 array}."""
    n = rec_arrays["rect"].shape[0]
    gx = (width + tile_w - 1) // tile_w
    gy = (height + tile_h - 1) // tile_h
    full = lambda x: np.full(n, x, np.int64)
    _, vals, ranges = bin_and_sort(rec_arrays, full(0), full(gx), full(width), full(height), tile_w, tile_h,
                                   gx * gy)
    return {t: vals[ranges[t, 0]:ranges[t, 1]].astype(np.int64) for t in range(gx * gy)}


# ----------------------------------------------------------------------------------------
# compositing (FP64, differentiable)
# ----------------------------------------------------------------------------------------
U32 = 2.0 ** -24                      # unit round-off of FP32 round-to-nearest
K_EXP = 0.5 / np.log(2.0)             # |k| = log2(e) / 2: G = 2^(k q), k = -log2(e) / 2
EX2_REL = 2.0 ** -22                  # ex2.approx.f32: 2 ulp of the result (PTX ISA bound)
ALPHA_MAX_F32_REL = abs(float(np.float32(ALPHA_MAX)) - ALPHA_MAX) / ALPHA_MAX
ALPHA_MIN_F32_REL = abs(float(np.float32(ALPHA_MIN)) - ALPHA_MIN) / ALPHA_MIN
T_MIN_F32_REL = abs(float(np.float32(T_MIN)) - T_MIN) / T_MIN
FLAG_SAFETY = 2.0                     # first-order bounds below, doubled


def fp32_alpha_error(dx, dy, A, beta, gamma, q, rec_dq=None, rec_do=None):
    """Bound on the relative error of an FP32 evaluation of sigma = o G (Eq. 2),
    G = exp(-q/2), q = A (dx + beta dy)^2 + gamma dy^2, from exact FP32 record values,
    with one rounding per operation (u_r = 2^-24, first order):
      dx = u - p_x, dy = v - p_y      |err| <= u_r |dx|, u_r |dy|
      t = beta dy + dx (fused)        |err| <= u_r (|t| + |beta dy| + |dx|)
      k A, k gamma (k = -log2(e)/2)   relative 2 u_r each (k and the product rounded)
      e = (kA t) t + k gamma (dy dy)  |err| <= |k| u_r (3 A t^2 + 2 A |t| (|t| + |beta dy|
                                       + |dx|) + 6 gamma dy^2 + q)
      G = 2^e                         relative ln 2 |err e| + 2^-22 (ex2.approx)
      o G                             relative + u_r; the 0.99 clamp's FP32 constant
                                      differs from 0.99 by 1e-8 relatively.
    rec_dq, rec_do (optional): first-order changes of q and absolute changes of o from
    perturbed record values (when the two sides project independently).
    Returns the bound as an array of dx's shape.
    """
    at = np.abs(dx + beta * dy)
    de = K_EXP * U32 * (3 * A * at * at + 2 * A * at * (at + np.abs(beta * dy) + np.abs(dx))
                        + 6 * gamma * dy * dy + q)
    eps = np.log(2.0) * de + EX2_REL + U32 + ALPHA_MAX_F32_REL
    if rec_dq is not None:
        eps = eps + 0.5 * rec_dq
    if rec_do is not None:
        eps = eps + rec_do
    return eps


def composite(px, py, xy, conic_f, opacity, rgb, bg, rec_delta=None):
    """Eq. 2 for P pixels over one depth-ordered list of L Gaussians.

    px, py: [P] float64 sample coordinates; xy [L,2], conic_f [L,3] = (A, beta,
    gamma), opacity [L],
    rgb [L,3] torch float64 in list order; bg [3]. Returns (color [P,3], T_final [P],
    stop [P], n_examined [P], n_contrib [P], flag [P]); stop is one past the last
    contributing list position, n_examined counts list entries looked at up to and
    including the one that triggers the cut-off.

    flag marks pixels where an FP32 evaluation of the same walk may take a different
    decision: an examined entry whose sigma lies within the FP32 error bound of
    sigma (fp32_alpha_error, times FLAG_SAFETY) of the 1/255 floor, or whose
    transmittance after it lies within the bound of the running FP32 product of
    1e-4. The product's bound after composited entries j <= k is
    rho_k = sum_j (sigma_j eps_j / (1 - sigma_j) + 2 u_r): 1 - sigma_j carries
    sigma_j's error, and 1 - sigma and T (1 - sigma) are rounded once each.
    rec_delta (optional, [L,6] absolute differences of (u, v, A, beta, gamma, o)
    between the records the two sides use) widens the bound by their first-order
    effect on q and o.
    """
    P = px.shape[0]
    L = xy.shape[0]
    dt = torch.float64
    bg = torch.as_tensor(bg, dtype=dt)
    if L == 0:
        z = np.zeros(P, np.int64)
        return (bg.expand(P, 3).clone(), torch.ones(P, dtype=dt), z, z, z, np.zeros(P, bool))
    pxt = torch.as_tensor(px, dtype=dt)[:, None]
    pyt = torch.as_tensor(py, dtype=dt)[:, None]
    dx = xy[None, :, 0] - pxt                                   # [P,L]
    dy = xy[None, :, 1] - pyt
    A = conic_f[None, :, 0]
    B = A * conic_f[None, :, 1]
    C = conic_f[None, :, 2] + B * conic_f[None, :, 1]
    power = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
    alpha = torch.clamp(opacity[None, :] * torch.exp(power), max=ALPHA_MAX)
    cand = ((power <= 0) & (alpha >= ALPHA_MIN)).detach()
    one_minus = torch.where(cand, 1.0 - alpha, torch.ones_like(alpha))
    T_after = torch.cumprod(one_minus, dim=1)
    hit = cand & (T_after < T_MIN).detach()
    idx = torch.arange(L)[None, :]
    first = torch.where(hit.any(1), hit.float().argmax(1), torch.full((P,), L))   # [P]
    active = cand & (idx < first[:, None])
    T_before = torch.cat([torch.ones(P, 1, dtype=dt), T_after[:, :-1]], 1)
    w = torch.where(active, alpha * T_before, torch.zeros_like(alpha))
    color = w @ rgb                                              # [P,3]
    T_final = torch.prod(torch.where(active, one_minus, torch.ones_like(one_minus)), dim=1)
    out = color + T_final[:, None] * bg[None, :]
    # integer diagnostics
    act = active.numpy()
    has = act.any(1)
    last = np.where(has, L - 1 - np.argmax(act[:, ::-1], axis=1), -1)
    stop = (last + 1).astype(np.int64)
    first_np = first.numpy()
    n_exam = np.minimum(first_np + 1, L).astype(np.int64)
    n_contrib = act.sum(1).astype(np.int64)
    # straddle flags on examined entries, from the derived FP32 error bounds
    exam = idx.numpy() < n_exam[:, None]
    a_np = alpha.detach().numpy()
    p_np = power.detach().numpy()
    dxn, dyn = dx.detach().numpy(), dy.detach().numpy()
    cf = conic_f.detach().numpy()
    An, bn, gn = cf[None, :, 0], cf[None, :, 1], cf[None, :, 2]
    q = -2.0 * p_np
    rec_dq = rec_do = None
    if rec_delta is not None:
        d = np.asarray(rec_delta, np.float64)[None]            # [1,L,6]
        tt = dxn + bn * dyn
        rec_dq = (np.abs(2 * An * tt) * d[..., 0] + np.abs(2 * An * tt * bn + 2 * gn * dyn) * d[..., 1]
                  + tt * tt * d[..., 2] + np.abs(2 * An * tt * dyn) * d[..., 3] + dyn * dyn * d[..., 4])
        op = opacity.detach().numpy()[None]
        rec_do = d[..., 5] / np.maximum(op, 1e-30)
    eps_a = fp32_alpha_error(dxn, dyn, An, bn, gn, q, rec_dq, rec_do)
    a_raw = opacity.detach().numpy()[None] * np.exp(p_np)     # sigma before the 0.99 clamp
    fa = exam & (p_np <= 0) & (np.abs(a_raw / ALPHA_MIN - 1.0) < FLAG_SAFETY * eps_a + ALPHA_MIN_F32_REL)
    candn = cand.numpy()
    term = np.where(candn, a_np * eps_a / np.maximum(1.0 - a_np, 1e-300) + 2 * U32, 0.0)
    rho = np.cumsum(term, axis=1)
    Tn = T_after.detach().numpy()
    ft = exam & candn & (np.abs(Tn / T_MIN - 1.0) < FLAG_SAFETY * rho + T_MIN_F32_REL)
    flag = fa.any(1) | ft.any(1)
    return out, T_final, stop, n_exam, n_contrib, flag


def tile_pixels(t, grid_x, tile_w, tile_h, width, height):
    tx, ty = t % grid_x, t // grid_x
    xs = np.arange(tx * tile_w, min((tx + 1) * tile_w, width))
    ys = np.arange(ty * tile_h, min((ty + 1) * tile_h, height))
    X, Y = np.meshgrid(xs, ys)
    return X.ravel(), Y.ravel()


def rasterize(rec, lists, width, height, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0),
              tiles=None, d_image=None, rec_delta=None):
    """Render one view from projected records.

    rec: dict of torch float64 tensors mean2d [N,2], conic_f [N,3], opacity [N],
    rgb [N,3] (leaves that may require grad). lists: {tile: record indices in
    depth order} (see tile_lists). tiles: subset of tiles to render (default all).
    If d_image [3,H,W] is given, the vector-Jacobian product sum(image * d_image)
    is back-propagated tile by tile into the leaves' .grad. rec_delta [N,6]: see
    composite (widens the straddle flags for records the other side computed itself).
    Returns dict of numpy arrays image [3,H,W], T_final, stop, n_examined,
    n_contrib, flag [H,W] (only the rendered tiles are filled).
    """
    gx = (width + tile_w - 1) // tile_w
    gy = (height + tile_h - 1) // tile_h
    image = np.zeros((3, height, width))
    T_final = np.ones((height, width))
    stop = np.zeros((height, width), np.int64)
    n_exam = np.zeros((height, width), np.int64)
    n_contrib = np.zeros((height, width), np.int64)
    flag = np.zeros((height, width), bool)
    if tiles is None:
        tiles = range(gx * gy)
    dimg = None if d_image is None else torch.as_tensor(np.asarray(d_image, np.float64))
    for t in tiles:
        X, Y = tile_pixels(t, gx, tile_w, tile_h, width, height)
        if X.size == 0:
            continue
        ids = torch.as_tensor(lists.get(t, np.zeros(0, np.int64)))
        out, Tf, st, ne, nc, fl = composite(
            X + 0.5, Y + 0.5, rec["mean2d"][ids], rec["conic_f"][ids], rec["opacity"][ids],
            rec["rgb"][ids], bg, None if rec_delta is None else np.asarray(rec_delta)[ids.numpy()])
        if dimg is not None and ids.numel() > 0:
            g = dimg[:, Y, X].T                                   # [P,3]
            s = (out * g).sum()
            if s.requires_grad:
                s.backward()
        image[:, Y, X] = out.detach().numpy().T
        T_final[Y, X] = Tf.detach().numpy()
        stop[Y, X] = st
        n_exam[Y, X] = ne
        n_contrib[Y, X] = nc
        flag[Y, X] = fl
    return dict(image=image, T_final=T_final, stop=stop, n_examined=n_exam,
                n_contrib=n_contrib, flag=flag)


def records_to_torch(mean2d, conic_f, opacity, rgb, requires_grad=False):
    mk = lambda a: torch.tensor(np.asarray(a, np.float64), requires_grad=requires_grad)
    return dict(mean2d=mk(mean2d), conic_f=mk(conic_f), opacity=mk(opacity), rgb=mk(rgb))


def raster_vjp(mean2d, conic_f, opacity, rgb, lists, width, height, d_image, tile_w=16,
               tile_h=16, bg=(0.0, 0.0, 0.0), tiles=None, rec_delta=None):
    """Gradients of sum(image * d_image) w.r.t. the projected records (FP64).

    Returns (render dict, grads dict with d_mean2d [N,2], d_conic [N,3] (w.r.t.
    (A, beta, gamma)), d_opacity [N], d_rgb [N,3])."""
    rec = records_to_torch(mean2d, conic_f, opacity, rgb, requires_grad=True)
    out = rasterize(rec, lists, width, height, tile_w, tile_h, bg, tiles, d_image, rec_delta)
    g = {}
    for k, name in (("mean2d", "d_mean2d"), ("conic_f", "d_conic"), ("opacity", "d_opacity"),
                    ("rgb", "d_rgb")):
        gr = rec[k].grad
        g[name] = np.zeros(rec[k].shape) if gr is None else gr.numpy()
    return out, g
