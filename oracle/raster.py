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
def composite(px, py, xy, conic_f, opacity, rgb, bg, flag_tol_alpha=5e-6, flag_tol_T=1e-3):
    """Eq. 2 for P pixels over one depth-ordered list of L Gaussians.

    px, py: [P] float64 sample coordinates; xy [L,2], conic_f [L,3] = (A, beta,
    gamma), opacity [L],
    rgb [L,3] torch float64 in list order; bg [3]. Returns (color [P,3], T_final [P],
    stop [P], n_examined [P], n_contrib [P], flag [P]); stop is one past the last
    contributing list position, n_examined counts list entries looked at up to and
    including the one that triggers the cut-off, flag marks pixels where a
    cut-off decision lies within the relative tolerances of its threshold.
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
    # straddle flags on examined entries
    exam = idx.numpy() < n_exam[:, None]
    a_np = alpha.detach().numpy()
    p_np = power.detach().numpy()
    fa = exam & (p_np <= 0) & (np.abs(a_np / ALPHA_MIN - 1.0) < flag_tol_alpha)
    Tn = T_after.detach().numpy()
    ft = exam & cand.numpy() & (np.abs(Tn / T_MIN - 1.0) < flag_tol_T)
    flag = fa.any(1) | ft.any(1)
    return out, T_final, stop, n_exam, n_contrib, flag


def tile_pixels(t, grid_x, tile_w, tile_h, width, height):
    tx, ty = t % grid_x, t // grid_x
    xs = np.arange(tx * tile_w, min((tx + 1) * tile_w, width))
    ys = np.arange(ty * tile_h, min((ty + 1) * tile_h, height))
    X, Y = np.meshgrid(xs, ys)
    return X.ravel(), Y.ravel()


def rasterize(rec, lists, width, height, tile_w=16, tile_h=16, bg=(0.0, 0.0, 0.0),
              tiles=None, d_image=None):
    """Render one view from projected records.

    rec: dict of torch float64 tensors mean2d [N,2], conic_f [N,3], opacity [N],
    rgb [N,3] (leaves that may require grad). lists: {tile: record indices in
    depth order} (see tile_lists). tiles: subset of tiles to render (default all).
    If d_image [3,H,W] is given, the vector-Jacobian product sum(image * d_image)
    is back-propagated tile by tile into the leaves' .grad.
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
            rec["rgb"][ids], bg)
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
               tile_h=16, bg=(0.0, 0.0, 0.0), tiles=None):
    """Gradients of sum(image * d_image) w.r.t. the projected records (FP64).

    Returns (render dict, grads dict with d_mean2d [N,2], d_conic [N,3] (w.r.t.
    (A, beta, gamma)), d_opacity [N], d_rgb [N,3])."""
    rec = records_to_torch(mean2d, conic_f, opacity, rgb, requires_grad=True)
    out = rasterize(rec, lists, width, height, tile_w, tile_h, bg, tiles, d_image)
    g = {}
    for k, name in (("mean2d", "d_mean2d"), ("conic_f", "d_conic"), ("opacity", "d_opacity"),
                    ("rgb", "d_rgb")):
        gr = rec[k].grad
        g[name] = np.zeros(rec[k].shape) if gr is None else gr.numpy()
    return out, g
