"""EWA projection of 3D Gaussians and SH colour (FP64) -- test infrastructure only.

Follows Sec. "Preliminary" of the paper: Eq. 1 (the Gaussian with covariance
Sigma = R S S^T R^T), the affine (Jacobian) projection Sigma' = J W Sigma W^T J^T,
and the SH-evaluated colour c_i of Eq. 2. Readings where the paper is silent:
  * activations: R from the normalised quaternion (w, x, y, z), S = diag(exp s),
    opacity = sigmoid(logit);
  * near-plane cull at t_z <= near (0.2);
  * J is evaluated at the camera-space mean with t_x/t_z, t_y/t_z clamped to
    +-1.3 * (W/2)/f_x, +-1.3 * (H/2)/f_y (no gradient through a clamped ratio);
  * a 0.3 px^2 low-pass dilation on the diagonal: Sigma'' = Sigma' + 0.3 I =
    [[a, b], [b, c]]; cull when det = ac - b^2 <= 0;
  * the exponent of Eq. 1 in screen space, -1/2 d^T Sigma''^-1 d, is carried in
    the factored form -1/2 (A (dx + beta dy)^2 + gamma dy^2) with A = c/det,
    beta = -b/c, gamma = 1/c (an exact re-parametrisation of the conic);
  * footprint: alpha = min(0.99, o G) reaches the 1/255 floor only where
    d^T Sigma''^-1 d <= q_max = 2 ln(255 o); Gaussians with o < 1/255 are culled; the
    tile rectangle covers the axis-aligned box of that ellipse, half-extents
    sqrt(q_max a), sqrt(q_max c) (enlarged by the binning margin), and "radius" is
    the larger half-extent rounded up (the 3-sigma square box of the 3DGS lineage
    is not used: it drops pixels the alpha floor keeps and keeps tiles it drops);
  * mean2D u = f_x t_x / t_z + c_x (pixel (i, j) covers [i, i+1) x [j, j+1));
  * colour = sum_k sh_k Y_k(dir) + 0.5 per channel, clamped at 0, with dir the
    unit vector from the camera centre to the mean.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .sh import sh_basis, num_coeffs

NEAR = 0.2
DILATION = 0.3
FOV_CLAMP = 1.3
ALPHA_MIN = 1.0 / 255.0
# Tiles are kept when their pixel-centre box meets the ellipse q <= q_max scaled by
# this factor: a margin that keeps the tile test conservative against the per-pixel
# alpha test's rounding.
BIN_MARGIN = 1.002


def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix of the normalised quaternion q = (w, x, y, z); [N,4] -> [N,3,3]."""
    q = q / torch.linalg.vector_norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    rows = [
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ]
    return torch.stack(rows, -2)


def covariance_3d(log_scales: torch.Tensor, quats: torch.Tensor) -> torch.Tensor:
    """Sigma = R S S^T R^T with S = diag(exp(log_scales)); [N,3,3]."""
    M = quat_to_rotmat(quats) * torch.exp(log_scales)[:, None, :]   # R S
    return M @ M.transpose(-1, -2)


def tile_grid(width: int, height: int, tile_w: int, tile_h: int):
    return (width + tile_w - 1) // tile_w, (height + tile_h - 1) // tile_h


def tile_rect(mean2d: np.ndarray, half: np.ndarray, tile_w: int, tile_h: int,
              grid_x: int, grid_y: int) -> np.ndarray:
    """Tile rectangle [x0, y0, x1, y1) covering the box mean2d +- half (half [N,2]).

    x0 = clamp(floor((u - hx) / tw), 0, gx), x1 = clamp(floor((u + hx) / tw) + 1, 0, gx),
    likewise for y, evaluated in mean2d's own dtype (each subtraction/addition and
    division one rounded operation of that precision). Rows with a negative
    half-extent are empty.
    """
    dt = mean2d.dtype.type
    u, v = mean2d[:, 0], mean2d[:, 1]
    hx, hy = half[:, 0].astype(mean2d.dtype), half[:, 1].astype(mean2d.dtype)
    tw, th = dt(tile_w), dt(tile_h)
    x0 = np.floor((u - hx) / tw)
    y0 = np.floor((v - hy) / th)
    x1 = np.floor((u + hx) / tw) + 1
    y1 = np.floor((v + hy) / th) + 1
    rect = np.stack([np.clip(x0, 0, grid_x), np.clip(y0, 0, grid_y),
                     np.clip(x1, 0, grid_x), np.clip(y1, 0, grid_y)], 1).astype(np.int64)
    rect[(half[:, 0] < 0) | (half[:, 1] < 0)] = 0
    return rect


def footprint_half(conic_f: np.ndarray, q_max: np.ndarray) -> np.ndarray:
    """Half-extents (sqrt(qb Sigma''_xx), sqrt(qb Sigma''_yy)) of the footprint ellipse
    from the factored conic: Sigma''_xx = 1/A + beta^2/gamma, Sigma''_yy = 1/gamma."""
    A, b, g = conic_f[:, 0], conic_f[:, 1], conic_f[:, 2]
    qb = q_max * BIN_MARGIN
    return np.stack([np.sqrt(qb * (1.0 / A + b * b / g)), np.sqrt(qb / g)], 1)


def box_min_q(u, v, conic, X0, X1, Y0, Y1):
    """Minimum over the box [X0, X1] x [Y0, Y1] of the screen-space quadratic form of
    Eq. 1, q(p) = d^T Sigma''^-1 d with d = mean - p, in FP64.

    conic = (a, b, c), the entries of Sigma''^-1 = [[a, b], [b, c]] (positive
    definite), so q = a dx^2 + 2 b dx dy + c dy^2. Plain convex geometry: if the mean
    lies in the box the minimum is 0; otherwise it lies on the box's boundary, and on
    each edge q is a 1-D quadratic whose unconstrained minimiser (dx = -b dy / a on
    a horizontal edge, dy = -b dx / c on a vertical one) is clamped to the edge.
    Every input is promoted to float64; arrays broadcast elementwise.
    """
    f = lambda x: np.asarray(x, np.float64)
    u, v, X0, X1, Y0, Y1 = map(f, (u, v, X0, X1, Y0, Y1))
    a, b, c = (f(x) for x in conic)
    # d = mean - p ranges over [u - X1, u - X0] x [v - Y1, v - Y0]
    dx_lo, dx_hi = u - X1, u - X0
    dy_lo, dy_hi = v - Y1, v - Y0

    def q(dx, dy):
        return a * dx * dx + 2.0 * b * dx * dy + c * dy * dy

    with np.errstate(invalid="ignore", divide="ignore"):
        best = np.full(np.broadcast(u, a, X0, Y0).shape, np.inf)
        for dy in (dy_lo, dy_hi):                     # horizontal edges
            dx = np.clip(-b * dy / a, dx_lo, dx_hi)
            best = np.minimum(best, q(dx, dy))
        for dx in (dx_lo, dx_hi):                     # vertical edges
            dy = np.clip(-b * dx / c, dy_lo, dy_hi)
            best = np.minimum(best, q(dx, dy))
    inside = (dx_lo <= 0) & (dx_hi >= 0) & (dy_lo <= 0) & (dy_hi >= 0)
    return np.where(inside, 0.0, best)


def expand_conic(A, beta, gamma):
    """(a, b, c) of Sigma''^-1 from the factored record conic (A, beta, gamma), FP64:
    A (dx + beta dy)^2 + gamma dy^2 = A dx^2 + 2 A beta dx dy + (gamma + A beta^2) dy^2."""
    A, beta, gamma = (np.asarray(x, np.float64) for x in (A, beta, gamma))
    return A, A * beta, gamma + A * beta * beta


def tile_hit(u, v, A, beta, gamma, qb, X0, X1, Y0, Y1):
    """True where the footprint ellipse q <= qb (the region where alpha can reach the
    1/255 floor, R9) meets the box of pixel centres [X0, X1] x [Y0, Y1]: the box
    minimum of q (box_min_q) against qb, in FP64. This is the reference test; the
    binning's FP32 decision procedure is band_span / band_hit below."""
    return box_min_q(u, v, expand_conic(A, beta, gamma), X0, X1, Y0, Y1) <= np.asarray(qb, np.float64)


def band_span(u, v, A, beta, gamma, qb, Y0, Y1):
    """x-extent [xl, xr] of the ellipse A (dx + beta dy)^2 + gamma dy^2 <= qb,
    d = mean - p, over the band of pixel centres Y0 <= y <= Y1.

    At fixed dy the ellipse covers x = u + beta dy +- sqrt((qb - gamma dy^2) / A).
    The right end is concave in dy with its maximum at the ellipse's rightmost
    point, dy_r = beta sqrt(qb A / (gamma (A beta^2 + gamma))) (where the conic's
    x-extreme dx = -(Sigma''_xx qb)^(1/2) sits, dy = -(B / C) dx), and the left end
    is convex with its minimum at -dy_r; over the band each end is therefore taken
    at the extreme clamped into [v - Y1, v - Y0]. A box [X0, X1] x [Y0, Y1] meets the
    ellipse exactly when ok and X1 >= xl and X0 <= xr and xl <= xr (band_hit).

    This is the decision procedure R9 fixes for the binning: evaluated in FP32 with
    one rounded operation each (dy_r and 1/A formed once per record; fmax/fmin
    ignore a NaN operand like C's), it defines the FP32 tile lists whose keys must
    match bit-exactly. Whether those lists are right is checked against the exact
    geometry instead: in FP64 it agrees with tile_hit, and in FP32 it stays within
    band_margin of it (both pinned in the tests).
    Returns (ok, xl, xr); ok is False where the band misses the ellipse.
    """
    dt = np.result_type(u, A)
    zero = dt.type(0)
    ab = A * beta
    den = ab * beta + gamma
    dyr = beta * np.sqrt((qb * A) / (gamma * den))
    inv_A = dt.type(1) / A
    dyl, dyh = v - Y1, v - Y0
    dr = np.fmin(np.fmax(dyr, dyl), dyh)
    dl = np.fmin(np.fmax(-dyr, dyl), dyh)
    wr = qb - gamma * (dr * dr)
    wl = qb - gamma * (dl * dl)
    ok = (wr >= zero) | (wl >= zero)
    xr = (u + beta * dr) + np.sqrt(np.fmax(wr, zero) * inv_A)
    xl = (u + beta * dl) - np.sqrt(np.fmax(wl, zero) * inv_A)
    return ok, xl, xr


def band_hit(u, v, A, beta, gamma, qb, X0, X1, Y0, Y1):
    """The binning's ellipse-box test through band_span (see there)."""
    with np.errstate(invalid="ignore", over="ignore", divide="ignore"):
        ok, xl, xr = band_span(u, v, A, beta, gamma, qb, Y0, Y1)
        return ok & (xl <= xr) & (X1 >= xl) & (X0 <= xr)


U32 = 2.0 ** -24      # unit round-off of FP32 round-to-nearest


def band_margin(u, v, beta, half_x, half_y, width, height):
    """How far the FP32 binning decision (band_span in FP32 over the FP32 tile
    rectangle) can sit from the exact test tile_hit, as a perturbation of the
    problem: (delta [px], eps [relative]) such that the FP32 decision for a box is
    the exact decision for some box within delta of it on every side and some bound
    within qb (1 +- eps).

    Derivation (u_r = 2^-24; inputs u, v, A, beta, gamma, q_max exact FP32 values,
    box edges exact; first order in u_r):
      * the band offsets dy = v - Y are rounded once: |error| <= u_r (|v| + H), the
        same as moving the band's rows;
      * dy_r only selects where the concave right end (convex left end) is read:
        its error changes xr, xl to second order;
      * w = qb - gamma dy^2: |error| <= 3 u_r qb (two products and a difference,
        gamma dy^2 <= qb where w >= 0); sqrt(w / A) with 1/A, the product and the
        root each rounded adds 3 u_r relatively to w/A, i.e. 6 u_r qb in w: together
        an ellipse bound within 9 u_r qb of qb, plus qb = fl(q_max * 1.002f) itself
        (u_r and the constant's own rounding, < 3e-8);
      * xr = (u + beta dy) + s: three roundings, |error| <= u_r (3 |u| +
        3 |beta| (|v| + H) + 2 s) with s <= half_x, the same as moving the box's
        columns;
      * the tile rectangle from the FP32 half-extents: |error| <= u_r (|u| + 2 half_x)
        per column edge and u_r (|v| + 2 half_y) per row edge, again a move of the
        box's sides.
    The returned pair is that bound times a safety factor of 4 (second-order terms).
    """
    f = lambda x: np.abs(np.asarray(x, np.float64))
    u, v, beta, hx, hy = f(u), f(v), f(beta), f(half_x), f(half_y)
    delta = 4.0 * U32 * (4.0 * u + 3.0 * beta * (v + height) + 4.0 * (hx + hy) + 2.0 * v + height + width)
    eps = 4.0 * (9.0 * U32 + U32) + 3e-8
    return delta, eps


def camera_tensors(cam):
    R = torch.as_tensor(np.asarray(cam.R, np.float64))
    t = torch.as_tensor(np.asarray(cam.t, np.float64))
    return R, t


def project(means, log_scales, quats, opacity_logits, sh, sh_degree, cam,
            tile_w=16, tile_h=16):
    """Project N Gaussians into one camera, FP64.

    Inputs are torch float64 tensors (they may require grad): means [N,3],
    log_scales [N,3], quats [N,4], opacity_logits [N], sh [N,K,3]. Returns a
    dict: mean2d [N,2], conic [N,3] = (A, B, C) of Sigma''^-1 (power =
    -1/2 (A dx^2 + C dy^2) - B dx dy), conic_f [N,3] = (A, beta, gamma), the same
    conic factored, q_max [N] = 2 ln(255 o), depth [N], opacity [N], rgb [N,3],
    radius [N] int64 (0 = culled), rect [N,4] int64, visible [N] bool,
    clamped [N,3] bool, and diagnostics (half-extents, det, cov2d = Sigma').
    Culled records carry zero gradient (their outputs are masked).
    """
    R, t = camera_tensors(cam)
    W, H = cam.width, cam.height
    n = means.shape[0]
    tcam = means @ R.T + t                                   # t = W mu + t_cw
    tz = tcam[:, 2]
    in_front = (tz > NEAR).detach()
    tz_safe = torch.where(in_front, tz, torch.ones_like(tz))
    lim_x = FOV_CLAMP * (W / 2.0) / cam.fx
    lim_y = FOV_CLAMP * (H / 2.0) / cam.fy
    rx = torch.clamp(tcam[:, 0] / tz_safe, -lim_x, lim_x)
    ry = torch.clamp(tcam[:, 1] / tz_safe, -lim_y, lim_y)
    zero = torch.zeros_like(tz)
    J = torch.stack([
        torch.stack([cam.fx / tz_safe, zero, -cam.fx * rx / tz_safe], -1),
        torch.stack([zero, cam.fy / tz_safe, -cam.fy * ry / tz_safe], -1),
    ], -2)                                                   # [N,2,3]; -f tx~/tz^2 = -f rx/tz
    Sigma = covariance_3d(log_scales, quats)
    T = J @ R                                                 # J W
    cov2 = T @ Sigma @ T.transpose(-1, -2)
    a = cov2[:, 0, 0] + DILATION
    b = cov2[:, 0, 1]
    c = cov2[:, 1, 1] + DILATION
    det = a * c - b * b
    ok = in_front & (det > 0).detach()
    det_safe = torch.where(ok, det, torch.ones_like(det))
    conic = torch.stack([c / det_safe, -b / det_safe, a / det_safe], -1)
    c_safe = torch.where(ok, c, torch.ones_like(c))
    conic_f = torch.stack([c / det_safe, -b / c_safe, 1.0 / c_safe], -1)      # (A, beta, gamma)
    opacity = torch.sigmoid(opacity_logits)
    o_np = opacity.detach().numpy()
    ok = ok & torch.as_tensor(o_np >= ALPHA_MIN)
    with np.errstate(divide="ignore", invalid="ignore"):
        q_max = np.where(o_np >= ALPHA_MIN, 2.0 * np.log(255.0 * o_np), -1.0)
        qb = q_max * BIN_MARGIN
        hx = np.sqrt(qb * a.detach().numpy())
        hy = np.sqrt(qb * c.detach().numpy())
    half = np.where(ok.numpy()[:, None], np.stack([hx, hy], 1), -1.0)
    u = cam.fx * tcam[:, 0] / tz_safe + cam.cx
    v = cam.fy * tcam[:, 1] / tz_safe + cam.cy
    mean2d = torch.stack([u, v], -1)
    gx, gy = tile_grid(W, H, tile_w, tile_h)
    rect = tile_rect(mean2d.detach().numpy(), half, tile_w, tile_h, gx, gy)
    area = (rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1])
    visible = torch.as_tensor(area > 0) & ok
    radius = torch.as_tensor(np.where(visible.numpy(), np.ceil(np.nan_to_num(np.maximum(hx, hy))), 0)
                             .astype(np.int64))
    rect[~visible.numpy()] = 0
    # colour from SH, direction from the camera centre to the mean
    center = -(R.T @ t)
    d = means - center
    d = d / torch.linalg.vector_norm(d, dim=-1, keepdim=True)
    K = num_coeffs(sh_degree)
    Y = sh_basis(d, sh_degree)                                # [N,K]
    raw = torch.einsum("nk,nkc->nc", Y, sh[:, :K, :]) + 0.5
    clamped = (raw < 0).detach()
    rgb = torch.clamp(raw, min=0.0)
    vis = visible[:, None]
    return dict(
        mean2d=torch.where(vis, mean2d, torch.zeros_like(mean2d)),
        conic=torch.where(vis, conic, torch.zeros_like(conic)),
        conic_f=torch.where(vis, conic_f, torch.zeros_like(conic_f)),
        q_max=np.where(visible.numpy(), q_max, 0.0),
        depth=torch.where(visible, tz, torch.zeros_like(tz)),
        opacity=torch.where(visible, opacity, torch.zeros_like(opacity)),
        rgb=torch.where(vis, rgb, torch.zeros_like(rgb)),
        radius=radius, rect=torch.as_tensor(rect), visible=visible, clamped=clamped & vis,
        half=half, det=det.detach(), cov2d=cov2.detach(),
        n=n, grid=(gx, gy),
    )


def params_to_torch(params: dict, requires_grad=False) -> dict:
    out = {}
    for k in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        out[k] = torch.tensor(np.asarray(params[k], np.float64), requires_grad=requires_grad)
    return out


def project_np(params: dict, sh_degree: int, cam, tile_w=16, tile_h=16) -> dict:
    """Convenience wrapper: numpy float32/float64 params -> numpy FP64 outputs."""
    p = params_to_torch(params)
    with torch.no_grad():
        out = project(p["means"], p["log_scales"], p["quats"], p["opacity_logits"], p["sh"],
                      sh_degree, cam, tile_w, tile_h)
    res = {}
    for k, v in out.items():
        res[k] = v.numpy() if isinstance(v, torch.Tensor) else v
    return res
