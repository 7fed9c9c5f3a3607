"""EWA projection of 3D Gaussians and SH colour (FP64) -- test infrastructure only.

Follows Sec. "Preliminary" of the paper: Eq. 1 (the Gaussian with covariance
Sigma = R S S^T R^T), the affine (Jacobian) projection Sigma' = J W Sigma W^T J^T,
and the SH-evaluated colour c_i of Eq. 2. Readings where the paper is silent:
  * activations: R from the normalised quaternion (w, x, y, z), S = diag(exp s),
    opacity = sigmoid(logit);
  * near-plane cull at t_z <= near (0.2);
  * J is evaluated at the camera-space mean with t_x/t_z, t_y/t_z clamped to
    +-1.3 * (W/2)/f_x, +-1.3 * (H/2)/f_y (no gradient through a clamped ratio);
  * a 0.3 px^2 low-pass dilation on the diagonal of Sigma'; cull when det <= 0;
  * extent r = ceil(3 sqrt(lambda_max)), lambda_max = m + sqrt(max(0.1, m^2 - det));
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
EXTENT_SIGMAS = 3.0


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


def tile_rect(mean2d: np.ndarray, radius: np.ndarray, tile_w: int, tile_h: int,
              grid_x: int, grid_y: int) -> np.ndarray:
    """Tile rectangle [x0, y0, x1, y1) of each record; all-zero for radius 0.

    x0 = clamp(floor((u - r) / tw), 0, gx), x1 = clamp(floor((u + (r + tw - 1)) / tw), 0, gx),
    likewise for y. The arithmetic runs in mean2d's own dtype (FP32 for FP32
    records): each of the subtraction/addition and the division is one rounded
    operation of that precision, r and r + tw - 1 being exact integers.
    """
    dt = mean2d.dtype.type
    u = mean2d[:, 0]
    v = mean2d[:, 1]
    r = radius.astype(mean2d.dtype)
    tw, th = dt(tile_w), dt(tile_h)
    x0 = np.floor((u - r) / tw)
    y0 = np.floor((v - r) / th)
    x1 = np.floor((u + (radius + (tile_w - 1)).astype(mean2d.dtype)) / tw)
    y1 = np.floor((v + (radius + (tile_h - 1)).astype(mean2d.dtype)) / th)
    rect = np.stack([np.clip(x0, 0, grid_x), np.clip(y0, 0, grid_y),
                     np.clip(x1, 0, grid_x), np.clip(y1, 0, grid_y)], 1).astype(np.int64)
    rect[radius <= 0] = 0
    return rect


def camera_tensors(cam):
    R = torch.as_tensor(np.asarray(cam.R, np.float64))
    t = torch.as_tensor(np.asarray(cam.t, np.float64))
    return R, t


def project(means, log_scales, quats, opacity_logits, sh, sh_degree, cam,
            tile_w=16, tile_h=16):
    """Project N Gaussians into one camera, FP64.

    Inputs are torch float64 tensors (they may require grad): means [N,3],
    log_scales [N,3], quats [N,4], opacity_logits [N], sh [N,K,3]. Returns a
    dict: mean2d [N,2], conic [N,3] = (A, B, C) of Sigma'^-1 (power =
    -1/2 (A dx^2 + C dy^2) - B dx dy), depth [N], opacity [N], rgb [N,3],
    radius [N] int64 (0 = culled), rect [N,4] int64, visible [N] bool,
    clamped [N,3] bool, and the diagnostics extent (3 sqrt(lambda_max)).
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
    mid = 0.5 * (a + c)
    lam = mid + torch.sqrt(torch.clamp(mid * mid - det, min=0.1))
    extent = EXTENT_SIGMAS * torch.sqrt(lam)
    radius = torch.where(ok, torch.ceil(extent.detach()), torch.zeros_like(extent)).to(torch.int64)
    u = cam.fx * tcam[:, 0] / tz_safe + cam.cx
    v = cam.fy * tcam[:, 1] / tz_safe + cam.cy
    mean2d = torch.stack([u, v], -1)
    gx, gy = tile_grid(W, H, tile_w, tile_h)
    rect = tile_rect(mean2d.detach().numpy(), radius.numpy(), tile_w, tile_h, gx, gy)
    area = (rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1])
    visible = torch.as_tensor(area > 0) & ok
    radius = torch.where(visible, radius, torch.zeros_like(radius))
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
    opacity = torch.sigmoid(opacity_logits)
    vis = visible[:, None]
    return dict(
        mean2d=torch.where(vis, mean2d, torch.zeros_like(mean2d)),
        conic=torch.where(vis, conic, torch.zeros_like(conic)),
        depth=torch.where(visible, tz, torch.zeros_like(tz)),
        opacity=torch.where(visible, opacity, torch.zeros_like(opacity)),
        rgb=torch.where(vis, rgb, torch.zeros_like(rgb)),
        radius=radius, rect=torch.as_tensor(rect), visible=visible, clamped=clamped & vis,
        extent=extent.detach(), det=det.detach(), cov2d=cov2.detach(),
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
