"""Seeded synthetic scenes and cameras for the Gaussian-splatting hot path.

This module only draws random numbers and builds camera poses; it holds none of
the rasterizer's arithmetic. Both the CUDA path and the FP64 oracle consume the
arrays it returns, so it imports nothing but numpy.

The paper evaluates on MipNeRF-360, Deep Blending and Tanks & Temples initialised
from SfM point clouds (Sec. "Datasets and metrics"). Those datasets are not used
here: the generators below produce scenes with the same shape -- about a million
Gaussians concentrated on a few surfaces plus a sparse background, 1246x826
views on an orbit, spherical-harmonic colour up to degree 3 -- so that tile-list
lengths, overlap and early termination behave like a real capture.

Conventions (shared by every consumer):
  * Gaussians are SoA float32: means [N,3], log_scales [N,3], quats [N,4] as
    (w, x, y, z) and unnormalised, opacity_logits [N], sh [N, K, 3] with
    K = (deg+1)^2 coefficients per colour channel.
  * A camera is world->camera R (3x3, row-major) and t (3,), OpenCV axes
    (x right, y down, z forward), pinhole fx, fy, cx, cy, width, height.
  * Images are planar float32 [3, H, W].
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NEAR_PLANE = 0.2


@dataclass
class Camera:
    R: np.ndarray          # (3, 3) float32, world -> camera rotation
    t: np.ndarray          # (3,) float32, world -> camera translation
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = NEAR_PLANE

    @property
    def center(self) -> np.ndarray:
        """Camera centre in world coordinates, -R^T t (float64)."""
        return -(self.R.astype(np.float64).T @ self.t.astype(np.float64))


@dataclass
class Scene:
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    opacity_logits: np.ndarray
    sh: np.ndarray
    sh_degree: int
    cameras: list = field(default_factory=list)
    targets: list = field(default_factory=list)   # [3, H, W] float32 per camera
    name: str = ""

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def params(self) -> dict:
        return dict(means=self.means, log_scales=self.log_scales, quats=self.quats,
                    opacity_logits=self.opacity_logits, sh=self.sh)


def look_at_camera(center, width, height, fx, fy=None, cx=None, cy=None,
                   target=(0.0, 0.0, 0.0), down=(0.0, 1.0, 0.0)) -> Camera:
    """Pinhole camera at `center` looking at `target`; world 'down' is +y.

    Rows of R are the camera axes expressed in world coordinates:
    z = forward, x = down x forward (right), y = forward x right (down).
    """
    c = np.asarray(center, np.float64)
    z = np.asarray(target, np.float64) - c
    z /= np.linalg.norm(z)
    x = np.cross(np.asarray(down, np.float64), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ c
    fy = fx if fy is None else fy
    cx = width / 2.0 if cx is None else cx
    cy = height / 2.0 if cy is None else cy
    return Camera(R=R.astype(np.float32), t=t.astype(np.float32), fx=float(fx), fy=float(fy),
                  cx=float(cx), cy=float(cy), width=int(width), height=int(height))


def orbit_camera(radius, azimuth, elevation_deg, width, height, f) -> Camera:
    """Camera on a sphere of `radius` around the origin; elevation is above the
    horizon, i.e. towards world -y (world up = -y)."""
    el = math.radians(elevation_deg)
    center = (radius * math.cos(el) * math.sin(azimuth),
              -radius * math.sin(el),
              -radius * math.cos(el) * math.cos(azimuth))
    return look_at_camera(center, width, height, f)


def _unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _ball(rng, n, radius):
    d = rng.standard_normal((n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * rng.uniform(0.0, 1.0, n) ** (1.0 / 3.0)
    return d * r[:, None]


def _tangent_frame(nrm):
    a = np.array([1.0, 0.0, 0.0]) if abs(nrm[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    u = np.cross(nrm, a)
    u /= np.linalg.norm(u)
    v = np.cross(nrm, u)
    return u, v


def surface_points(rng, n, n_patches=20, center_radius=2.0, background_frac=0.1,
                   background_radius=10.0, size_scale=1.0):
    """Means on `n_patches` planar squares / spherical caps plus a uniform ball.

    Each patch is, with probability 1/2, a square of half-extent U[0.3, 1.0]
    with a uniformly random normal, else a hemispherical cap of radius
    U[0.2, 0.8] around a uniformly random axis; centres are uniform in a ball of
    `center_radius`. Surface points are split among patches in proportion to
    patch area; points are uniform over each patch.
    """
    n_bg = int(round(background_frac * n))
    n_surf = n - n_bg
    kinds, sizes, centers, axes, areas = [], [], [], [], []
    for _ in range(n_patches):
        planar = rng.uniform() < 0.5
        c = _ball(rng, 1, center_radius)[0]
        ax = rng.standard_normal(3)
        ax /= np.linalg.norm(ax)
        if planar:
            h = rng.uniform(0.3, 1.0) * size_scale
            area = 4.0 * h * h
        else:
            h = rng.uniform(0.2, 0.8) * size_scale
            area = 2.0 * math.pi * h * h
        kinds.append(planar); sizes.append(h); centers.append(c); axes.append(ax); areas.append(area)
    areas = np.asarray(areas)
    counts = rng.multinomial(n_surf, areas / areas.sum())
    pts = []
    for planar, h, c, ax, k in zip(kinds, sizes, centers, axes, counts):
        u, v = _tangent_frame(ax)
        if planar:
            a = rng.uniform(-h, h, k)
            b = rng.uniform(-h, h, k)
            p = c + a[:, None] * u + b[:, None] * v
        else:
            cz = rng.uniform(0.0, 1.0, k)          # cos of the polar angle, hemisphere
            phi = rng.uniform(0.0, 2.0 * math.pi, k)
            sz = np.sqrt(np.maximum(0.0, 1.0 - cz * cz))
            d = (sz * np.cos(phi))[:, None] * u + (sz * np.sin(phi))[:, None] * v + cz[:, None] * ax
            p = c + h * d
        pts.append(p)
    pts.append(_ball(rng, n_bg, background_radius))
    pts = np.concatenate(pts, axis=0)
    return pts[rng.permutation(n)]


def _sh_coeffs(rng, n, degree, rest_std=0.05):
    k = (degree + 1) ** 2
    sh = np.zeros((n, k, 3), np.float64)
    sh[:, 0, :] = rng.uniform(0.0, 1.0, (n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, rest_std, (n, k - 1, 3))
    return sh


def _target(rng, cam):
    return rng.uniform(0.0, 1.0, (cam.height, cam.width, 3)).astype(np.float32).transpose(2, 0, 1).copy()


def _f32(*arrs):
    return [np.ascontiguousarray(a, dtype=np.float32) for a in arrs]


def small_scene(seed: int = 0, n: int = 2000, width: int = 64, height: int = 64) -> Scene:
    """2,000 Gaussians, SH degree 0, one 64x64 camera at (0,0,-4), fx=fy=64.

    Means U[-1,1]^3, log-scales N(-3, 0.5) per axis, uniformly random rotations,
    opacity logits N(0,1), DC coefficient U[0,1]; the L1 target is uniform
    [0,1] drawn after the parameters from the same generator.
    """
    rng = np.random.default_rng(seed)
    means = rng.uniform(-1.0, 1.0, (n, 3))
    log_scales = rng.normal(-3.0, 0.5, (n, 3))
    quats = _unit_quats(rng, n)
    logits = rng.normal(0.0, 1.0, n)
    sh = rng.uniform(0.0, 1.0, (n, 1, 3))
    cam = Camera(R=np.eye(3, dtype=np.float32), t=np.array([0, 0, 4], np.float32),
                 fx=float(width), fy=float(height), cx=width / 2.0, cy=height / 2.0,
                 width=width, height=height)
    target = _target(rng, cam)
    m, s, q, o, c = _f32(means, log_scales, quats, logits, sh)
    return Scene(m, s, q, o, c, 0, [cam], [target], name=f"small-{n}")


def surface_scene(seed: int, n: int, sh_degree: int = 3, center_radius=2.0,
                  background_radius=10.0, size_scale=1.0, log_scale_mean=-4.0,
                  log_scale_std=0.7) -> Scene:
    """Surface-patch scene without cameras (see `surface_points`).

    Log-scales N(-4, 0.7) per axis, uniformly random rotations, opacity logits
    N(0,1), DC coefficients U[0,1], higher SH bands N(0, 0.05).
    """
    rng = np.random.default_rng(seed)
    means = surface_points(rng, n, center_radius=center_radius,
                           background_radius=background_radius, size_scale=size_scale)
    log_scales = rng.normal(log_scale_mean, log_scale_std, (n, 3))
    quats = _unit_quats(rng, n)
    logits = rng.normal(0.0, 1.0, n)
    sh = _sh_coeffs(rng, n, sh_degree)
    m, s, q, o, c = _f32(means, log_scales, quats, logits, sh)
    return Scene(m, s, q, o, c, sh_degree, name=f"surface-{n}")


def orbit_scene(seed: int = 1, n: int = 1_500_000, width: int = 1246, height: int = 826,
                f: float = 1246.0, sh_degree: int = 3) -> Scene:
    """1.5M-Gaussian surface scene, SH degree 3, one 1246x826 view on a
    radius-4 orbit (seeded azimuth, 15 deg elevation), fx=fy=1246."""
    sc = surface_scene(seed, n, sh_degree)
    rng = np.random.default_rng(seed + 1000)
    az = rng.uniform(0.0, 2.0 * math.pi)
    cam = orbit_camera(4.0, az, 15.0, width, height, f)
    sc.cameras = [cam]
    sc.targets = [_target(rng, cam)]
    sc.name = f"orbit-{n}-{width}x{height}"
    return sc


MIXED_RES = ((312, 207, 0.25), (623, 413, 0.5), (1246, 826, 1.0))


def mixed_resolution_cameras(n_views: int = 12, radius: float = 4.0, base_f: float = 1246.0,
                             seed: int = 2):
    """`n_views` cameras at azimuth 2*pi*k/n_views; view k uses the resolution
    MIXED_RES[k % 3] (1/4, 1/2 and full 1246x826, focal scaled alike)."""
    rng = np.random.default_rng(seed + 2000)
    cams, targets = [], []
    for k in range(n_views):
        w, h, s = MIXED_RES[k % 3]
        cam = orbit_camera(radius, 2.0 * math.pi * k / n_views, 15.0, w, h, base_f * s)
        cams.append(cam)
        targets.append(_target(rng, cam))
    return cams, targets


def batched_scene(seed: int = 2, n: int = 500_000, n_views: int = 12) -> Scene:
    """500k-Gaussian surface scene with 12 mixed-resolution orbit views."""
    sc = surface_scene(seed, n, 3)
    sc.cameras, sc.targets = mixed_resolution_cameras(n_views, seed=seed)
    sc.name = f"batched-{n}-{n_views}views"
    return sc


def large_scene(seed: int = 4, n: int = 5_000_000, n_views: int = 4, width=1600, height=1060,
                f=1600.0) -> Scene:
    """5M Gaussians: the surface generator scaled x3 (patch centres in a
    radius-6 ball, background in a radius-30 ball), 4 views at 1600x1060 on a
    radius-12 orbit, fx=fy=1600."""
    sc = surface_scene(seed, n, 3, center_radius=6.0, background_radius=30.0, size_scale=3.0)
    rng = np.random.default_rng(seed + 4000)
    cams, targets = [], []
    for k in range(n_views):
        cam = orbit_camera(12.0, 2.0 * math.pi * k / n_views + 0.3, 15.0, width, height, f)
        cams.append(cam)
        targets.append(_target(rng, cam))
    sc.cameras, sc.targets = cams, targets
    sc.name = f"large-{n}-{n_views}views"
    return sc


def sfm_like_init(gt: Scene, n: int, seed: int = 3, jitter: float = 0.01, sh_degree: int = 3,
                  colour_noise: float = 0.1) -> Scene:
    """An initial scene of the kind a structure-from-motion point cloud gives the 3DGS
    lineage, drawn from a ground-truth scene instead of from its generator: n of its
    means (without replacement) jittered by N(0, jitter^2) per axis, the colour of the
    picked Gaussian (its DC coefficient plus N(0, colour_noise^2)), isotropic
    log-scales log(mean distance to the 3 nearest picked points), identity
    rotations, opacity 0.1 and zero higher SH bands."""
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    idx = rng.choice(gt.n, n, replace=False)
    means = gt.means[idx].astype(np.float64) + rng.normal(0.0, jitter, (n, 3))
    d, _ = cKDTree(means).query(means, k=4)
    scale = np.maximum(d[:, 1:].mean(1), 1e-7)
    log_scales = np.repeat(np.log(scale)[:, None], 3, 1)
    quats = np.zeros((n, 4))
    quats[:, 0] = 1.0
    logits = np.full(n, math.log(0.1 / 0.9))
    sh = np.zeros((n, (sh_degree + 1) ** 2, 3))
    sh[:, 0, :] = gt.sh[idx, 0, :] + rng.normal(0.0, colour_noise, (n, 3))
    m, s, q, o, c = _f32(means, log_scales, quats, logits, sh)
    return Scene(m, s, q, o, c, sh_degree, name=f"sfm-init-{n}")


def random_records(seed: int, n: int, width: int, height: int, max_radius: int = 40,
                   cull_frac: float = 0.1):
    """Synthetic projected records (mean2d, depth, radius) for testing binning
    and sorting in isolation: means uniform over a margin-extended image,
    depths log-uniform in [0.3, 30] with deliberate exact ties, radii uniform in
    [1, max_radius] with a fraction culled (radius 0)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(-max_radius, width + max_radius, n)
    v = rng.uniform(-max_radius, height + max_radius, n)
    depth = np.exp(rng.uniform(math.log(0.3), math.log(30.0), n))
    tie = rng.uniform(size=n) < 0.05
    depth[tie] = depth[rng.integers(0, n, tie.sum())]
    radius = rng.integers(1, max_radius + 1, n)
    radius[rng.uniform(size=n) < cull_frac] = 0
    return (np.stack([u, v], 1).astype(np.float32), depth.astype(np.float32),
            radius.astype(np.int32))
