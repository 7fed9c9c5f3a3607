"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test checks one oracle function against a closed form, a textbook or library
routine, brute force on tiny inputs, an invariant, or central finite differences,
so that a dropped term, a wrong sign or index, or a transposed operand fails.
"""
import math
import os

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import sh as osh
from oracle import project as oproj
from oracle import raster as oras
from oracle import densify as oden
from oracle import pipeline as opipe
from oracle.loss import l1_loss_grad
from paper_2507_20239_gb300.synth import Camera, small_scene, look_at_camera

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ spherical harmonics
def _sphere_quadrature(n_theta=24, n_phi=48):
    zs, wz = np.polynomial.legendre.leggauss(n_theta)       # exact for polynomials in z
    phis = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi   # exact for trig polys < n_phi
    Z, PHI = np.meshgrid(zs, phis, indexing="ij")
    S = np.sqrt(1 - Z ** 2)
    dirs = np.stack([S * np.cos(PHI), S * np.sin(PHI), Z], -1).reshape(-1, 3)
    w = (wz[:, None] * np.full(n_phi, 2 * math.pi / n_phi)[None, :]).reshape(-1)
    return dirs, w


def test_sh_orthonormal_by_quadrature():
    dirs, w = _sphere_quadrature()
    Y = osh.sh_basis(torch.tensor(dirs), 3).numpy()
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_addition_theorem():
    rng = np.random.default_rng(0)
    d = rng.standard_normal((50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = osh.sh_basis(torch.tensor(d), 3).numpy()
    for l in range(4):
        s = (Y[:, l * l:(l + 1) ** 2] ** 2).sum(1)
        assert np.allclose(s, (2 * l + 1) / (4 * math.pi), atol=1e-13)


def test_sh_closed_forms_golden():
    rng = np.random.default_rng(1)
    d = rng.standard_normal((20, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = osh.sh_basis(torch.tensor(d), 2).numpy()
    x, y, z = d.T
    env = dict(sqrt=math.sqrt, pi=math.pi, x=x, y=y, z=z)
    n = 0
    with open(os.path.join(GOLDEN, "real_sh_closed_forms.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, l, m, coef, mono = line.split()
            want = eval(coef, env) * eval(mono, env) * np.ones_like(x)
            assert np.allclose(Y[:, int(k)], want, atol=1e-14), (k, l, m)
            n += 1
    assert n == 9
    assert abs(osh.norm_const(0, 0) - 0.28209479177387814) < 1e-16


# ------------------------------------------------------------------ rotation / covariance
def test_quaternion_matches_scipy_rotation():
    rng = np.random.default_rng(2)
    q = rng.standard_normal((64, 4)) * 3.0          # unnormalised on purpose
    R = oproj.quat_to_rotmat(torch.tensor(q)).numpy()
    ref = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()   # scipy is scalar-last
    assert np.abs(R - ref).max() < 1e-13
    assert np.abs(R - oproj.quat_to_rotmat(torch.tensor(-q)).numpy()).max() < 1e-13


def test_covariance_eigendecomposition():
    rng = np.random.default_rng(3)
    s = rng.normal(-2, 0.5, (16, 3))
    q = rng.standard_normal((16, 4))
    Sig = oproj.covariance_3d(torch.tensor(s), torch.tensor(q)).numpy()
    Rm = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    for i in range(16):
        for k in range(3):
            v = Rm[i][:, k]
            assert np.allclose(Sig[i] @ v, math.exp(2 * s[i, k]) * v, rtol=1e-12, atol=1e-15)


# ------------------------------------------------------------------ projection
def _cam(W=64, H=48, f=50.0, R=None, t=(0, 0, 0)):
    return Camera(R=np.eye(3, dtype=np.float32) if R is None else np.asarray(R, np.float32),
                  t=np.asarray(t, np.float32), fx=f, fy=f * 1.1, cx=W / 2, cy=H / 2,
                  width=W, height=H)


def _one(mean, log_scale, quat=(1, 0, 0, 0), logit=0.0, sh=None, deg=0):
    sh = np.zeros((1, (deg + 1) ** 2, 3)) if sh is None else np.asarray(sh, np.float64)[None]
    return dict(means=np.array([mean], np.float64), log_scales=np.array([log_scale], np.float64),
                quats=np.array([quat], np.float64), opacity_logits=np.array([logit], np.float64),
                sh=sh)


def test_isotropic_on_axis_closed_form():
    cam = Camera(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=80.0, fy=80.0,
                 cx=32.0, cy=32.0, width=64, height=64)
    d, sig = 5.0, 0.1
    out = oproj.project_np(_one([0, 0, d], [math.log(sig)] * 3), 0, cam)
    s2 = (80.0 * sig / d) ** 2 + 0.3
    assert np.allclose(out["cov2d"][0], np.diag([s2 - 0.3, s2 - 0.3]), atol=1e-13)
    assert np.allclose(out["conic"][0], [1 / s2, 0.0, 1 / s2], rtol=1e-13)
    assert np.allclose(out["mean2d"][0], [32.0, 32.0])
    assert out["depth"][0] == d
    assert np.allclose(out["conic_f"][0], [1 / s2, 0.0, 1 / s2], rtol=1e-13)
    # alpha >= 1/255 inside the circle rho^2 <= s2 q_max, q_max = 2 ln(255 o), o = 1/2
    q_max = 2 * math.log(255 * 0.5)
    assert abs(out["q_max"][0] - q_max) < 1e-12
    assert out["radius"][0] == math.ceil(math.sqrt(q_max * 1.002 * s2))


def _pinhole(p, cam):
    return np.array([cam.fx * p[0] / p[2] + cam.cx, cam.fy * p[1] / p[2] + cam.cy])


def _fd_jacobian(p, cam, h=1e-6):
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3); e[k] = h
        J[:, k] = (_pinhole(p + e, cam) - _pinhole(p - e, cam)) / (2 * h)
    return J


def test_projection_matches_fd_jacobian_off_axis():
    rng = np.random.default_rng(4)
    Rw = Rotation.from_euler("xyz", [0.2, -0.3, 0.1]).as_matrix()
    cam = _cam(R=Rw, t=(0.1, -0.2, 3.0))
    for _ in range(10):
        mu = rng.uniform(-0.5, 0.5, 3)
        ls = rng.normal(-2.5, 0.4, 3)
        q = rng.standard_normal(4)
        out = oproj.project_np(_one(mu, ls, q), 0, cam)
        pc = Rw @ mu + np.array([0.1, -0.2, 3.0])
        assert np.allclose(out["mean2d"][0], _pinhole(pc, cam), atol=1e-9)
        J = _fd_jacobian(pc, cam)
        Rm = Rotation.from_quat(q[[1, 2, 3, 0]]).as_matrix()
        Sig = Rm @ np.diag(np.exp(2 * ls)) @ Rm.T
        ref = J @ Rw @ Sig @ Rw.T @ J.T
        assert np.abs(out["cov2d"][0] - ref).max() < 1e-6 * np.abs(ref).max()


def test_projection_jacobian_clamped_off_screen():
    cam = _cam(W=64, H=48, f=50.0)
    lim = 1.3 * 32 / 50.0
    mu = np.array([3.0 * lim * 4.0, 0.0, 4.0])       # t_x / t_z = 3 lim: far off screen
    ls = [math.log(0.3)] * 3
    out = oproj.project_np(_one(mu, ls), 0, cam)
    Jc = _fd_jacobian(np.array([lim * 4.0, 0.0, 4.0]), cam)   # evaluated at the clamped point
    ref = Jc @ np.diag([0.09] * 3) @ Jc.T
    assert np.abs(out["cov2d"][0] - ref).max() < 1e-6 * np.abs(ref).max()


def test_near_plane_and_offscreen_cull():
    cam = _cam()
    p = _one([0, 0, 0.19], [-3] * 3)
    assert oproj.project_np(p, 0, cam)["radius"][0] == 0
    p = _one([0, 0, 0.21], [-3] * 3)
    assert oproj.project_np(p, 0, cam)["radius"][0] > 0
    p = _one([100.0, 0, 1.0], [-5] * 3)       # far right of the image: empty rect
    out = oproj.project_np(p, 0, cam)
    assert out["radius"][0] == 0 and not out["visible"][0]


def test_sh_colour_degree0_and_clamp():
    cam = _cam()
    out = oproj.project_np(_one([0, 0, 2], [-3] * 3, sh=[[0.4, -0.2, -3.0]]), 0, cam)
    c0 = 1 / (2 * math.sqrt(math.pi))
    assert np.allclose(out["rgb"][0], [c0 * 0.4 + 0.5, c0 * -0.2 + 0.5, 0.0], atol=1e-15)
    assert list(out["clamped"][0]) == [False, False, True]


def test_sh_colour_direction_from_camera_centre():
    # camera centre at (0, 0, -4): a Gaussian at the origin is seen along +z, so a
    # degree-1 coefficient on Y_1,0 (= sqrt(3/4pi) z) contributes fully
    cam = Camera(R=np.eye(3, dtype=np.float32), t=np.array([0, 0, 4], np.float32), fx=64.0,
                 fy=64.0, cx=32.0, cy=32.0, width=64, height=64)
    sh = np.zeros((4, 3)); sh[2] = [1.0, 0.0, 0.0]
    out = oproj.project_np(_one([0, 0, 0], [-3] * 3, sh=sh, deg=1), 1, cam)
    assert abs(out["rgb"][0][0] - (math.sqrt(3 / (4 * math.pi)) + 0.5)) < 1e-14


def test_tile_rect_integer_bounds_brute_force():
    rng = np.random.default_rng(5)
    tw, th, gx, gy = 16, 8, 5, 7
    u = rng.integers(-40, 120, 200).astype(np.float32)
    v = rng.integers(-40, 100, 200).astype(np.float32)
    half = rng.integers(0, 30, (200, 2)).astype(np.float32)
    rect = oproj.tile_rect(np.stack([u, v], 1), half, tw, th, gx, gy)
    for i in range(200):
        # tiles whose pixel span [t*tw, (t+1)*tw) meets the closed box [u - hx, u + hx]
        xs = [tx for tx in range(gx) if tx * tw <= u[i] + half[i, 0] and (tx + 1) * tw > u[i] - half[i, 0]]
        ys = [ty for ty in range(gy) if ty * th <= v[i] + half[i, 1] and (ty + 1) * th > v[i] - half[i, 1]]
        want = (xs[0], ys[0], xs[-1] + 1, ys[-1] + 1) if xs and ys else None
        got = tuple(rect[i])
        if want is None:
            assert (got[2] - got[0]) * (got[3] - got[1]) == 0
        else:
            assert got == want, (i, got, want)


def _rand_conic_f(rng, n, dtype=np.float64):
    L = rng.uniform(0.5, 12, (n, 2))
    th_ = rng.uniform(0, math.pi, n)
    out = np.zeros((n, 3))
    for g in range(n):
        Rm = np.array([[math.cos(th_[g]), -math.sin(th_[g])], [math.sin(th_[g]), math.cos(th_[g])]])
        Ci = np.linalg.inv(Rm @ np.diag(L[g] ** 2) @ Rm.T)
        out[g] = [Ci[0, 0], Ci[0, 1] / Ci[0, 0], Ci[1, 1] - Ci[0, 1] ** 2 / Ci[0, 0]]
    return out.astype(dtype)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_tile_hit_matches_dense_sampling(dtype):
    rng = np.random.default_rng(12)
    n = 400
    cf = _rand_conic_f(rng, n, dtype)
    u = rng.uniform(-20, 50, n).astype(dtype)
    v = rng.uniform(-20, 50, n).astype(dtype)
    qb = rng.uniform(1, 12, n).astype(dtype)
    X0, X1, Y0, Y1 = (np.full(n, x, dtype) for x in (8.5, 23.5, 16.5, 31.5))
    hit = oproj.tile_hit(u, v, cf[:, 0], cf[:, 1], cf[:, 2], qb, X0, X1, Y0, Y1)
    g = np.linspace(0, 1, 61)
    for i in range(n):
        px = X0[i] + g * (X1[i] - X0[i])
        py = Y0[i] + g * (Y1[i] - Y0[i])
        PX, PY = np.meshgrid(px.astype(np.float64), py.astype(np.float64))
        dx, dy = float(u[i]) - PX, float(v[i]) - PY
        A, b, c = (float(x) for x in cf[i])
        q = A * (dx + b * dy) ** 2 + c * dy ** 2
        if q.min() <= float(qb[i]) * (1 - 1e-5):
            assert hit[i], i                         # a sampled point inside: must hit
        # the true box minimum lies within the grid spacing of a sample
        step = np.hypot((X1[i] - X0[i]) / 60, (Y1[i] - Y0[i]) / 60)
        if hit[i]:
            grad = 2 * math.sqrt(max(A, c)) * math.sqrt(q.min()) * (1 + abs(b)) * step + 1e-6
            assert q.min() <= float(qb[i]) * (1 + 1e-5) + grad, i


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_band_hit_matches_dense_sampling(dtype):
    # the binning's test: a box meets the ellipse iff its column range meets the
    # ellipse's x-extent over the box's rows; checked against sampled q values
    rng = np.random.default_rng(13)
    n = 400
    cf = _rand_conic_f(rng, n, dtype)
    u = rng.uniform(-20, 50, n).astype(dtype)
    v = rng.uniform(-20, 50, n).astype(dtype)
    qb = rng.uniform(1, 12, n).astype(dtype)
    X0, X1, Y0, Y1 = (np.full(n, x, dtype) for x in (8.5, 23.5, 16.5, 31.5))
    hit = oproj.band_hit(u, v, cf[:, 0], cf[:, 1], cf[:, 2], qb, X0, X1, Y0, Y1)
    assert 50 < hit.sum() < n - 50
    g = np.linspace(0, 1, 61)
    for i in range(n):
        PX, PY = np.meshgrid((X0[i] + g * (X1[i] - X0[i])).astype(np.float64),
                             (Y0[i] + g * (Y1[i] - Y0[i])).astype(np.float64))
        dx, dy = float(u[i]) - PX, float(v[i]) - PY
        A, b, c = (float(x) for x in cf[i])
        q = A * (dx + b * dy) ** 2 + c * dy ** 2
        if q.min() <= float(qb[i]) * (1 - 1e-5):
            assert hit[i], i
        step = np.hypot((X1[i] - X0[i]) / 60, (Y1[i] - Y0[i]) / 60)
        if hit[i]:
            grad = 2 * math.sqrt(max(A, c)) * math.sqrt(q.min()) * (1 + abs(b)) * step + 1e-6
            assert q.min() <= float(qb[i]) * (1 + 1e-5) + grad, i


def test_band_hit_equals_box_minimum_test_in_fp64():
    # two exact formulations of "ellipse meets box" (x-extent over the band vs the
    # clamped minimum of q on the box): identical except within rounding of qb
    rng = np.random.default_rng(14)
    n = 20000
    cf = _rand_conic_f(rng, n)
    u = rng.uniform(-25, 55, n)
    v = rng.uniform(-25, 55, n)
    qb = rng.uniform(0.5, 12, n)
    X0, X1, Y0, Y1 = (np.full(n, x) for x in (8.5, 23.5, 16.5, 31.5))
    a = oproj.band_hit(u, v, cf[:, 0], cf[:, 1], cf[:, 2], qb, X0, X1, Y0, Y1)
    b = oproj.tile_hit(u, v, cf[:, 0], cf[:, 1], cf[:, 2], qb, X0, X1, Y0, Y1)
    near = np.zeros(n, bool)
    for s in (1 - 1e-9, 1 + 1e-9):
        near |= oproj.tile_hit(u, v, cf[:, 0], cf[:, 1], cf[:, 2], qb * s, X0, X1, Y0, Y1) != b
    assert 0.15 * n < b.sum() < 0.85 * n
    assert np.array_equal(a[~near], b[~near])


def test_fp32_band_decision_within_derived_margin_of_exact_test():
    # The FP32 binning decision (band_span in FP32, the procedure the CUDA lists
    # follow) against the exact FP64 box-minimum test, at the coordinate magnitudes
    # of a 2048-pixel frame: every box the exact test keeps with the derived margin
    # (box shrunk by delta, bound qb (1 - eps)) is kept in FP32, and every box FP32
    # keeps is kept exactly once grown by delta with bound qb (1 + eps).
    rng = np.random.default_rng(15)
    n = 200_000
    W, H = 2048, 1400
    cf = _rand_conic_f(rng, n)
    # elongated splats too: beta up to ~10
    cf[: n // 4, 1] *= rng.uniform(1, 10, n // 4)
    qb = rng.uniform(0.5, 12, n)
    X0 = rng.integers(0, W // 16, n) * 16 + 0.5
    Y0 = rng.integers(0, H // 16, n) * 16 + 0.5
    X1, Y1 = X0 + 15.0, Y0 + 15.0
    # means within a few footprint radii of the box
    half = oproj.footprint_half(cf, qb / oproj.BIN_MARGIN)
    u = X0 + rng.uniform(-1.5, 2.5, n) * (half[:, 0] + 8)
    v = Y0 + rng.uniform(-1.5, 2.5, n) * (half[:, 1] + 8)
    f32 = lambda x: np.asarray(x, np.float32)
    u, v, qb = f32(u).astype(np.float64), f32(v).astype(np.float64), f32(qb).astype(np.float64)
    cf = f32(cf).astype(np.float64)
    got = oproj.band_hit(f32(u), f32(v), f32(cf[:, 0]), f32(cf[:, 1]), f32(cf[:, 2]), f32(qb),
                         f32(X0), f32(X1), f32(Y0), f32(Y1))
    delta, eps = oproj.band_margin(u, v, cf[:, 1], half[:, 0], half[:, 1], W, H)
    must = oproj.tile_hit(u, v, cf[:, 0], cf[:, 1], cf[:, 2], qb * (1 - eps),
                          X0 + delta, X1 - delta, Y0 + delta, Y1 - delta)
    may = oproj.tile_hit(u, v, cf[:, 0], cf[:, 1], cf[:, 2], qb * (1 + eps),
                         X0 - delta, X1 + delta, Y0 - delta, Y1 + delta)
    assert 0.1 * n < must.sum() and may.sum() < 0.9 * n
    assert not np.any(must & ~got), np.nonzero(must & ~got)[0][:5]
    assert not np.any(got & ~may), np.nonzero(got & ~may)[0][:5]
    # the margin is tight enough to mean something: few boxes fall between
    assert (may & ~must).sum() < 1e-3 * n


def test_box_min_q_brute_force():
    # the exact box minimum against a fine grid search over the box, and its
    # special cases: mean inside -> 0; axis-aligned -> separable closed form
    rng = np.random.default_rng(16)
    for _ in range(200):
        a, c = rng.uniform(0.05, 2, 2)
        b = rng.uniform(-0.95, 0.95) * math.sqrt(a * c)
        u, v = rng.uniform(-10, 30, 2)
        X0, Y0 = rng.uniform(0, 10, 2)
        X1, Y1 = X0 + rng.uniform(1, 12), Y0 + rng.uniform(1, 12)
        got = float(oproj.box_min_q(u, v, (a, b, c), X0, X1, Y0, Y1))
        xs, ys = np.meshgrid(np.linspace(X0, X1, 801), np.linspace(Y0, Y1, 801))
        dx, dy = u - xs, v - ys
        brute = (a * dx * dx + 2 * b * dx * dy + c * dy * dy).min()
        assert got <= brute + 1e-12
        assert brute - got <= 2e-3 * (1 + brute)
    assert oproj.box_min_q(5.0, 5.0, (1.0, 0.3, 2.0), 0.5, 10.5, 0.5, 10.5) == 0.0
    # b = 0: q = a dist_x^2 + c dist_y^2 with the per-axis distances to the box
    assert math.isclose(float(oproj.box_min_q(20.0, -3.0, (0.5, 0.0, 2.0), 0.5, 10.5, 0.5, 10.5)),
                        0.5 * 9.5 ** 2 + 2.0 * 3.5 ** 2)


def test_band_span_closed_form_axis_aligned():
    # beta = 0: the ellipse x^2 A + y^2 gamma <= qb; over a band containing dy = 0 the
    # extent is u +- sqrt(qb / A); over a band at distance h it is u +- sqrt((qb - gamma h^2) / A)
    A, g, qb = 0.25, 0.04, 9.0
    ok, xl, xr = oproj.band_span(np.float64(10.0), np.float64(20.0), A, 0.0, g, qb, 15.5, 25.5)
    assert ok and xl == 10.0 - 6.0 and xr == 10.0 + 6.0
    ok, xl, xr = oproj.band_span(np.float64(10.0), np.float64(20.0), A, 0.0, g, qb, 30.0, 40.0)
    assert ok and math.isclose(xr - 10.0, math.sqrt((qb - g * 100.0) / A)) and math.isclose(xl, 20.0 - xr)
    ok, _, _ = oproj.band_span(np.float64(10.0), np.float64(20.0), A, 0.0, g, qb, 36.0, 40.0)
    assert not ok                                    # |dy| > sqrt(qb / gamma) = 15


# ------------------------------------------------------------------ binning and sorting
def _all_pass_records(rect, depth, n):
    """Records whose footprint covers every candidate tile (q_max huge)."""
    return dict(mean2d=np.zeros((n, 2)), conic_f=np.tile([1e-6, 0.0, 1e-6], (n, 1)), q_max=np.full(n, 1e30),
                rect=rect, depth=depth)


def test_bin_and_sort_brute_force():
    rng = np.random.default_rng(6)
    n, gx, gy = 60, 4, 3
    rect = np.zeros((n, 4), np.int64)
    for i in range(n):
        x0, y0 = rng.integers(0, gx), rng.integers(0, gy)
        rect[i] = [x0, y0, rng.integers(x0, gx + 1), rng.integers(y0, gy + 1)]
    depth = rng.choice(np.float32([0.5, 1.0, 1.5, 2.25]), n)     # many exact ties
    full = lambda x: np.full(n, x, np.int64)
    keys, vals, ranges = oras.bin_and_sort(_all_pass_records(rect, depth, n), full(0), full(gx), full(64),
                                           full(48), 16, 16, gx * gy)
    pairs = []
    for i in range(n):
        for ty in range(rect[i, 1], rect[i, 3]):
            for tx in range(rect[i, 0], rect[i, 2]):
                pairs.append((ty * gx + tx, float(depth[i]), i))
    pairs.sort()
    assert [p[2] for p in pairs] == list(vals)
    assert [p[0] for p in pairs] == list((keys >> np.uint64(32)).astype(int))
    assert np.all((keys & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.float32)
                  == np.float32([p[1] for p in pairs]))
    for t in range(gx * gy):
        sel = [k for k, p in enumerate(pairs) if p[0] == t]
        start = sum(1 for p in pairs if p[0] < t)
        assert tuple(ranges[t]) == (start, start + len(sel))


def test_tight_lists_do_not_change_the_image():
    # dropping (record, tile) pairs whose footprint misses the tile leaves Eq. 2 unchanged
    sc = small_scene(1, n=300)
    cam = sc.cameras[0]
    res = opipe.render_view(sc.params(), 0, cam)
    pr = res["proj"]
    n = sc.n
    loose = dict(opipe.proj_record_arrays(pr))
    loose["q_max"] = np.where(pr["visible"], 1e30, 0.0)
    lists_loose = oras.tile_lists(loose, cam.width, cam.height)
    tight = sum(len(l) for l in res["lists"].values())
    assert tight < sum(len(l) for l in lists_loose.values())
    rec = oras.records_to_torch(pr["mean2d"], pr["conic_f"], pr["opacity"], pr["rgb"])
    with torch.no_grad():
        out = oras.rasterize(rec, lists_loose, cam.width, cam.height)
    assert np.abs(out["image"] - res["render"]["image"]).max() < 1e-14
    assert np.abs(out["T_final"] - res["render"]["T_final"]).max() < 1e-14


# ------------------------------------------------------------------ compositing
def _records(n):
    return dict(mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), opacity=np.zeros(n),
                rgb=np.zeros((n, 3)))


def _to_factored(conic):
    conic = np.asarray(conic, np.float64)
    A, B, C = conic[:, 0], conic[:, 1], conic[:, 2]
    return np.stack([A, B / A, C - B * B / A], 1)


def _render(recs, W, H, depth, radius=20, tw=16, th=16, bg=(0, 0, 0)):
    n = len(depth)
    rect = oproj.tile_rect(recs["mean2d"].astype(np.float32), np.full((n, 2), radius, np.float32), tw, th,
                           *oproj.tile_grid(W, H, tw, th))
    arr = dict(mean2d=recs["mean2d"], conic_f=_to_factored(recs["conic"]), q_max=np.full(n, 1e30), rect=rect,
               depth=np.float32(depth))
    lists = oras.tile_lists(arr, W, H, tw, th)
    rt = oras.records_to_torch(recs["mean2d"], arr["conic_f"], recs["opacity"], recs["rgb"])
    with torch.no_grad():
        return oras.rasterize(rt, lists, W, H, tw, th, bg)


def test_single_gaussian_footprint_closed_form():
    s2, o, c = 9.0, 0.8, np.array([0.2, 0.5, 0.9])
    r = _records(1)
    r["mean2d"][0] = [15.3, 17.6]
    r["conic"][0] = [1 / s2, 0, 1 / s2]
    r["opacity"][0] = o
    r["rgb"][0] = c
    out = _render(r, 32, 32, [1.0])
    X, Y = np.meshgrid(np.arange(32) + 0.5, np.arange(32) + 0.5)
    rho2 = (X - 15.3) ** 2 + (Y - 17.6) ** 2
    a = np.minimum(0.99, o * np.exp(-rho2 / (2 * s2)))
    a = np.where(a >= 1 / 255, a, 0.0)
    assert np.abs(out["image"] - c[:, None, None] * a[None]).max() < 1e-14
    assert np.abs(out["T_final"] - (1 - a)).max() < 1e-14


def test_two_gaussian_order_swap():
    r = _records(2)
    r["mean2d"][:] = [[8.0, 8.0], [8.0, 8.0]]
    r["conic"][:] = [[0.01, 0, 0.01]] * 2
    r["opacity"][:] = [0.6, 0.3]
    r["rgb"][:] = [[1, 0, 0], [0, 1, 0]]
    out = _render(r, 16, 16, [1.0, 2.0])
    a1 = 0.6 * math.exp(-0.5 * 0.01 * 0.5)     # pixel (7,7) centre is 0.5 px off in x and y
    a2 = 0.3 * math.exp(-0.5 * 0.01 * 0.5)
    assert abs(out["image"][0, 7, 7] - a1) < 1e-14
    assert abs(out["image"][1, 7, 7] - a2 * (1 - a1)) < 1e-14
    out = _render(r, 16, 16, [2.0, 1.0])
    assert abs(out["image"][0, 7, 7] - a1 * (1 - a2)) < 1e-14
    assert abs(out["image"][1, 7, 7] - a2) < 1e-14


def _brute_force_render(mean2d, conic, opacity, rgb, depth, rect, W, H, tw, th, bg):
    """Per-pixel sequential loop, no vectorisation, no cumulative products."""
    gx = (W + tw - 1) // tw
    img = np.zeros((3, H, W)); Tf = np.ones((H, W))
    stop = np.zeros((H, W), int); nex = np.zeros((H, W), int)
    for j in range(H):
        for i in range(W):
            tx, ty = i // tw, j // th
            cands = [g for g in range(len(depth))
                     if rect[g, 0] <= tx < rect[g, 2] and rect[g, 1] <= ty < rect[g, 3]]
            cands.sort(key=lambda g: (np.float32(depth[g]).view(np.uint32), g))
            T, C = 1.0, np.zeros(3)
            for pos, g in enumerate(cands):
                nex[j, i] = pos + 1
                dx = mean2d[g, 0] - (i + 0.5)
                dy = mean2d[g, 1] - (j + 0.5)
                P = -0.5 * (conic[g, 0] * dx * dx + conic[g, 2] * dy * dy) - conic[g, 1] * dx * dy
                if P > 0:
                    continue
                a = min(0.99, opacity[g] * math.exp(P))
                if a < 1 / 255:
                    continue
                Tn = T * (1 - a)
                if Tn < 1e-4:
                    break
                C += rgb[g] * a * T
                T = Tn
                stop[j, i] = pos + 1
            img[:, j, i] = C + T * np.asarray(bg)
            Tf[j, i] = T
    return img, Tf, stop, nex


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_compositing_matches_brute_force(seed):
    rng = np.random.default_rng(10 + seed)
    n, W, H, tw, th = 16, 32, 24, 16, 8
    mean2d = rng.uniform(-4, 36, (n, 2))
    L = rng.uniform(0.5, 6, (n, 2))
    th_ = rng.uniform(0, math.pi, n)
    conic = np.zeros((n, 3))
    for g in range(n):
        Rm = np.array([[math.cos(th_[g]), -math.sin(th_[g])], [math.sin(th_[g]), math.cos(th_[g])]])
        Ci = np.linalg.inv(Rm @ np.diag(L[g] ** 2) @ Rm.T)
        conic[g] = [Ci[0, 0], Ci[0, 1], Ci[1, 1]]
    opacity = rng.uniform(0.3, 1.0, n)     # >= 0.99 clamp exercised
    rgb = rng.uniform(0, 1, (n, 3))
    depth = rng.choice(np.float32([1.0, 1.25, 2.0, 3.0, 3.5]), n)
    gx, gy = oproj.tile_grid(W, H, tw, th)
    rect = oproj.tile_rect(mean2d.astype(np.float32), np.full((n, 2), 12, np.float32), tw, th, gx, gy)
    arr = dict(mean2d=mean2d, conic_f=_to_factored(conic), q_max=np.full(n, 1e30), rect=rect, depth=depth)
    lists = oras.tile_lists(arr, W, H, tw, th)
    rt = oras.records_to_torch(mean2d, arr["conic_f"], opacity, rgb)
    bg = (0.1, 0.2, 0.3)
    with torch.no_grad():
        out = oras.rasterize(rt, lists, W, H, tw, th, bg)
    img, Tf, stop, nex = _brute_force_render(mean2d, conic, opacity, rgb, depth, rect, W, H,
                                             tw, th, bg)
    assert np.abs(out["image"] - img).max() < 1e-12
    assert np.abs(out["T_final"] - Tf).max() < 1e-12
    assert np.array_equal(out["stop"], stop)
    assert np.array_equal(out["n_examined"], nex)


def test_compositing_invariants_small_scene():
    sc = small_scene(0)
    res = opipe.render_view(sc.params(), 0, sc.cameras[0])
    r = res["render"]
    assert np.all(r["T_final"] >= 1e-4) and np.all(r["T_final"] <= 1.0)
    acc = 1.0 - r["T_final"]
    assert np.all(acc >= 0) and np.all(acc <= 1)
    rgb_max = res["proj"]["rgb"].max(0)
    assert np.all(r["image"] >= 0)
    assert np.all(r["image"] <= rgb_max[:, None, None] * acc[None] + 1e-12)
    assert np.all(r["stop"] <= r["n_examined"])
    # every list is depth-sorted (non-decreasing FP32 depth)
    d32 = res["proj"]["depth"].astype(np.float32)
    for lst in res["lists"].values():
        assert np.all(np.diff(d32[lst]) >= 0)
    assert r["n_examined"].sum() > 0


def test_compositing_transmittance_non_increasing():
    rng = np.random.default_rng(7)
    L = 40
    xy = torch.tensor(rng.uniform(0, 16, (L, 2)))
    conic = torch.tensor(np.tile([0.05, 0.0, 0.05], (L, 1)))        # isotropic: (A, beta, gamma)
    op = torch.tensor(rng.uniform(0.2, 0.9, L))
    rgb = torch.tensor(rng.uniform(0, 1, (L, 3)))
    px = np.arange(16) + 0.5
    prev = np.ones(16)
    for k in range(1, L + 1):
        _, Tf, *_ = oras.composite(px, px, xy[:k], conic[:k], op[:k], rgb[:k], (0, 0, 0))
        Tf = Tf.numpy()
        assert np.all(Tf <= prev + 1e-15)
        prev = Tf


# ------------------------------------------------------------------ gradients (central FD)
def _tiny_scene(seed, n=10, deg=2, W=32, H=32):
    rng = np.random.default_rng(100 + seed)
    cam = look_at_camera((0.3, -0.4, -3.0), W, H, fx=30.0)
    p = dict(means=rng.uniform(-0.6, 0.6, (n, 3)), log_scales=rng.normal(-1.7, 0.3, (n, 3)),
             quats=rng.standard_normal((n, 4)), opacity_logits=rng.normal(0, 0.8, n),
             sh=np.concatenate([rng.uniform(0, 1, (n, 1, 3)),
                                rng.normal(0, 0.2, (n, (deg + 1) ** 2 - 1, 3))], 1))
    w = rng.standard_normal((3, H, W))
    return p, cam, w


def _objective(p, deg, cam, w):
    res = opipe.render_view(p, deg, cam)
    r = res["render"]
    sig = (r["stop"].tobytes(), r["n_examined"].tobytes(), r["n_contrib"].tobytes(),
           res["proj"]["radius"].tobytes(), res["proj"]["rect"].tobytes(),
           res["proj"]["clamped"].tobytes())
    return float((r["image"] * w).sum()), sig


@pytest.mark.parametrize("seed", [0, 1])
def test_pipeline_gradients_central_differences(seed):
    deg = 2
    p, cam, w = _tiny_scene(seed, deg=deg)
    res = opipe.render_view(p, deg, cam, d_image=w)
    g = res["param_grads"]
    _, sig0 = _objective(p, deg, cam, w)
    rng = np.random.default_rng(seed)
    for key in opipe.PARAM_KEYS:
        fd, an = [], []
        flat = p[key].reshape(-1)
        picks = rng.choice(flat.size, min(flat.size, 24), replace=False)
        rejected = 0
        for idx in picks:
            th = flat[idx]
            h = 1e-6 * max(1.0, abs(th))
            q = {k: v.copy() for k, v in p.items()}
            q[key].reshape(-1)[idx] = th + h
            fp, sp = _objective(q, deg, cam, w)
            q[key].reshape(-1)[idx] = th - h
            fm, sm = _objective(q, deg, cam, w)
            if sp != sig0 or sm != sig0:
                rejected += 1
                continue
            fd.append((fp - fm) / (2 * h))
            an.append(g[key].reshape(-1)[idx])
        fd, an = np.array(fd), np.array(an)
        assert len(fd) >= len(picks) // 2, (key, rejected)
        if np.abs(fd).max() == 0:
            assert np.abs(an).max() < 1e-12
            continue
        rel = np.linalg.norm(fd - an) / np.linalg.norm(fd)
        assert rel < 1e-6, (key, rel)


def test_culled_records_have_zero_gradient():
    deg = 0
    p, cam, w = _tiny_scene(3, n=6, deg=deg)
    p["means"][0] = [0.0, 0.0, -2.95]         # just in front of the camera centre (z < near)
    res = opipe.render_view(p, deg, cam, d_image=w)
    assert res["proj"]["radius"][0] == 0
    for k in opipe.PARAM_KEYS:
        assert np.all(res["param_grads"][k][0] == 0)


def test_l1_loss_grad():
    img = np.zeros((3, 2, 2)); tgt = np.zeros((3, 2, 2))
    img[0, 0, 0] = 0.5; tgt[1, 1, 1] = 0.25
    loss, g = l1_loss_grad(img, tgt)
    assert loss == pytest.approx(0.75 / 12)
    assert g[0, 0, 0] == 1 / 12 and g[1, 1, 1] == -1 / 12 and np.count_nonzero(g) == 2


# ------------------------------------------------------------------ densification
def test_stats_accumulation_exact():
    s = 2.0 ** -12
    g = np.array([[0.75 * s, s], [0.0, 0.0], [3 * s, 4 * s]], np.float32)
    acc, cnt = oden.accumulate_stats([g, g], [np.array([1, 1, 0]), np.array([1, 0, 0])],
                                     [(2, 2), (4, 2)])
    # view 0 (W/2 = H/2 = 1): |(0.75s, s)| = 1.25 s; view 1 (W/2 = 2, H/2 = 1): |(1.5s, s)|
    assert acc[0] == np.float32(1.25 * s) + np.float32(math.sqrt(1.5 ** 2 + 1) * s)
    assert acc[1] == 0 and acc[2] == 0
    assert list(cnt) == [2, 1, 0]


def test_split_clone_predicates_boundaries():
    thr = np.float32(2e-4)
    up = np.nextafter(thr, np.float32(1))
    accum = np.array([thr, up, up, up, 0.0, 3 * up], np.float32)
    count = np.array([1, 1, 1, 1, 0, 3], np.int32)
    ls = np.array([[-3, -3, -1], [-3, -3, -1], [-3, -3, -3], [-3, -2.5, -3], [0, 0, 0],
                   [-1, -1, -1]], np.float32)
    thr_s = np.float32(-2.5)
    sp, cl = oden.select(accum, count, ls, oden.ADAPTIVE, thr, thr_s)
    # row 0: avg == thr (not >); row 1: big; row 2: small; row 3: max == thr_s (not big);
    # row 4: count 0; row 5: 3*up/3 rounds to up (> thr)
    assert list(sp) == [False, True, False, False, False, True]
    assert list(cl) == [False, False, True, True, False, False]
    sp, cl = oden.select(accum, count, ls, oden.SPLIT_ONLY, thr, thr_s)
    assert list(sp) == [False, True, False, False, False, True] and not cl.any()
    sp, cl = oden.select(accum, count, ls, oden.ALL_SPLIT, thr, thr_s)
    assert list(sp) == [False, True, True, True, False, True] and not cl.any()
    sp, cl = oden.select(accum, count, ls, oden.ALL_CLONE, thr, thr_s)
    assert list(cl) == [False, True, True, True, False, True] and not sp.any()


def test_adaptive_tau_matches_partition_of_multiset():
    rng = np.random.default_rng(8)
    n = 5000
    logits = rng.normal(-1, 2, n).astype(np.float32)
    logits[::7] = logits[3]                          # ties
    split = rng.uniform(size=n) < 0.1
    clone = ~split & (rng.uniform(size=n) < 0.2)
    for p, tau_u in ((0.03, 0.05), (0.03, 0.9), (0.5, 0.99), (0.999999, 0.999)):
        tau = oden.prune_threshold(logits, split, clone, p=p, tau_u=tau_u)
        multiset = np.concatenate([logits, logits[split | clone]])
        k = min(int(math.floor(multiset.size * p)), multiset.size - 1)
        kth = np.partition(multiset, k)[k]
        want = min(kth, np.float32(math.log(tau_u / (1 - tau_u))))
        assert tau == want
    assert oden.prune_threshold(logits, split, clone, fixed_tau=0.005) == \
        np.float32(math.log(0.005 / 0.995))


def test_philox_known_answer_vectors():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            rows.append((w[0:4], w[4:6], w[6:10]))
    assert len(rows) == 3
    for ctr, key, want in rows:
        assert list(oden.philox4x32_10(ctr, key)) == want


def test_child_normals_distribution():
    z = np.array([oden.child_normals(7, 3, g, c) for g in range(4000) for c in range(2)])
    assert np.abs(z.mean(0)).max() < 0.05
    assert np.abs(z.std(0) - 1).max() < 0.05
    assert abs(np.corrcoef(z.T)[0, 1]) < 0.05


def _dense_params(n, rng):
    return dict(means=rng.normal(0, 1, (n, 3)).astype(np.float32),
                log_scales=rng.normal(-2, 0.5, (n, 3)).astype(np.float32),
                quats=rng.standard_normal((n, 4)).astype(np.float32),
                opacity_logits=rng.normal(0, 1, n).astype(np.float32),
                sh=rng.normal(0, 1, (n, 4, 3)).astype(np.float32))


def test_apply_order_and_counts_brute_force():
    rng = np.random.default_rng(9)
    n = 300
    p = _dense_params(n, rng)
    split = rng.uniform(size=n) < 0.2
    clone = ~split & (rng.uniform(size=n) < 0.3)
    tau = np.float32(-0.5)
    m = {"m": rng.normal(size=(n, 3)).astype(np.float32)}
    out, ex, idx = oden.apply(p, split, clone, tau, seed=11, event=2, extra=m)
    want_src = []
    for g in range(n):
        if p["opacity_logits"][g] >= tau and not split[g]:
            want_src.append(g)
    n_surv = len(want_src)
    for g in range(n):
        if p["opacity_logits"][g] >= tau and clone[g]:
            want_src.append(g)
    for g in range(n):
        if p["opacity_logits"][g] >= tau and split[g]:
            want_src += [g, g]
    assert list(idx["source"]) == want_src
    assert np.array_equal(out["opacity_logits"], p["opacity_logits"][want_src])
    assert np.array_equal(out["sh"], p["sh"][want_src])
    base = len(want_src) - 2 * len(idx["splits"])
    assert np.array_equal(out["log_scales"][base:],
                          p["log_scales"][want_src[base:]] - np.float32(math.log(1.6)))
    assert np.array_equal(out["means"][:base], p["means"][want_src[:base]].astype(np.float64))
    assert np.all(ex["m"][n_surv:] == 0)
    assert np.array_equal(ex["m"][:n_surv], m["m"][want_src[:n_surv]])


def test_split_children_follow_parent_gaussian():
    # many identical parents: child offsets must have covariance R diag(exp(2s)) R^T
    n = 6000
    q = np.array([0.9, 0.2, -0.3, 0.1], np.float32)
    ls = np.array([-1.0, -2.0, -1.5], np.float32)
    p = dict(means=np.zeros((n, 3), np.float32), log_scales=np.tile(ls, (n, 1)),
             quats=np.tile(q, (n, 1)), opacity_logits=np.zeros(n, np.float32),
             sh=np.zeros((n, 1, 3), np.float32))
    out, _, idx = oden.apply(p, np.ones(n, bool), np.zeros(n, bool), np.float32(-10), 5, 1)
    d = out["means"]
    assert d.shape == (2 * n, 3)
    Rm = Rotation.from_quat(q[[1, 2, 3, 0]].astype(np.float64)).as_matrix()
    want = Rm @ np.diag(np.exp(2 * ls.astype(np.float64))) @ Rm.T
    cov = d.T @ d / d.shape[0]
    assert np.abs(cov - want).max() < 0.06 * np.abs(want).max()


def test_anisotropic_footprint_matches_inverse_covariance():
    # Eq. 1 in screen space: alpha(p) = o exp(-1/2 d^T (Sigma' + 0.3 I)^-1 d), d = p - mean2D
    cam = Camera(R=np.eye(3, dtype=np.float32), t=np.zeros(3, np.float32), fx=40.0, fy=44.0,
                 cx=16.0, cy=16.0, width=32, height=32)
    p = _one([0.05, -0.03, 2.0], [math.log(0.25), math.log(0.08), math.log(0.12)],
             quat=(0.8, 0.3, -0.2, 0.5), logit=0.4, sh=[[1.0, 1.0, 1.0]])
    res = opipe.render_view(p, 0, cam)
    pr = res["proj"]
    Sinv = np.linalg.inv(pr["cov2d"][0] + 0.3 * np.eye(2))
    assert abs(Sinv[0, 1]) > 1e-3                       # genuinely anisotropic and rotated
    o = 1 / (1 + math.exp(-0.4))
    c = 0.5 + 1 / (2 * math.sqrt(math.pi))
    X, Y = np.meshgrid(np.arange(32) + 0.5, np.arange(32) + 0.5)
    d = np.stack([X - pr["mean2d"][0, 0], Y - pr["mean2d"][0, 1]], -1)
    q = np.einsum("hwi,ij,hwj->hw", d, Sinv, d)
    a = np.minimum(0.99, o * np.exp(-0.5 * q))
    a = np.where(a >= 1 / 255, a, 0.0)                  # the tile lists lose no such pixel
    assert np.abs(res["render"]["image"][0] - c * a).max() < 1e-13


def test_fp32_band_lists_hold_every_exact_pair():
    # the tile lists of the FP32 decision procedure (band_span over the FP32 tile
    # rectangle), on a 60k-Gaussian view, against the exact FP64 box-minimum test
    # with the derived margin: nothing the exact test keeps is missing, nothing
    # listed lies outside
    from tests.gs_fixtures import exact_list_check, oracle_lists, oracle_records_fp32, scene
    sc = scene("orbit_small")
    cam = sc.cameras[0]
    rec = oracle_records_fp32(sc.params(), sc.sh_degree, cam)
    lists = oracle_lists(rec)
    tiles = np.concatenate([np.full(len(l), t) for t, l in lists.items()])
    recs = np.concatenate([l for l in lists.values()])
    listed, must, between = exact_list_check(rec["mean2d"], rec["conic_f"], rec["q_max"], rec["radius"],
                                             cam.width, cam.height, (16, 16), tiles, recs)
    assert listed > 50_000 and must > 0.99 * listed and between < 1e-3 * listed


def test_provenance_follows_lineage_simulation():
    # two densification events on a tiny set, tracked as a plain object lineage
    # (each Gaussian a record (origin, splits, clones); a split makes two children
    # and removes the parent, a clone adds a copy, a Gaussian whose logit is below
    # tau is dropped with everything it would produce) against the oracle's arrays
    rng = np.random.default_rng(17)
    n = 40
    params = dict(means=rng.normal(size=(n, 3)).astype(np.float32),
                  log_scales=rng.normal(-3, 0.3, (n, 3)).astype(np.float32),
                  quats=rng.normal(size=(n, 4)).astype(np.float32),
                  opacity_logits=rng.normal(size=n).astype(np.float32),
                  sh=rng.normal(size=(n, 1, 3)).astype(np.float32))
    prov = dict(origin=np.arange(n, dtype=np.int32), splits=np.zeros(n, np.int32), clones=np.zeros(n, np.int32))
    lineage = [(g, 0, 0) for g in range(n)]
    tau = np.float32(-1.0)
    for event in range(2):
        m = params["means"].shape[0]
        split = rng.uniform(size=m) < 0.2
        clone = ~split & (rng.uniform(size=m) < 0.2)
        logits = params["opacity_logits"].copy()
        params, _, idx = oden.apply(params, split, clone, tau, seed=5, event=event, provenance=prov)
        prov = idx["provenance"]
        surv, clones, children = [], [], []
        for i, (o, sp, cl) in enumerate(lineage):
            if logits[i] < tau:
                continue
            if split[i]:
                children += [(o, sp + 1, cl), (o, sp + 1, cl)]
            else:
                surv.append((o, sp, cl))
                if clone[i]:
                    clones.append((o, sp, cl + 1))
        lineage = surv + clones + children
        got = list(zip(prov["origin"].tolist(), prov["splits"].tolist(), prov["clones"].tolist()))
        assert got == lineage
        assert params["means"].shape[0] == len(lineage)
    assert any(sp == 2 for _, sp, _ in lineage) or any(cl >= 1 and sp >= 1 for _, sp, cl in lineage)
