"""Pins of the training-step oracles: the D-SSIM loss (oracle/loss.py) and the
Adam / opacity-reset / learning-rate steps (oracle/optim.py) (no GPU)."""
import math

import numpy as np
import pytest

from oracle import loss as oloss
from oracle import optim as oopt


def test_gaussian_window_is_normalised_and_symmetric():
    g = oloss.gaussian_window()
    assert g.shape == (11,) and abs(g.sum() - 1) < 1e-15 and np.allclose(g, g[::-1])
    assert g[5] / g[6] == pytest.approx(math.exp(1 / (2 * 1.5 ** 2)))


def test_ssim_identity_and_constant_closed_form():
    rng = np.random.default_rng(0)
    x = rng.uniform(size=(3, 20, 24))
    assert np.allclose(oloss.ssim_map(x, x).numpy(), 1.0)
    loss, g = oloss.photometric_loss_grad(x, x)
    assert loss == pytest.approx(0.0, abs=1e-12) and np.abs(g).max() < 1e-12
    a, b = 0.3, 0.7
    m = oloss.ssim_map(np.full((1, 30, 30), a), np.full((1, 30, 30), b)).numpy()
    want = (2 * a * b + oloss.SSIM_C1) / (a * a + b * b + oloss.SSIM_C1)   # sigma = 0 inside
    assert np.allclose(m[0, 5:-5, 5:-5], want, atol=1e-12)


def test_photometric_gradient_against_central_differences():
    rng = np.random.default_rng(1)
    x = rng.uniform(size=(3, 9, 11))
    y = rng.uniform(size=(3, 9, 11))
    _, g = oloss.photometric_loss_grad(x, y)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 4, 5), (2, 8, 10), (0, 3, 9), (2, 6, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (oloss.photometric_loss_grad(xp, y)[0] - oloss.photometric_loss_grad(xm, y)[0]) / (2 * h)
        assert fd == pytest.approx(g[idx], rel=1e-5, abs=1e-9)


def test_adam_first_step_and_constant_gradient_closed_form():
    p = np.array([[1.0, -2.0], [0.5, 0.0]])
    g = np.array([[0.3, -4.0], [1e-3, 2.0]])
    z = np.zeros_like(p)
    p1, m1, v1 = oopt.adam_step(p, g, z, z, lr=0.01, t=1, eps=1e-15)
    assert np.allclose(p1, p - 0.01 * np.sign(g), atol=1e-12)          # m_hat = g, v_hat = g^2
    pt, mt, vt = p, z, z
    for t in range(1, 6):
        pt, mt, vt = oopt.adam_step(pt, g, mt, vt, lr=0.01, t=t)
    assert np.allclose(pt, p - 5 * 0.01 * np.sign(g), atol=1e-12)


def test_sparse_adam_leaves_invisible_rows_untouched():
    rng = np.random.default_rng(2)
    p, g, m, v = (rng.normal(size=(6, 3)) for _ in range(4))
    v = np.abs(v)
    vis = np.array([1, 0, 1, 0, 0, 1], bool)
    p1, m1, v1 = oopt.adam_step(p, g, m, v, lr=0.1, t=3, visible=vis)
    assert np.array_equal(p1[~vis], p[~vis]) and np.array_equal(m1[~vis], m[~vis]) and np.array_equal(v1[~vis], v[~vis])
    full = oopt.adam_step(p, g, m, v, lr=0.1, t=3)
    assert np.allclose(p1[vis], full[0][vis])


def test_opacity_reset_and_position_lr():
    lg = np.array([-5.0, 0.0, 3.0])
    cap = math.log(0.01 / 0.99)
    assert np.allclose(oopt.opacity_reset(lg), [-5.0, cap, cap])
    assert oopt.position_lr(100, 1e-3, 1e-5, 500, 1500) == 1e-3
    assert oopt.position_lr(1000, 1e-3, 1e-5, 500, 1500) == pytest.approx(1e-4)
    assert oopt.position_lr(1500, 1e-3, 1e-5, 500, 1500) == pytest.approx(1e-5)
