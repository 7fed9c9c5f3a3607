"""Pins of the energy-schedule oracle (oracle/schedule.py) against closed forms,
brute force and the filter's defining properties (no GPU)."""
import math

import numpy as np
import pytest

from oracle import schedule as osch


def test_downscale_weights_are_a_normalised_triangle():
    W = osch.aa_weights(12, 6)                      # scale 2
    assert np.allclose(W.sum(1), 1.0)
    # interior row: taps at c-1.5 .. c+1.5 with weights 1/8, 3/8, 3/8, 1/8
    c = 2 * 2 + 0.5
    assert np.allclose(W[2, 3:7], [0.125, 0.375, 0.375, 0.125]) and W[2, :3].sum() == 0 and W[2, 7:].sum() == 0
    # scale 1 is the identity
    assert np.allclose(osch.aa_weights(7, 7), np.eye(7))


def test_downscale_keeps_constants_and_interior_ramps():
    img = np.full((3, 40, 60), 0.37)
    assert np.allclose(osch.downscale(img, 4), 0.37)
    x = np.arange(64, dtype=np.float64)
    ramp = np.broadcast_to(0.1 + 0.01 * x, (1, 32, 64))
    d = osch.downscale(ramp, 2)
    j = np.arange(2, 30)                            # away from the borders
    assert np.allclose(d[0, 5, j], 0.1 + 0.01 * ((j + 0.5) * 2 - 0.5))


def test_nyquist_checkerboard_vanishes_inside_after_anti_aliasing():
    y, x = np.mgrid[0:64, 0:96]
    cb = ((-1.0) ** (x + y))[None]
    d = osch.downscale(cb, 2)
    assert np.abs(d[0, 1:-1, 1:-1]).max() < 1e-12
    # without the filter (point sampling) the pattern would keep its energy
    assert osch.spectrum_l1(cb) == pytest.approx(64 * 96)
    assert osch.spectrum_l1(d) < 0.05 * osch.spectrum_l1(cb) * 4


def test_spectrum_l1_closed_forms_and_brute_force():
    H, W = 24, 30
    assert osch.spectrum_l1(np.full((2, H, W), 0.5)) == pytest.approx(2 * 0.5 * H * W)
    x = np.arange(W)
    cosine = np.broadcast_to(np.cos(2 * math.pi * 3 * x / W), (1, H, W))
    assert osch.spectrum_l1(cosine) == pytest.approx(H * W)          # two peaks of H W / 2
    rng = np.random.default_rng(0)
    img = rng.normal(size=(1, 5, 6))
    k, n = np.arange(5), np.arange(6)
    F = np.zeros((5, 6), complex)
    for a in range(5):
        for b in range(6):
            F[a, b] = (img[0] * np.exp(-2j * math.pi * (np.outer(a * k / 5, np.ones(6)) +
                                                         np.outer(np.ones(5), b * n / 6)))).sum()
    assert osch.spectrum_l1(img) == pytest.approx(np.abs(F).sum(), rel=1e-12)


def test_energy_normalisation_and_constant_image_schedule():
    img = np.full((3, 80, 120), 0.25)               # sizes divisible by 1, 2, 4, 8
    E = osch.energies([img], 8)
    for r in (1, 2, 4, 8):
        assert E[r - 1] == pytest.approx(3 * 0.25 * 80 * 120)
    T = osch.iterations(E, 25000)
    assert T[0] == 25000 and T[1] == 25000        # all energy at DC: every scale gets everything


def test_iteration_rounding_clamp_and_monotonicity():
    E = np.array([10.0, 8.0, 8.5, 3.0, 0.0])
    T = osch.iterations(E, 100)
    assert list(T) == [100, 80, 80, 30, 0]
    assert list(osch.iterations(np.array([4.0, 1.0]), 10)) == [10, 3]     # 2.5 rounds half up
    assert osch.stages(T) == [(0, 30, 4), (30, 80, 3), (80, 100, 1)]


def test_natural_image_schedule_is_coarse_to_fine():
    rng = np.random.default_rng(1)
    y, x = np.mgrid[0:96, 0:128]
    img = np.stack([np.sin(x / 9.0) + 0.3 * rng.normal(size=x.shape) for _ in range(3)])
    E = osch.energies([img], 4)
    assert E[0] > E[1] > E[2] > E[3] > 0
    T = osch.iterations(E, 1000)
    assert T[0] == 1000 and all(T[i] >= T[i + 1] for i in range(3))
