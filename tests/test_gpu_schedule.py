"""gs_downscale / gs_spectrum_l1 and the energy-guided schedule built on them,
against the FP64 oracle (oracle/schedule.py) on the same FP32 images."""
import numpy as np
import pytest
import torch

from oracle import schedule as osch
from paper_2507_20239_gb300 import schedule as S

pytestmark = pytest.mark.gpu


def _image(seed, C, H, W):
    rng = np.random.default_rng(seed)
    y, x = np.mgrid[0:H, 0:W]
    base = 0.5 + 0.3 * np.sin(x / 7.0 + seed) * np.cos(y / 11.0)
    return np.stack([base + 0.1 * rng.normal(size=(H, W)) for _ in range(C)]).astype(np.float32)


@pytest.mark.parametrize("r", [1, 2, 3, 4, 8])
def test_downscale_matches_oracle(r):
    img = _image(0, 3, 207, 311)
    got = S.downscale(torch.as_tensor(img).cuda(), r).cpu().numpy()
    want = osch.downscale(img, r)
    assert got.shape == want.shape == (3, osch.downscaled_size(207, r), osch.downscaled_size(311, r))
    assert np.abs(got - want).max() < 1e-5


@pytest.mark.parametrize("shape", [(3, 413, 623), (1, 37, 53), (2, 1, 1)])
def test_spectrum_l1_matches_oracle(shape):
    img = _image(1, *shape)
    got = S.spectrum_l1(torch.as_tensor(img).cuda())
    want = osch.spectrum_l1(img)
    assert abs(got - want) <= 1e-5 * want


def test_energy_schedule_matches_oracle():
    imgs = [_image(s, 3, 413, 623) for s in (2, 3)]
    E, T, st = S.energy_schedule(imgs, K=8, T_densify=25000)
    Eo = osch.energies(imgs, 8)
    assert np.all(np.abs(E - Eo) <= 1e-5 * Eo)
    To = osch.iterations(Eo, 25000)
    # a T_r may differ by one only where E_r / E_1 T_densify lies within the FP32
    # error of a rounding boundary
    frac = Eo / Eo[0] * 25000 + 0.5
    near = np.abs(frac - np.round(frac)) < 1e-5 * 25000
    assert np.all((T == To) | (near & (np.abs(T - To) == 1)))
    assert st == osch.stages(To) or near.any()
    assert T[0] == 25000 and all(T[i] >= T[i + 1] for i in range(7))


def test_spectrum_rejects_oversized_images():
    assert S.lib().gs_spectrum_workspace_size(3, 4097, 100) == 0
    with pytest.raises(RuntimeError):
        S.spectrum_l1(torch.zeros(1, 4097, 8, device="cuda"))


def test_energy_schedule_drives_training():
    from paper_2507_20239_gb300 import rasterizer as R, synth
    from paper_2507_20239_gb300.train import Schedule, Trainer, energy_stages, orbit_views, render_targets
    full = orbit_views(2, 320, 212, 320.0, divisors=(1,))[1]
    gt = synth.surface_scene(13, 60_000, 3)
    targets = render_targets(gt.params(), 3, full)
    stages, views, (E, T) = energy_stages(full, targets, 4, 300)
    assert stages[0][0] == 0 and stages[-1][1] == 1
    assert [s[1] for s in stages] == sorted((s[1] for s in stages), reverse=True)      # coarse to fine
    assert all(m == R.DENSIFY_SPLIT_ONLY for _, r, m in stages if r > 1)
    for r, (cams, imgs) in views.items():
        assert imgs[0].shape == (3, S.downscaled_size(212, r), S.downscaled_size(320, r))
        assert cams[0].width == imgs[0].shape[2]
    sched = Schedule(stages=stages, total=400, densify_until=300, sh_every=100)
    tr = Trainer(synth.surface_scene(3, 10_000, 3).params(), views, sched, extent=4.4)
    hist = tr.run(log_every=100)
    assert tr.event == 3 and hist[-1][2] < hist[0][2]
