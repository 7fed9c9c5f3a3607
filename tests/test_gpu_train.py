"""The training-loop workload, shortened: the global-to-local schedule (split-only
at 1/4 and 1/2 resolution, clone re-enabled at full resolution, prune below
opacity 0.005, SH degree rising) trained on the library's kernels, with every
densification event checked against the oracle on the same FP32 tensors: split and
clone masks, the prune threshold and the whole compaction (parameters and the Adam
moments carried through it) bit-exact, split children's means within 1e-5; once
with fixed and once with adaptive opacity pruning."""
import math

import numpy as np
import pytest
import torch

from oracle import densify as oden
from paper_2507_20239_gb300 import rasterizer as R
from paper_2507_20239_gb300 import synth
from paper_2507_20239_gb300.train import Schedule, Trainer, orbit_views, render_targets

pytestmark = pytest.mark.gpu


def _checker(events, adaptive):
    """on_densify callback: the event recomputed by the oracle on the same FP32 tensors."""
    def check(ev):
        np_ = lambda t: t.detach().cpu().numpy()
        p = {k: np_(v) for k, v in ev["params"].items()}
        accum, count = np_(ev["accum"]), np_(ev["count"])
        ws_, wc = oden.select(accum, count, p["log_scales"], ev["mode"], np.float32(2e-4), ev["thr_s"])
        assert np.array_equal(np_(ev["split"]).astype(bool), ws_)
        assert np.array_equal(np_(ev["clone"]).astype(bool), wc)
        if adaptive:
            assert ev["prune_ratio"] == 0.03 and ev["prune_upper_tau"] == 0.05
            tau = oden.prune_threshold(p["opacity_logits"], ws_, wc, p=0.03, tau_u=0.05)
        else:
            tau = oden.prune_threshold(p["opacity_logits"], ws_, wc, fixed_tau=0.005)
        assert np.float32(ev["tau"].item()) == tau
        extra = {k: np_(v) for k, v in ev["extra"].items()}
        prov = {k: np_(v) for k, v in ev["prov"].items()}
        want, wex, idx = oden.apply(p, ws_, wc, tau, ev["seed"], ev["event"], extra=extra, provenance=prov)
        out = {k: np_(v) for k, v in ev["out"].items()}
        for k in R.PROV_KEYS:
            assert np.array_equal(out[k], idx["provenance"][k]), k
        assert out["means"].shape[0] == len(idx["source"])
        for k in ("log_scales", "quats", "opacity_logits", "sh"):
            assert np.array_equal(out[k], want[k]), k
        for k in extra:
            assert np.array_equal(np_(ev["out_extra"][k]), wex[k]), k
        base = out["means"].shape[0] - 2 * len(idx["splits"])
        assert np.array_equal(out["means"][:base], want["means"][:base].astype(np.float32))
        if base < out["means"].shape[0]:
            assert np.abs(out["means"][base:] - want["means"][base:]).max() < 1e-5
        n_pruned = len(p["means"]) + int(wc.sum()) + int(ws_.sum()) - len(idx["source"])
        events.append((ev["it"], ev["mode"], int(ws_.sum()), int(wc.sum()), len(idx["source"]), n_pruned,
                       float(tau)))
    return check


def test_global_to_local_training_with_checked_densification():
    events = []
    check = _checker(events, adaptive=False)

    cams = orbit_views(4, 623, 413, 623.0)
    gt = synth.surface_scene(13, 200_000, 3)
    views = {r: (c, render_targets(gt.params(), 3, c)) for r, c in cams.items()}
    init = synth.surface_scene(3, 20_000, 3).params()
    sched = Schedule(stages=[(0, 4, R.DENSIFY_SPLIT_ONLY), (200, 2, R.DENSIFY_SPLIT_ONLY),
                             (400, 1, R.DENSIFY_ADAPTIVE)], total=600, densify_until=500, sh_every=150)
    tr = Trainer(init, views, sched, extent=1.1 * 4.0, on_densify=check)
    hist = tr.run(log_every=50)
    assert [e[0] for e in events] == [100, 200, 300, 400, 500]
    assert all(e[1] == R.DENSIFY_SPLIT_ONLY for e in events[:3]) and events[3][1] == R.DENSIFY_ADAPTIVE
    assert all(e[3] == 0 for e in events[:3])                     # no clones in the split-only phase
    assert sum(e[2] for e in events) > 0 and sum(e[3] for e in events[3:]) > 0
    assert tr.n > 20_000
    assert hist[-1][2] < hist[0][2]                                # the L1 loss went down


def test_adaptive_opacity_pruning_in_training():
    """The same schedule with adaptive pruning (p = 0.03, tau_u = 0.05): every event's
    threshold is the k-th smallest logit of the post-densification multiset, capped
    at logit(tau_u), and the whole event is bit-exact against the oracle."""
    events = []
    cams = orbit_views(4, 312, 207, 312.0)
    gt = synth.surface_scene(13, 60_000, 3)
    views = {r: (c, render_targets(gt.params(), 3, c)) for r, c in cams.items()}
    init = synth.surface_scene(3, 10_000, 3).params()
    sched = Schedule(stages=[(0, 4, R.DENSIFY_SPLIT_ONLY), (200, 2, R.DENSIFY_SPLIT_ONLY),
                             (400, 1, R.DENSIFY_ADAPTIVE)], total=600, densify_until=500, sh_every=150,
                     prune_ratio=0.03, prune_upper_tau=0.05)
    tr = Trainer(init, views, sched, extent=1.1 * 4.0, on_densify=_checker(events, adaptive=True))
    hist = tr.run(log_every=100)
    assert [e[0] for e in events] == [100, 200, 300, 400, 500]
    # adaptive pruning removes at most 3% of the post-densification set at an event
    # (fewer when the cap logit(tau_u) binds)
    assert sum(e[5] for e in events) > 0
    assert all(e[5] <= math.floor(0.03 * (e[4] + e[5])) for e in events)
    assert hist[-1][2] < hist[0][2]


def test_checkpoint_resume_continues_training(tmp_path):
    """Training saved at iteration 150 and resumed in a fresh trainer: the restored
    state (parameters, Adam moments and step count, densification statistics,
    provenance, event counter, history) equals the saved one bit for bit, and the
    resumed run densifies at the same iterations as the uninterrupted one, to the
    same size up to the run-to-run spread of the atomically summed gradients."""
    from paper_2507_20239_gb300 import train as T
    gt = synth.surface_scene(13, 60_000, 3)
    cams = T.orbit_views(4, 320, 212, 320.0)
    views = {r: (c, T.render_targets(gt.params(), 3, c)) for r, c in cams.items()}
    init = synth.sfm_like_init(gt, 8_000, seed=3).params()
    sched = T.Schedule(stages=[(0, 4, R.DENSIFY_SPLIT_ONLY), (100, 2, R.DENSIFY_SPLIT_ONLY),
                               (200, 1, R.DENSIFY_ADAPTIVE)], total=300, densify_from=50,
                       densify_until=250, densify_every=50, sh_every=75)
    path = str(tmp_path / "state.npz")
    a = T.Trainer(init, views, sched, extent=1.1 * 4.0)
    a.run(log_every=50, stop=150, checkpoint=path, checkpoint_every=150)
    saved = a.state_dict(151)
    b = T.Trainer(init, views, sched, extent=1.1 * 4.0)
    start = b.load(path)
    assert start == 151
    restored = b.state_dict(151)
    assert set(saved) == set(restored)
    for k in saved:
        assert np.array_equal(saved[k], restored[k]), k
    a.run(log_every=50, start=151)
    b.run(log_every=50, start=151)
    assert [e[0] for e in a.events] == [e[0] for e in b.events] == [50, 100, 150, 200, 250]
    assert abs(a.n - b.n) <= 0.02 * a.n, (a.n, b.n)
    assert b.history[-1][0] == 300 and b.history[-1][2] < b.history[0][2]
    assert int(b.prov["origin"].max()) < 8_000 and int(b.prov["origin"].min()) >= 0
