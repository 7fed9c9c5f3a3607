"""gs_densify_*: statistics, split/clone masks, the pruning threshold and the
compaction bit-exact against the oracle on the same FP32 tensors."""
import math

import numpy as np
import pytest
import torch

from oracle import densify as oden
from paper_2507_20239_gb300 import rasterizer as R
from paper_2507_20239_gb300 import synth

pytestmark = pytest.mark.gpu


def _stats_inputs(seed, n, V):
    rng = np.random.default_rng(seed)
    # pixel-space mean2D gradients of the size a training view produces
    g = (rng.standard_normal((V, n, 2)) * np.exp(rng.normal(-10, 1.5, (V, n, 1)))).astype(np.float32)
    rad = np.where(rng.uniform(size=(V, n)) < 0.7, rng.integers(1, 30, (V, n)), 0).astype(np.int32)
    return g, rad


def test_densify_accum_bit_exact():
    cams, _ = synth.mixed_resolution_cameras(6)
    n = 50000
    g, rad = _stats_inputs(0, n, len(cams))
    frame = R.Frame(cams)
    acc0 = np.abs(np.random.default_rng(1).normal(0, 1e-3, n)).astype(np.float32)
    cnt0 = np.random.default_rng(2).integers(0, 5, n).astype(np.int32)
    acc = torch.as_tensor(acc0).cuda()
    cnt = torch.as_tensor(cnt0).cuda()
    R.densify_accum(torch.as_tensor(g.reshape(-1, 2)).cuda(), torch.as_tensor(rad.reshape(-1)).cuda(), frame,
                    n, acc, cnt)
    want_a, want_c = oden.accumulate_stats(list(g), list(rad), [(c.width, c.height) for c in cams], acc0, cnt0)
    assert np.array_equal(acc.cpu().numpy(), want_a)
    assert np.array_equal(cnt.cpu().numpy(), want_c)


def _select_inputs(seed, n):
    rng = np.random.default_rng(seed)
    p = synth.surface_scene(seed, n, 1).params()
    count = rng.integers(0, 40, n).astype(np.int32)
    accum = (count * np.exp(rng.normal(math.log(2e-4), 0.6, n))).astype(np.float32)
    # exact boundary cases: avg == threshold, max log-scale == threshold
    thr_s = np.float32(math.log(0.01 * 4.4))
    accum[:50] = np.float32(2e-4) * count[:50].astype(np.float32)
    p["log_scales"][50:100, 1] = thr_s
    p["opacity_logits"][100:200] = p["opacity_logits"][99]
    return p, accum, count, thr_s


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
@pytest.mark.parametrize("adaptive", [False, True])
def test_densify_select_bit_exact(mode, adaptive):
    n = 80000
    p, accum, count, thr_s = _select_inputs(3, n)
    P = {k: torch.as_tensor(v).cuda() for k, v in p.items()}
    kw = dict(prune_ratio=0.03, prune_upper_logit=oden.logit_threshold(0.05)) if adaptive else \
        dict(prune_logit=oden.logit_threshold(0.005))
    cfg = R.densify_cfg(mode=mode, log_scale_threshold=thr_s, **kw)
    split, clone, tau, new_n, ws = R.densify_select(cfg, P, torch.as_tensor(accum).cuda(),
                                                    torch.as_tensor(count).cuda())
    torch.cuda.synchronize()
    ws_, wc = oden.select(accum, count, p["log_scales"], mode, np.float32(2e-4), thr_s)
    assert np.array_equal(split.cpu().numpy().astype(bool), ws_)
    assert np.array_equal(clone.cpu().numpy().astype(bool), wc)
    if adaptive:
        want_tau = oden.prune_threshold(p["opacity_logits"], ws_, wc, p=0.03, tau_u=0.05)
    else:
        want_tau = oden.prune_threshold(p["opacity_logits"], ws_, wc, fixed_tau=0.005)
    assert np.float32(tau.item()) == want_tau
    _, _, idx = oden.apply(p, ws_, wc, want_tau, 0, 0)
    assert int(new_n.item()) == len(idx["source"])


@pytest.mark.parametrize("adaptive", [False, True])
def test_densify_apply_bit_exact(adaptive):
    n = 30000
    p, accum, count, thr_s = _select_inputs(5, n)
    P = {k: torch.as_tensor(v).cuda() for k, v in p.items()}
    kw = dict(prune_ratio=0.03, prune_upper_logit=oden.logit_threshold(0.05)) if adaptive else \
        dict(prune_logit=oden.logit_threshold(0.005))
    cfg = R.densify_cfg(mode=0, log_scale_threshold=thr_s, seed=1234567, event=7, **kw)
    split, clone, tau, new_n, ws = R.densify_select(cfg, P, torch.as_tensor(accum).cuda(),
                                                    torch.as_tensor(count).cuda())
    rng = np.random.default_rng(9)
    m1 = rng.normal(size=(n, 3)).astype(np.float32)
    # provenance from an earlier event: origins and counts of an arbitrary lineage
    prov = dict(origin=rng.integers(0, 10 * n, n).astype(np.int32), splits=rng.integers(0, 4, n).astype(np.int32),
                clones=rng.integers(0, 3, n).astype(np.int32))
    cap = int(new_n.item())
    out, ex, got_n, err = R.densify_apply(cfg, P, 1, split, clone, tau, cap, extra={"m1": torch.as_tensor(m1).cuda()},
                                          ws=ws, prov={k: torch.as_tensor(v).cuda() for k, v in prov.items()})
    torch.cuda.synchronize()
    assert int(err.item()) == 0 and int(got_n.item()) == cap
    ws_, wc = oden.select(accum, count, p["log_scales"], 0, np.float32(2e-4), thr_s)
    want, wex, idx = oden.apply(p, ws_, wc, np.float32(tau.item()), 1234567, 7, extra={"m1": m1},
                                provenance=prov)
    assert cap == len(idx["source"])
    for k in R.PROV_KEYS:
        assert np.array_equal(out[k].cpu().numpy(), idx["provenance"][k]), k
    for k in ("log_scales", "quats", "opacity_logits", "sh"):
        assert np.array_equal(out[k].cpu().numpy(), want[k]), k
    assert np.array_equal(ex["m1"].cpu().numpy(), wex["m1"])
    base = cap - 2 * len(idx["splits"])
    gm = out["means"].cpu().numpy()
    assert np.array_equal(gm[:base], want["means"][:base].astype(np.float32))
    assert np.abs(gm[base:] - want["means"][base:]).max() < 1e-5
    assert len(idx["splits"]) > 10 and len(idx["clones"]) > 10


def test_densify_apply_capacity_overflow():
    n = 5000
    p, accum, count, thr_s = _select_inputs(6, n)
    P = {k: torch.as_tensor(v).cuda() for k, v in p.items()}
    cfg = R.densify_cfg(mode=0, log_scale_threshold=thr_s, prune_logit=-20.0)
    split, clone, tau, new_n, ws = R.densify_select(cfg, P, torch.as_tensor(accum).cuda(),
                                                    torch.as_tensor(count).cuda())
    need = int(new_n.item())
    assert need > n
    out, ex, got_n, err = R.densify_apply(cfg, P, 1, split, clone, tau, need - 1, ws=ws)
    torch.cuda.synchronize()
    assert int(err.item()) == 2 and int(got_n.item()) == need
