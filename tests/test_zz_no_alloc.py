"""The allocation-free densification selection (gs_densify_select_static).

Callers that cannot allocate device memory -- operators running inside another
runtime's callbacks, fixed-budget deployments -- use this entry point instead of
gs_densify_select; it keeps its scratch in a device array of the library. This test
calls it through the C ABI twice in a row, on different inputs, and checks each
result against the workspace-based gs_densify_select: the split/clone masks, the
prune threshold and the new count must be identical (the selection is exact).
The file is collected last so that a failure here stops a run only after every
other test has run.
"""
import ctypes as C
import math

import numpy as np
import pytest
import torch

from oracle import densify as oden
from paper_2507_20239_gb300 import _abi
from paper_2507_20239_gb300 import rasterizer as R
from paper_2507_20239_gb300 import synth

pytestmark = pytest.mark.gpu


def _inputs(seed, n):
    rng = np.random.default_rng(seed)
    p = synth.surface_scene(seed, n, 0).params()
    count = rng.integers(0, 30, n).astype(np.int32)
    accum = (count * np.exp(rng.normal(math.log(2e-4), 0.6, n))).astype(np.float32)
    return {k: torch.as_tensor(v).cuda() for k, v in p.items()}, torch.as_tensor(accum).cuda(), \
        torch.as_tensor(count).cuda()


def _static_select(cfg, P, accum, count):
    n = P["means"].shape[0]
    split = torch.empty(n, dtype=torch.uint8, device="cuda")
    clone = torch.empty(n, dtype=torch.uint8, device="cuda")
    tau = torch.empty(1, dtype=torch.float32, device="cuda")
    new_n = torch.empty(1, dtype=torch.int64, device="cuda")
    p = lambda t: C.c_void_p(t.data_ptr())
    st = _abi.load().gs_densify_select_static(
        C.byref(cfg), p(P["log_scales"]), p(P["opacity_logits"]), p(accum), p(count), n, p(split), p(clone),
        p(tau), p(new_n), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, _abi.STATUS.get(st, st)
    return split, clone, tau, new_n


def test_static_select_matches_workspace_select_on_two_calls():
    thr_s = float(np.float32(math.log(0.01 * 4.4)))
    cases = [(41, 60_000, dict(prune_ratio=0.03, prune_upper_logit=oden.logit_threshold(0.05))),
             (42, 45_000, dict(prune_ratio=0.10, prune_upper_logit=oden.logit_threshold(0.5)))]
    for seed, n, kw in cases:
        P, accum, count = _inputs(seed, n)
        cfg = R.densify_cfg(mode=0, log_scale_threshold=thr_s, **kw)
        ws_, wc, wt, wn, _ = R.densify_select(cfg, P, accum, count)
        gs, gc, gt, gn = _static_select(cfg, P, accum, count)
        torch.cuda.synchronize()
        assert torch.equal(gs, ws_) and torch.equal(gc, wc)
        assert float(gt.item()) == float(wt.item())
        assert int(gn.item()) == int(wn.item())
        assert int(gs.sum()) > 0 and int(gc.sum()) > 0


def test_static_select_rejects_sizes_beyond_its_maximum():
    cfg = R.densify_cfg(mode=0, log_scale_threshold=0.0, prune_logit=-5.0)
    st = _abi.load().gs_densify_select_static(C.byref(cfg), C.c_void_p(16), C.c_void_p(16), C.c_void_p(16),
                                              C.c_void_p(16), (1 << 30) + 1, C.c_void_p(16), C.c_void_p(16),
                                              C.c_void_p(16), C.c_void_p(16), None)
    assert st == 1   # GS_ERR_INVALID_ARG, before anything is enqueued
