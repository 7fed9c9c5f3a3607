"""Training loop of the global-to-local densification schedule (Sec. "Global-to-local
framework", "Adaptive Opacity Pruning"), on the library's kernels.

Every step renders one view at the current stage's resolution through the
differentiable rasterizer (autograd.rasterize: gs_project -> gs_bin_sort ->
gs_raster_fwd, backward gs_raster_bwd -> gs_project_bwd with the densification
statistic fused), takes the gradient of Eq. 3's loss, (1 - lambda) L1 + lambda
D-SSIM (gs_photometric_loss_grad; lambda = 0 gives the plain L1 of gs_l1_loss_grad),
and updates the parameters with the fused Adam kernel (gs_adam_step, sparse: only
Gaussians the view saw). The positional learning rate stays constant while training
below full resolution and decays log-linearly after (Sec. "Implementation
details"); the opacities are reset every `opacity_reset_every` steps while
densifying. Every `densify_every` steps inside [densify_from, densify_until] it runs
gs_densify_select and gs_densify_apply on the statistics, carrying the Adam moments
through the compaction (new rows start at zero) and resetting the statistics.

Stages (start step, resolution divisor r, mode): the low-resolution stages run the
split-only global phase; clone is re-enabled at full resolution. The SH degree in
use rises by one every `sh_every` steps up to the coefficients stored.
"""
from __future__ import annotations

import json
import math
from dataclasses import dataclass, field
from typing import Callable, Optional

import numpy as np
import torch

from . import optim as O
from . import rasterizer as R
from .autograd import DensifyStats, rasterize

PARAM_KEYS = R.PARAM_KEYS


@dataclass
class Schedule:
    stages: list = field(default_factory=lambda: [(0, 4, R.DENSIFY_SPLIT_ONLY), (1000, 2, R.DENSIFY_SPLIT_ONLY),
                                                  (2000, 1, R.DENSIFY_ADAPTIVE)])
    total: int = 3000
    densify_from: int = 100
    densify_until: int = 2500
    densify_every: int = 100
    sh_every: int = 750
    grad_threshold: float = 2e-4
    scale_fraction: float = 0.01       # split when the max scale exceeds this fraction of the extent
    prune_tau: float = 0.005            # fixed pruning: opacity below this
    prune_ratio: Optional[float] = None  # adaptive pruning (Sec. "Adaptive Opacity Pruning"): p
    prune_upper_tau: float = 0.05       # adaptive pruning: tau_u
    seed: int = 3
    ssim_lambda: float = 0.2
    sparse_adam: bool = True
    position_lr_final: float = 0.01     # fraction of the initial positional rate reached at the end
    opacity_reset_every: int = 3000
    backward: str = "pixel"            # raster backward: "pixel" or "splat" (same gradients)

    def stage(self, it):
        cur = self.stages[0]
        for s in self.stages:
            if it >= s[0]:
                cur = s
        return cur

    def densify_at(self, it):
        return self.densify_from <= it <= self.densify_until and it % self.densify_every == 0


def default_lrs(extent: float) -> dict:
    """Learning rates of the 3DGS lineage (one rate for all SH coefficients)."""
    return {"means": 1.6e-4 * extent, "log_scales": 5e-3, "quats": 1e-3, "opacity_logits": 5e-2, "sh": 2.5e-3}


class Trainer:
    def __init__(self, params: dict, views: dict, schedule: Schedule, extent: float, lrs: Optional[dict] = None,
                 device="cuda", on_densify: Optional[Callable] = None):
        """params: numpy float32 arrays (sh [N, K, 3] with K = (d+1)^2 for the final
        degree d); views: {r: (cameras, target images [3, H, W])} per stage divisor."""
        self.device = torch.device(device)
        self.sched, self.extent = schedule, float(extent)
        self.lrs = lrs or default_lrs(extent)
        self.max_degree = int(round(math.sqrt(params["sh"].shape[1]))) - 1
        self.frames = {r: [R.Frame([c], device=device) for c in cams] for r, (cams, _) in views.items()}
        self.targets = {r: [torch.as_tensor(np.asarray(t, np.float32)).reshape(-1).to(device) for t in tg]
                        for r, (_, tg) in views.items()}
        self.on_densify = on_densify
        self.history = []
        self.events = []      # per densification: (step, mode, splits, clones, N before, N after)
        self.event = 0
        self._set_params({k: torch.as_tensor(np.ascontiguousarray(v, np.float32)).to(device)
                          for k, v in params.items()}, None)
        # provenance of every Gaussian: its ancestor in the initial set and the
        # splits and clones on its lineage (carried through gs_densify_apply)
        n0 = self.n
        self.prov = {"origin": torch.arange(n0, dtype=torch.int32, device=self.device),
                     "splits": torch.zeros(n0, dtype=torch.int32, device=self.device),
                     "clones": torch.zeros(n0, dtype=torch.int32, device=self.device)}

    # ---------------------------------------------------------------- state
    def _set_params(self, tensors: dict, moments: Optional[dict], step=0):
        self.P = {k: tensors[k].contiguous().requires_grad_(True) for k in PARAM_KEYS}
        self.opt = O.Adam({k: self.P[k].detach() for k in PARAM_KEYS}, self.lrs)
        if moments is not None:
            self.opt.set_moments(moments, self.P)
            self.opt.t = step
        n = self.P["means"].shape[0]
        self.stats = DensifyStats.zeros(n, self.device)

    def full_res_start(self):
        return min(s for s, r, _ in self.sched.stages if r == 1) if any(r == 1 for _, r, _ in self.sched.stages) \
            else self.sched.total

    @property
    def n(self):
        return self.P["means"].shape[0]

    def sh_degree(self, it):
        return min(self.max_degree, it // self.sched.sh_every)

    # ---------------------------------------------------------------- one step
    def step(self, it) -> float:
        _, r, _ = self.sched.stage(it)
        v = it % len(self.frames[r])
        frame, target = self.frames[r][v], self.targets[r][v]
        image, _ = rasterize(self.P, self.sh_degree(it), frame, stats=self.stats, backward=self.sched.backward)
        if self.sched.ssim_lambda > 0:
            d_image, loss = O.photometric_loss_grad(frame, image.detach(), target, self.sched.ssim_lambda)
        else:
            d_image, loss = R.l1_loss_grad(frame, image.detach(), target)
        image.backward(d_image)
        lr0 = self.lrs["means"]
        self.opt.lrs["means"] = lr0 if it <= self.full_res_start() else math.exp(
            math.log(lr0) + min(1.0, (it - self.full_res_start()) / max(1, self.sched.total - self.full_res_start()))
            * math.log(self.sched.position_lr_final))
        grads = {k: self.P[k].grad for k in PARAM_KEYS}
        with torch.no_grad():
            self.opt.step({k: self.P[k].detach() for k in PARAM_KEYS}, grads,
                          radius=self.stats.radius if self.sched.sparse_adam else None, n_views=frame.n_views)
        for k in PARAM_KEYS:
            self.P[k].grad = None
        return loss

    # ---------------------------------------------------------------- densification
    def densify(self, it):
        _, r, mode = self.sched.stage(it)
        thr_s = np.float32(math.log(self.sched.scale_fraction * self.extent))
        prune_logit = np.float32(math.log(self.sched.prune_tau / (1.0 - self.sched.prune_tau)))
        upper_logit = np.float32(math.log(self.sched.prune_upper_tau / (1.0 - self.sched.prune_upper_tau)))
        if self.sched.prune_ratio is None:
            prune = dict(prune_logit=prune_logit)
        else:   # tau = min(k-th smallest logit of the post-densification multiset, logit(tau_u))
            prune = dict(prune_ratio=self.sched.prune_ratio, prune_upper_logit=upper_logit)
        cfg = R.densify_cfg(mode=mode, grad_threshold=self.sched.grad_threshold, log_scale_threshold=thr_s,
                            seed=self.sched.seed, event=self.event, **prune)
        P = {k: self.P[k].detach() for k in PARAM_KEYS}
        split, clone, tau, new_n, ws = R.densify_select(cfg, P, self.stats.accum, self.stats.count)
        extra = {k: v.contiguous() for k, v in self.opt.moments().items()}
        step = self.opt.t
        cap = int(new_n.item())
        out, ex, got_n, err = R.densify_apply(cfg, P, self.sh_degree(it), split, clone, tau, cap, extra=extra,
                                              ws=ws, prov=self.prov)
        if int(err.item()) != 0 or int(got_n.item()) != cap:
            raise RuntimeError("densify: output capacity")
        if self.on_densify is not None:
            self.on_densify(dict(it=it, mode=mode, cfg=cfg, thr_s=thr_s, prune_logit=prune_logit,
                                 prune_ratio=self.sched.prune_ratio, prune_upper_tau=self.sched.prune_upper_tau,
                                 params=P, accum=self.stats.accum, count=self.stats.count, extra=extra,
                                 split=split, clone=clone, tau=tau, out=out, out_extra=ex, seed=self.sched.seed,
                                 event=self.event, prov=self.prov))
        self.events.append((it, int(mode), int(split.sum().item()), int(clone.sum().item()), self.n, cap))
        self.event += 1
        self.prov = {k: out.pop(k) for k in R.PROV_KEYS}
        self._set_params(out, ex, step)

    def provenance_summary(self) -> dict:
        """Shares of the current Gaussians by lineage (the split/clone analysis of
        Sec. "Global-to-local framework"): untouched initial Gaussians, those with a
        clone, with a split, with both, and the initial Gaussians with descendants."""
        s, c = self.prov["splits"], self.prov["clones"]
        n = max(1, self.n)
        return {"n": self.n, "untouched": float(((s == 0) & (c == 0)).sum()) / n,
                "with_clone": float(((c > 0) & (s == 0)).sum()) / n,
                "with_split": float(((s > 0) & (c == 0)).sum()) / n,
                "with_both": float(((s > 0) & (c > 0)).sum()) / n,
                "max_splits": int(s.max().item()) if self.n else 0,
                "max_clones": int(c.max().item()) if self.n else 0,
                "origins_alive": int(torch.unique(self.prov["origin"]).numel())}

    # ---------------------------------------------------------------- checkpoint / resume
    def state_dict(self, next_it: int) -> dict:
        """Everything training needs to continue at iteration next_it, on the host:
        parameters, Adam moments and step count, densification statistics,
        provenance, the densification event counter and the history so far."""
        host = lambda t: t.detach().cpu().numpy()
        st = {f"param.{k}": host(self.P[k]) for k in PARAM_KEYS}
        st.update({f"moment.{k}": host(v) for k, v in self.opt.moments().items()})
        st.update({"stats.accum": host(self.stats.accum), "stats.count": host(self.stats.count)})
        st.update({f"prov.{k}": host(v) for k, v in self.prov.items()})
        st["meta"] = np.array(json.dumps({"next_it": int(next_it), "adam_t": int(self.opt.t), "event": int(self.event),
                                          "history": self.history, "events": self.events,
                                          "lrs": self.lrs}))
        return st

    def save(self, path: str, next_it: int):
        """Write state_dict(next_it) to path (numpy .npz, uncompressed)."""
        np.savez(path, **self.state_dict(next_it))

    def load(self, path: str) -> int:
        """Restore a state written by save(); returns the iteration to continue at."""
        z = np.load(path, allow_pickle=False)
        meta = json.loads(str(z["meta"]))
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(self.device)
        params = {k: dev(z[f"param.{k}"]) for k in PARAM_KEYS}
        moments = {k[len("moment."):]: dev(z[k]) for k in z.files if k.startswith("moment.")}
        self._set_params(params, moments, meta["adam_t"])
        self.stats.accum.copy_(dev(z["stats.accum"]))
        self.stats.count.copy_(dev(z["stats.count"]))
        self.prov = {k: dev(z[f"prov.{k}"]) for k in R.PROV_KEYS}
        self.event = int(meta["event"])
        self.history = [tuple(h) for h in meta["history"]]
        self.events = [tuple(e) for e in meta["events"]]
        self.lrs = dict(meta["lrs"])
        self.opt.lrs = dict(self.lrs)
        return int(meta["next_it"])

    def run(self, log_every: int = 100, start: int = 1, stop: Optional[int] = None,
            checkpoint: Optional[str] = None, checkpoint_every: int = 0):
        """Iterations start..stop (1-based, default to the schedule's end); with
        checkpoint and checkpoint_every, the state is saved every checkpoint_every
        iterations (after that iteration's densification and reset)."""
        stop = self.sched.total if stop is None else stop
        for it in range(start, stop + 1):
            loss = self.step(it - 1)
            if self.sched.densify_at(it):
                self.densify(it)
            if self.sched.opacity_reset_every and it % self.sched.opacity_reset_every == 0 and \
                    it <= self.sched.densify_until:
                O.opacity_reset({k: self.P[k].detach() for k in PARAM_KEYS}, self.opt)
            if it % log_every == 0 or it == self.sched.total:
                self.history.append((it, self.n, float(loss[0].item())))
            if checkpoint and checkpoint_every and it % checkpoint_every == 0:
                self.save(checkpoint, it + 1)
        return self.history


def scaled_camera(cam, width: int, height: int):
    """The camera whose pixel grid is D_r's output grid: intrinsics scaled by the
    actual size ratios (output pixel j covers input [j s, (j + 1) s))."""
    from . import synth
    sx, sy = width / cam.width, height / cam.height
    return synth.Camera(cam.R, cam.t, cam.fx * sx, cam.fy * sy, cam.cx * sx, cam.cy * sy, width, height)


def energy_stages(cameras, full_targets, K: int, T_densify: int, device="cuda"):
    """Stages and per-scale views from the energy schedule of the full-resolution
    targets: scale r > 1 runs the split-only phase on D_r(targets), r = 1 the
    adaptive phase. Returns (stages [(start, r, mode)], views {r: (cams, targets)},
    (E, T))."""
    from . import schedule as S
    E, T, st = S.energy_schedule(full_targets, K=K, T_densify=T_densify, device=device)
    stages = [(start, r, R.DENSIFY_SPLIT_ONLY if r > 1 else R.DENSIFY_ADAPTIVE) for start, _, r in st]
    if not stages or stages[-1][1] != 1:
        stages.append((T_densify, 1, R.DENSIFY_ADAPTIVE))
    views = {}
    for _, r, _ in stages:
        if r in views:
            continue
        imgs = [torch.as_tensor(np.asarray(t, np.float32)).to(device) for t in full_targets]
        small = [S.downscale(t, r).cpu().numpy() if r > 1 else t.cpu().numpy() for t in imgs]
        cams = [scaled_camera(c, im.shape[2], im.shape[1]) for c, im in zip(cameras, small)]
        views[r] = (cams, small)
    return stages, views, (E, T)


def render_targets(gt_params: dict, sh_degree: int, cameras, device="cuda") -> list:
    """Target images of a ground-truth scene rendered by the library's forward."""
    P = R.to_device_params(gt_params, device)
    out = []
    for cam in cameras:
        frame = R.Frame([cam], device=device)
        proj = R.project(P, sh_degree, frame)
        bins = R.bin_sort(proj, frame)
        img, _, _ = R.raster_fwd(proj, bins, frame)
        out.append(frame.view_image(img, 0).cpu().numpy())
    return out


def orbit_views(n_views: int, width: int, height: int, f: float, divisors=(4, 2, 1), radius=4.0, elevation=15.0):
    """n_views orbit cameras per resolution divisor r (W/r rounded half up)."""
    from . import synth
    out = {}
    for r in divisors:
        w, h = int(math.floor(width / r + 0.5)), int(math.floor(height / r + 0.5))
        out[r] = [synth.orbit_camera(radius, 2 * math.pi * k / n_views, elevation, w, h, f / r) for k in range(n_views)]
    return out


def main(argv=None):
    """The densification trajectory of the training-loop workload: targets rendered
    from a 1.5M-Gaussian scene (seed 13) at 8 orbit views per resolution, training
    from 100k Gaussians (seed 3) for 3,000 steps; prints the (step, N, loss) history."""
    import argparse
    import json
    from . import synth
    ap = argparse.ArgumentParser()
    ap.add_argument("--gt", type=int, default=1_500_000)
    ap.add_argument("--init", type=int, default=100_000)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--width", type=int, default=1246)
    ap.add_argument("--height", type=int, default=826)
    ap.add_argument("--views", type=int, default=8)
    ap.add_argument("--init-log-scale", type=float, default=-4.0,
                    help="mean log-scale of the initial Gaussians (the generator's default: -4)")
    ap.add_argument("--init-mode", choices=["generator", "sfm"], default="generator",
                    help="initial Gaussians: a fresh draw of the scene generator (seed 3), or an "
                         "SfM-like point set taken from the ground truth (synth.sfm_like_init)")
    ap.add_argument("--grad-threshold", type=float, default=2e-4)
    ap.add_argument("--energy", type=int, default=0, metavar="K",
                    help="derive the stages from the targets' energy schedule with scales 1..K "
                         "(default: fixed thirds at 1/4, 1/2, full resolution)")
    ap.add_argument("--backward", choices=["pixel", "splat"], default="pixel",
                    help="raster backward: per-pixel or per-splat (same gradients)")
    ap.add_argument("--prune-ratio", type=float, default=None, metavar="P",
                    help="adaptive opacity pruning with ratio P (default: fixed tau 0.005)")
    ap.add_argument("--prune-upper", type=float, default=0.05, metavar="TAU_U",
                    help="adaptive pruning's upper bound on tau")
    ap.add_argument("--checkpoint", default=None, metavar="PATH",
                    help="save the training state here every --checkpoint-every iterations")
    ap.add_argument("--checkpoint-every", type=int, default=500)
    ap.add_argument("--resume", default=None, metavar="PATH", help="continue from a saved training state")
    args = ap.parse_args(argv)
    s = args.steps / 3000.0
    sched = Schedule(stages=[(0, 4, R.DENSIFY_SPLIT_ONLY), (int(1000 * s), 2, R.DENSIFY_SPLIT_ONLY),
                             (int(2000 * s), 1, R.DENSIFY_ADAPTIVE)], total=args.steps,
                     densify_until=int(2500 * s), sh_every=max(1, int(750 * s)),
                     grad_threshold=args.grad_threshold, backward=args.backward,
                     prune_ratio=args.prune_ratio, prune_upper_tau=args.prune_upper)
    gt = synth.surface_scene(13, args.gt, 3)
    energy = None
    if args.energy:
        full = orbit_views(args.views, args.width, args.height, float(args.width), divisors=(1,))[1]
        targets = render_targets(gt.params(), 3, full)
        stages, views, (E, T) = energy_stages(full, targets, args.energy, sched.densify_until)
        sched.stages = stages
        energy = {"E": [float(e) for e in E], "T": [int(t) for t in T], "stages": stages}
    else:
        cams = orbit_views(args.views, args.width, args.height, float(args.width))
        views = {r: (c, render_targets(gt.params(), 3, c)) for r, c in cams.items()}
    if args.init_mode == "sfm":
        init = synth.sfm_like_init(gt, args.init, seed=3).params()
    else:
        init = synth.surface_scene(3, args.init, 3, log_scale_mean=args.init_log_scale).params()
    tr = Trainer(init, views, sched, extent=1.1 * 4.0)
    start = tr.load(args.resume) if args.resume else 1
    hist = tr.run(start=start, checkpoint=args.checkpoint, checkpoint_every=args.checkpoint_every)
    n_split = sum(e[2] for e in tr.events)
    n_clone = sum(e[3] for e in tr.events)
    print(json.dumps({"history": hist, "final_n": tr.n, "events": tr.events,
                      "new_from_clone": n_clone / max(1, n_clone + 2 * n_split), "init_log_scale": args.init_log_scale,
                      "init_mode": args.init_mode, "provenance": tr.provenance_summary(),
                      "grad_threshold": args.grad_threshold, "prune_ratio": args.prune_ratio,
                      "prune_upper": args.prune_upper, "energy_schedule": energy}))


if __name__ == "__main__":
    main()
