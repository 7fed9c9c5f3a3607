"""FP64 CPU oracle for the Gaussian-splatting hot path -- TEST INFRASTRUCTURE ONLY.

A plain, slow restatement of what the differentiable tile rasterizer and the
densification bookkeeping compute, written from the paper (Sec. "Preliminary":
Eq. 1 Gaussian, the EWA projection Sigma' = J W Sigma W^T J^T, Eq. 2 front-to-back
alpha compositing; the densification rule; Sec. "Adaptive Opacity Pruning").
Where the paper is silent, the reading taken is the one listed in the design notes
(near plane 0.2, 0.3 px^2 low-pass dilation, the 1/255-floor footprint, 1/255 alpha floor,
alpha clamp 0.99, transmittance cutoff 1e-4, ...); each function states it.

Rules this package obeys:
  * It shares no code, constants or tables with the CUDA library and never
    imports it; the CUDA library never imports this package.
  * Only tests, the smoke check and the benchmark's CPU-baseline leg use it.
    The product path must never route through it.
  * Floating point is FP64, except where floating point decides an integer that
    must match bit-exactly (tile rectangles from FP32 inputs, FP32 depth sort
    keys, densification predicates on FP32 statistics): there the decision is
    taken in FP32, the precision of the data it is applied to.
  * Gradients are the exact derivatives of the FP64 forward, obtained by
    reverse-mode differentiation of plain torch ops (no hand-derived backward).

Modules: sh (real spherical harmonics), project (EWA projection + SH colour),
raster (tile binning, depth sort, Eq. 2 compositing, gradients), densify
(statistics, split/clone/prune masks, compaction, Philox4x32-10), loss (L1).
"""
