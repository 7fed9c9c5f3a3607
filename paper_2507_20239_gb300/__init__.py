"""GB300-native differentiable tile rasterizer for 3D Gaussian splatting.

Implements the hot path of "Decomposing Densification in Gaussian Splatting for
Faster 3D Scene Reconstruction" (arXiv 2507.20239): EWA projection and SH colour,
tile binning and depth sort, Eq. 2 front-to-back compositing and its gradient,
and the densification bookkeeping (split/clone/prune and compaction). The compute
lives in libgs.so (CUDA, sm_103a, C ABI in include/gs.h); this package holds the
build script, a ctypes binding and a torch.autograd wrapper.

Submodules are imported lazily so that `synth` (numpy only) and `build` work on a
machine without a GPU.
"""
__all__ = ["build", "synth", "rasterizer", "autograd"]
