"""GB300 (sm_103a) differentiable tile rasterizer for 3D Gaussian Splatting
(Kerbl et al., SIGGRAPH 2023, arXiv 2308.04079).

The C ABI (include/gs.h) exposes the four stages of Algorithm 2 -- gs_preprocess,
gs_bin_sort, gs_render_forward, gs_render_backward -- implemented as hand-written CUDA
kernels in ``csrc/`` and built into ``libgs_gb300.so`` by :mod:`.build`.  :mod:`._abi` is
the ctypes binding with the same names; :mod:`.rasterizer` adds workspace management and a
``torch.autograd.Function``.  Importing this package does not load the library; the first
call does, and fails loudly if it has not been built.
"""
from .rasterizer import Frame, FrameBatch, GaussianTensors, RasterizeFunction, make_config, rasterize, render

__all__ = ["Frame", "FrameBatch", "GaussianTensors", "RasterizeFunction", "make_config", "rasterize", "render"]
