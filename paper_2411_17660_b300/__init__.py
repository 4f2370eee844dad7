"""B300 (sm_103a) differentiable Gaussian rasteriser: the dense renderer's
hot path of DROID-Splat (arXiv 2411.17660, Sec. 3.3).

The CUDA kernels and their C ABI (include/gsr.h) live in csrc/ and build to
_build/libgsr.so; `binding` marshals arguments into it and `render` wraps it
for PyTorch tensors and autograd.  `scenes` draws the seeded synthetic inputs.
"""
