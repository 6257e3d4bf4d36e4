"""GB300-native granule-grid coupling substep of the Granule-In-Cell method.

The compute path is the CUDA library libgic.so (C ABI in include/gic.h);
`gic` is its ctypes binding, `window` runs K-substep windows forward and
backward (torch.autograd.Function with checkpointing).
"""
__all__ = ["gic", "window", "build"]
