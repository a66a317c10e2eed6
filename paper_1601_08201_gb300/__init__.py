"""GB300-native spectrally grouped TV (SGTV) reconstruction with ADMM.

The hot path (forward projection, backprojection fused with the per
hyper-voxel update, group shrinkage with the dual update, FP64 objective
reductions) runs as sm_103a CUDA kernels inside ``libsgtv.so`` behind a C ABI
(``include/sgtv.h``); ``paper_1601_08201_gb300.sgtv`` is its thin ctypes
binding. ``synth`` draws seeded synthetic problems.
"""
__all__ = ["synth", "sgtv"]
