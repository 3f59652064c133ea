"""GB300-native differentiable FDTD hot path (arxiv 2609.30039).

The compute path is the C-ABI library `libgbfdtd.so` (hand-written sm_103a CUDA kernels,
declared in include/fdtd.h).  `fdtd` is its thin ctypes binding; `adjoint` wraps the
transposed sweep as a torch.autograd.Function with binomial checkpoint replay.
Importing this package loads nothing; the library is loaded on first use and its absence
is an error (there is no CPU fallback).
"""
__all__ = ["fdtd", "workloads"]
