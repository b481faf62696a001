"""GB300-native time-varying linear prediction (Yu & Fazekas, arXiv 2406.05128).

The hot path is the sample-wise time-varying all-pole filter (Eq. 5) and its
adjoint (Eqs. 11-12), batched over signals, implemented as hand-written CUDA
kernels for sm_103a behind a C ABI (include/tvlp.h, libtvlp.so).

Submodules:
  ops     PyTorch front end (lp_filter autograd op, lp_tv_forward/backward)
  _lib    ctypes binding of the C ABI
  inputs  seeded synthetic workloads
  build   in-tree nvcc build of libtvlp.so
"""
__all__ = ["ops", "inputs", "build"]
