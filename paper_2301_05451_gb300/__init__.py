"""GB300-native batched tensor-network contraction of parameterised circuits.

Layers: ``include/tdq.h`` (C ABI) over ``csrc/`` (CUDA kernels for sm_103a and
the C++ host side); ``_abi`` (ctypes binding), ``api`` (torch-facing wrappers
and the autograd function), ``workloads`` (seeded synthetic circuits),
``build`` (nvcc build of libtdq.so).  Importing this package loads nothing;
``api`` loads the library on first use and fails loudly if it is missing.
"""
__all__ = ["api", "workloads", "build"]
