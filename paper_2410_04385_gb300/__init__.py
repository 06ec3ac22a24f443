"""GB300-native HaTT: Hadamard-avoiding recompression of tensor-train products.

The compute path is the C-ABI library libhatt (include/hatt.h, CUDA kernels
under csrc/ for sm_103a); `binding` is its ctypes interface and `workloads`
the seeded synthetic inputs.
"""
