"""B300 (sm_103a) proximal message passing for network utility maximization.

Modules:
  capi       thin ctypes binding of the C ABI in include/num_pmp.h (loads lib/libnum_pmp.so)
  build      nvcc build of the CUDA sources in csrc/ into lib/libnum_pmp.so
  workloads  seeded synthetic instances (shared by the tests, the benchmark and the oracle)

Importing the package loads nothing; `from paper_2509_10722_b300 import capi` loads the
CUDA library and fails loudly when it has not been built.
"""
