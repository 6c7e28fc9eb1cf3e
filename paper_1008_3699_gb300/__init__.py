"""GB300-native decomposed sequential sweep (SOR / SSOR / ILU(0)) on
structured n-diagonal matrices, after Tavakoli, arXiv 1008.3699.

The compute path is the CUDA library libndiag.so (include/ndiag.h); the
Python module `ndiag` is its binding and `workloads` builds seeded inputs.
"""
