"""GB300-native state-vector gate engine (arXiv 2506.09198 hot path).

The compute lives in libqs.so (hand-written sm_103a CUDA kernels behind the C
ABI declared in include/qs.h); ``paper_2506_09198_gb300.qs`` is its ctypes
binding.  Build with ``paper_2506_09198_gb300.build.build()``.
"""
