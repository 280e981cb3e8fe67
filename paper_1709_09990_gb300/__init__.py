"""Exact treewidth on one GB300 (sm_103a): the breadth-first elimination-
ordering DP of van der Zanden & Bodlaender (arXiv 1709.09990) as CUDA kernels
behind the C ABI in include/tw.h.

Submodules:
  graphgen - seeded synthetic graph generators (input generation only)
  native   - ctypes binding of libtw.so (argument marshalling only)
  build    - nvcc build of libtw.so
  learned  - the learned starting bound (training data, training, proposal)
"""
__all__ = ["graphgen", "native", "build"]
