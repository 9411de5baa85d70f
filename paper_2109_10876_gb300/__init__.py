"""GB300-native short-range molecular dynamics (arXiv:2109.10876 hot path).

The compute path is a C-ABI shared library of hand-written sm_103a CUDA
kernels (csrc/), declared in include/md.h and reached through the thin ctypes
binding in `md` (same function names as the C ABI).  Importing this package
does not load the library; `paper_2109_10876_gb300.md` does, and fails loudly
if it has not been built.
"""
__all__ = ["inputs", "md", "build"]
