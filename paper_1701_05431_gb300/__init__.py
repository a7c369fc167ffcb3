"""GB300-native first-order finite-volume step (arXiv:1701.05431).

The library is libfv.so (CUDA, sm_103a) behind the C ABI of include/fv.h;
`fvlib` is its Python binding and `build` compiles it in-tree with nvcc.
"""
from . import build, fvlib  # noqa: F401

__all__ = ["build", "fvlib"]
