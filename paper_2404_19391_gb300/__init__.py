"""GB300-native ZSMILES codec (arXiv 2404.19391): CUDA kernels for sm_103a behind a C ABI (libzsmiles.so).

``zsmiles`` is the Python binding (same names as include/zsmiles.h). Building: ``build.build()``.
"""
from . import build  # noqa: F401
