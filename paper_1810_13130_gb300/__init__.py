"""GB300 (sm_103a) library for real-time TDKS propagation with spectral finite
elements and the second-order Magnus-Lanczos step (arXiv 1810.13130).

The compute path is libtdks.so (hand-written CUDA, C ABI in include/tdks.h);
`tdks` is its ctypes binding.  Importing this package does not load the library.
"""
from .build import build  # noqa: F401
