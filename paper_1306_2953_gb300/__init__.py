"""GB300-native real-space Kohn-Sham hot path (arXiv:1306.2953).

The computation lives in ``librsdft.so`` (CUDA for sm_103a behind the C ABI
of include/rsdft.h); ``_lib`` binds it with ctypes and ``api`` wraps it
for torch tensors.  There is no CPU fallback.
"""
from ._lib import RS_F32, RS_F64, RsError  # noqa: F401
