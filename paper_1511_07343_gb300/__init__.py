"""GB300-native (sm_103a) Fourier Domain Acceleration Search.

The compute path lives in the CUDA library ``_build/libfdas_gb300.so``
(sources in ``csrc/``, C ABI in ``include/fdas.h``); ``fdas`` is its ctypes
binding (argument marshalling only) and ``serve`` a continuous-batching
serving loop over it.
"""
from . import fdas  # noqa: F401
