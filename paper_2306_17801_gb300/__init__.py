"""Asynchronous device-scalar Jacobi-preconditioned CG for NVIDIA GB300 (sm_103a).

The compute path is the C-ABI library ``libapcg.so`` (CUDA kernels written
for sm_103a); ``apcg`` is its thin ctypes binding.  There is no CPU fallback:
loading fails loudly when the library has not been built.
"""

from . import apcg  # noqa: F401

__all__ = ["apcg"]
