"""GB300-native SSLBM / BGK solver for the 2D SEIRD reaction-diffusion model.

The compute path is the C-ABI library ``libsslbm.so`` (hand-written sm_103a CUDA
kernels, declared in ``include/sslbm.h``).  ``paper_2603_19789_gb300.sslbm`` is a
thin ctypes binding with the same entry-point names; importing this package does
not load the library, the first call into the binding does, and it raises if the
library has not been built (there is no CPU fallback).
"""

__all__ = ["inputs"]
