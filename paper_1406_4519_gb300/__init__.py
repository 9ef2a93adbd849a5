"""GB300-native DFacTo: sparse CP decomposition (MTTKRP, ALS, GD) in CUDA.

The compute path is the C-ABI library ``libdfacto.so`` (sm_103a kernels, see
``include/dfacto.h``); :mod:`paper_1406_4519_gb300.dfacto` is its thin ctypes
binding.  Importing this package loads nothing; the binding loads the library on
first use and raises if it has not been built.
"""
__all__ = ["dfacto", "synth"]
