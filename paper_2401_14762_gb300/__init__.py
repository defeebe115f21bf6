"""GB300-native per-pixel sparse recovery of compressively sensed hyperspectral cubes.

The compute lives in ``libcs_hsi.so`` (hand-written CUDA for sm_103a behind a C ABI,
declared in ``include/cs_hsi.h``).  ``paper_2401_14762_gb300.cs`` is the thin ctypes
binding with the same call names; it loads the library on first use and raises if
the library or a CUDA device is missing -- there is no CPU fallback.
"""
__all__ = ["cs", "synthetic"]
