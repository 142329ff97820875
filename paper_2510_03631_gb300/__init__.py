"""GB300-native LWE-style PIR Response engine for QPADL spectrum databases.

The compute path is a C-ABI CUDA library (sm_103a) declared in
include/qpadl_pir.h; `paper_2510_03631_gb300.pir` is its thin ctypes binding.
Importing this package loads nothing: the library is loaded on first use and
every entry point raises if it is missing.  There is no CPU fallback.
"""

__all__ = ["inputs", "pir"]
