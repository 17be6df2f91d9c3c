"""GB300 (sm_103a) implementation of the MBE(3)-OSV-MP2 pair-solve path.

The compute lives in ``libosvmp2.so`` (C ABI, include/osvmp2.h); this package
holds its build script and a thin ctypes binding (``osvmp2``).
"""
from . import osvmp2  # noqa: F401
from .osvmp2 import Context, generate_B, mbe3_fragments, OSVMP2Error  # noqa: F401
