"""GB300-native Poisson-lognormal MAP reconstruction (Kitaura, Jasche & Metcalf).

The solver itself is the CUDA library libplc.so (C ABI in include/plc.h);
this package holds its ctypes binding, the seeded mock generator and the
build script.  Import of the binding fails loudly if the library is missing.
"""
from ._lib import (PLC_FP64, PLC_MIXED, Batch, Context, MapResult, PlcError, default_opts, load)

__all__ = ["Batch", "Context", "MapResult", "PlcError", "default_opts", "load", "PLC_FP64",
           "PLC_MIXED"]
