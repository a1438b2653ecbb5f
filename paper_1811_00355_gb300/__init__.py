"""GB300 (sm_103a) 2-level DD-alpha-AMG solver for Wilson-clover fermions.

The solver is the CUDA library ``libddamg.so`` behind the C ABI of
``include/ddamg.h``; :mod:`._ddamg` is its ctypes binding.  Importing this
package loads nothing; :func:`load` (or creating a :class:`DDAMG`) loads the
library and fails loudly if it has not been built.
"""
from ._ddamg import (BF16, FP16, FP32, FP64, DDAMG, DDAMGError, Level2Params, Params, RequestInfo, Server,
                     SolveInfo, Stats, default_params, level2_default_params, load, pin_variant, tuning)

__all__ = ["BF16", "FP16", "FP32", "FP64", "DDAMG", "DDAMGError", "Level2Params", "Params", "RequestInfo", "Server",
           "SolveInfo", "Stats", "default_params", "level2_default_params", "load", "pin_variant", "tuning"]
