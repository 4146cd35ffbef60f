"""GB300-native hot path of the MULTIBAT Li-ion cell model with lithium plating
(arXiv:1704.04139): the implicit full-order step and the reduced-model online
solve, as a C-ABI CUDA library (libmb.so, include/mb.h) with a thin ctypes
binding."""
from .binding import (Cell, MBError, default_opts, lib, params_from_dict, PREC_FP64, PREC_MIXED)

__all__ = ["Cell", "MBError", "default_opts", "lib", "params_from_dict", "PREC_FP64", "PREC_MIXED"]
