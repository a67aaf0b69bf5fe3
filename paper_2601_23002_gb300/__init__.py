"""GB300-native finite-temperature orbital-free DFT hot path.

The compute runs in the CUDA library libofdft_gb300.so (C-ABI in
include/ofdft.h); this package is its Python binding.
"""
from ._lib import (TERM_TF, TERM_VW, TERM_NL, TERM_XC, TERM_HARTREE, TERM_LOC, TERMS_ALL,
                   OFDFT_FP32, OFDFT_FP64, load)
from .api import Plan, plan_for_cell, minimize, minimize_batch, OfdftError

__all__ = ["Plan", "plan_for_cell", "minimize", "minimize_batch", "OfdftError", "load", "TERM_TF", "TERM_VW", "TERM_NL", "TERM_XC",
           "TERM_HARTREE", "TERM_LOC", "TERMS_ALL", "OFDFT_FP32", "OFDFT_FP64"]
