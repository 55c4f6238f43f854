"""GB300 (sm_103a) implementation of the rank-1-lattice sparse FFT for arbitrary frequency
candidate sets (Kaemmerer, Krahmer, Volkmer, arXiv 2006.13053).

The CUDA library libsfft.so (C ABI in include/sfft.h) does all computation; this package
binds it.  Importing the package fails when the library has not been built.
"""
from ._native import (CAND_I8, CAND_I32, COMBINE_HYBRID, COMBINE_LSQ, COMBINE_MEDIAN, DFT_DF64, DFT_FP32,  # noqa: F401
                      FP32, FP64, L_COR26, L_EQ42, L_FALLBACK, SfftError, default_dimincr_params, default_params)
from .api import Batch, Plan, SopReconstruct, dim_incremental  # noqa: F401
