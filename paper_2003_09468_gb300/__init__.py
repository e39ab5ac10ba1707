"""GB300-native k-point phaseless AFQMC walker step (arXiv:2003.09468).

The compute lives in libafqmc_kp.so (hand-written CUDA for sm_103a behind the C
ABI in include/afqmc_kp.h); this package only marshals arguments.
"""
from .binding import (AfqmcError, DenseAFQMC, KPointAFQMC, KPointGroup, LocalEnergy, LIB_PATH,  # noqa: F401
                      SIGNATURES, load_library)

__all__ = ["AfqmcError", "DenseAFQMC", "KPointAFQMC", "KPointGroup", "LocalEnergy", "LIB_PATH", "SIGNATURES", "load_library"]
