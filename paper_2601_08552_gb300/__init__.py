"""GB300-native (sm_103a) hot path of linear canonical-ensemble QMC (LEC-QMC).

The sweep runs in the CUDA library built from ``csrc/`` (C ABI in
``include/lecqmc.h``); ``lecqmc`` is its ctypes binding.
"""
from .lecqmc import (LQ_CHECKERBOARD, LQ_EXACT, LQ_FP64, LQ_MAX_PARTICLES, LQ_MIXED, LQ_MIXED_DW, LQ_NOBS, LQ_SWAP_NEIGHBOUR, LQ_SWAP_UNIFORM,  # noqa: F401
                     OBS_NAMES, Lattice, LqError, Server, Sim, device_fp64_rate, load)
