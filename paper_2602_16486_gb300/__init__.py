"""GB300-native fluctuating central-moment lattice Boltzmann (arXiv:2602.16486).

The compute path is the CUDA library ``_build/libflbm.so`` (sources in ``csrc/``,
ABI in ``include/flbm.h``); ``flbm`` is its ctypes binding. Importing this package
fails loudly when the library has not been built.
"""
from .flbm import *  # noqa: F401,F403
from .flbm import Lattice, Batch, Domain, FlbmError, flbm_stats_t, LIB_PATH  # noqa: F401
