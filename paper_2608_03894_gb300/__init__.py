"""GB300-native kagome DQMC time-slice sweep (arXiv 2608.03894 hot path).

The compute path is the CUDA library libdqmc_gb300.so (built for sm_103a by
``_build.build()``), reached through its C ABI (include/dqmc.h). This package
holds only the ctypes binding: importing it loads the library and fails
loudly if it is missing; there is no CPU fallback.
"""

from ._lib import DQMCError, LIB_PATH, load  # noqa: F401

load()

from .dqmc import DQMC, OBS_NAMES, Batch, autotune  # noqa: E402,F401
from . import ops  # noqa: E402,F401

__all__ = ["DQMC", "Batch", "autotune", "DQMCError", "OBS_NAMES", "ops", "load", "LIB_PATH"]
