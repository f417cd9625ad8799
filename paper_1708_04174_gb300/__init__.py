"""GB300-native HSDE ADMM for sum-of-squares programs (libsos + binding).

The solver itself is ``libsos.so`` (C-ABI in include/sos.h, CUDA kernels for
sm_103a under csrc/).  ``capi`` is its ctypes binding; ``build`` compiles it.
"""

from . import capi  # noqa: F401
