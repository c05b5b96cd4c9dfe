"""GB300 (sm_103a) library for the explicit semi-Lagrangian spectral (DSEM-SL) transport step
of arXiv:1910.06476: CUDA kernels behind a C ABI (include/sl.h) with a ctypes binding."""
from .binding import *  # noqa: F401,F403
from .binding import Batch, Context, SlError, lib, load_library, options, velocity  # noqa: F401
