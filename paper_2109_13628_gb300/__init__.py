"""GB300-native immersed interface Poisson solver (Gabbard, Gillis, Chatelain, van Rees,
Sec. 4.2): CUDA kernels behind the C ABI of include/iim.h, with a thin ctypes binding."""
from .binding import *  # noqa: F401,F403
from .binding import Geometry, IIMError, load  # noqa: F401
