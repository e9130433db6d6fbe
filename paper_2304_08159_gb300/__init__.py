"""GB300-native WaterLily time step: CUDA kernels for sm_103a behind a C ABI
(include/wl.h, libwl.so) with a thin ctypes binding (``wl``)."""
from . import wl  # noqa: F401
from .wl import Sim, WLError  # noqa: F401
