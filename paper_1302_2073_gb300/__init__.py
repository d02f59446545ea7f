"""pROST's per-frame update (arXiv:1302.2073) on GB300: CUDA kernels for
sm_103a behind the C ABI of include/prost.h, with a ctypes binding."""

from .prost import *  # noqa: F401,F403
from .prost import ProstError, lib, make_params, header_functions  # noqa: F401
from . import window  # noqa: F401,E402  (the windowed cost as a torch.autograd.Function)
