"""GB300 (sm_103a) Delay-and-Sum and tiDAS operators.

C ABI: include/tidas.h, implemented in csrc/ and built into _build/libtidas.so.
capi.py binds it with ctypes under the same names; ops.py wraps it for torch
tensors.  Importing this package does not touch the GPU.
"""
from . import capi  # noqa: F401
from .capi import TidasError  # noqa: F401
