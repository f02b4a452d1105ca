"""GB300 (sm_103a) Fourier Domain Acceleration Search -- the data-parallel hot
path of arXiv:2211.13517 (White, Adamek, Armour) behind a C ABI.

The compute runs in hand-written CUDA kernels in libfdas.so (csrc/); this
package only builds the library (build.py) and binds it (capi.py).
"""
from .build import build, LIB  # noqa: F401
from . import capi  # noqa: F401
from .capi import Plan, FdasError  # noqa: F401

__all__ = ["build", "LIB", "capi", "Plan", "FdasError"]
