"""GB300-native assembly-free transient heat solver (Loeb & Earls, arXiv 1905.07622).

The compute path is the CUDA library ``lib/libheatgb.so`` behind the C ABI of
``include/heat.h``; this package only marshals arguments to it (``api``).
Importing the package loads the library and raises if it is missing: there is
no CPU fallback.
"""
from .api import *  # noqa: F401,F403
from .api import HeatError, load_library  # noqa: F401
