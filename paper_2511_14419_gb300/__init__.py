"""GB300 (sm_103a) CUDA implementation of the FlowRoI hot path.

The computation lives in the CUDA library built from ``csrc/`` (C ABI in
``include/flowroi.h``); ``flowroi`` is its ctypes binding.
"""
from . import flowroi  # noqa: F401
from ._build import LIB, build  # noqa: F401
