"""Split-CTMRG engine for one GB300 GPU (sm_103a), arXiv 2502.10298.

Thin Python binding of the C ABI in ``include/splitctmrg.h``.  Every step of
the method runs in the CUDA kernels of ``csrc/``; this module only marshals
arguments (PyTorch provides device memory and the stream).  It raises if the
in-tree library ``libsplitctmrg.so`` is missing: there is no fallback.
"""
from .api import *  # noqa: F401,F403
from .api import __all__  # noqa: F401
from .optimize import lbfgs  # noqa: F401
