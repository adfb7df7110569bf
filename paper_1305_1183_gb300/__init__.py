"""libkf: fused BLAS-1/BLAS-2 sequences for NVIDIA GB300 (sm_103a).

The compute path is the C-ABI shared library built from ``csrc/`` (see
``include/kf.h``); ``kf`` is its ctypes binding.
"""

from . import kf  # noqa: F401
from ._build import build  # noqa: F401
