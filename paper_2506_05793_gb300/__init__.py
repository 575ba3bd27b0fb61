"""GB300-native supernodal multifrontal sparse Cholesky (Tacho's hot path).

The numeric factorization ``P A P^T = L L^T`` and the supernodal forward/back
solves run in hand-written sm_103a CUDA kernels behind the C-ABI of
``include/mfchol.h`` (library ``lib/libmfchol.so``).  This package is the thin
Python binding: functions carry the C names and only marshal arguments.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import MFError, lib  # noqa: F401
from .build import build  # noqa: F401
