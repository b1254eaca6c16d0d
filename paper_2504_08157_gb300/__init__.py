"""GB300 (sm_103a) explicit CG Euler right-hand side, DSS, inverse mass and
SSP-RK3 stage update after Kang, Giraldo & Camp (arXiv 2504.08157).

The compute path is the CUDA library ``libxg.so`` behind the C ABI declared
in ``include/xg.h``; ``xg`` is its thin ctypes binding (same names, argument
marshalling only).  There is no CPU fallback: importing the binding fails
loudly when the library has not been built (``build.build()``).
"""

from . import xg  # noqa: F401
from .xg import *  # noqa: F401,F403
