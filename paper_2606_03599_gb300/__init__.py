"""GB300-native parity-blocked band solver for 3D anisotropic phononic crystals.

The compute path lives in ``libpcband.so`` (hand-written sm_103a CUDA behind
the C ABI of ``include/pcband.h``); ``_lib`` is a ctypes binding of it.
Importing this package raises ImportError when the library is not built.
"""

from ._lib import *  # noqa: F401,F403
from ._lib import lib, EXPORTED, PcError, PcNoConvergence, PcBreakdown  # noqa: F401
