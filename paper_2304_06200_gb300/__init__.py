"""GB300-native hard-coded-gradient (HG) GRAPE: cost + gradient evaluation on one GPU.

The computation runs in the CUDA library ``libgrape_hg.so`` (C ABI in
``include/grape_hg.h``); this package holds its build script and a thin Python
binding.  There is no CPU fallback: if the library cannot be built or loaded,
every entry point raises.
"""

from .hg import GrapeBatch, GrapeProblem, autotune, error_bound, grape_hg, select_ms  # noqa: F401
from ._abi import GrapeError, EXPORTED  # noqa: F401
