"""FP64 CPU oracle for AR-BC preconditioned Landweber restoration.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The GPU
library never calls it, shares no code with it, and imports nothing from it.
"""

from .ar_oracle import *  # noqa: F401,F403
from .spectral_correction import *  # noqa: F401,F403
