"""FP64 CPU reference oracle of the Spinsim method (arXiv 2204.05586).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, by the smoke check and
by the CPU-baseline leg of ``bench.py``.  The product library never imports
it.  The arithmetic lives in ``spinsim_oracle.c`` (plain C, libm, double
complex); this module only compiles it with gcc and marshals arguments.
"""
from .oracle import *  # noqa: F401,F403
