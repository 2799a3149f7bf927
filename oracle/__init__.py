"""FP64 CPU oracle of the Lagrangian-Decomposition dual bound.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only the tests, the smoke check and
the benchmark's CPU-baseline leg may import it.  It shares no code with the
CUDA path.
"""
from .ld_oracle import *  # noqa: F401,F403
