"""CPU oracle for region-adaptive DP pixelization.

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the CPU-baseline leg of the
benchmark may import this package.  The product library never imports, links or falls back to it.
"""
from .oracle import *  # noqa: F401,F403
