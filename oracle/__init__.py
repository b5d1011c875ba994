"""FP64 CPU oracle for Sim(3) essential-graph Levenberg-Marquardt.

TEST INFRASTRUCTURE ONLY: imported by the test-suite, the package smoke check
and the benchmark's CPU-baseline leg, never by the product path.  It shares no
code with the CUDA library.
"""
from .oracle import *  # noqa: F401,F403
