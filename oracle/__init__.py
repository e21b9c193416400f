"""FP64 CPU oracle for core-elements ALS.

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg. The CUDA library never imports or calls it, and
it imports nothing from the CUDA package.

Parity status of each function is listed in ``oracle/oracle.py``.
"""
from .oracle import *  # noqa: F401,F403
