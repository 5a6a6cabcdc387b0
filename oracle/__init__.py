"""Independent CPU oracle for the state-vector hot path (complex128).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg may use this package; the product library never does.
"""
from .oracle import *  # noqa: F401,F403
