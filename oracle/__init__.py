"""Plain FP64 CPU oracle for the MC 2->2 collision term (test infrastructure).

Only the test-suite, the smoke check and the CPU-baseline leg of the
benchmark may import this package.  It shares no code with the CUDA
library.
"""
from .oracle import *  # noqa: F401,F403
