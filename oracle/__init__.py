"""FP64 CPU oracle for the kernel polynomial method (test infrastructure only).

Only tests, the smoke check and the benchmark's CPU-baseline leg may import
this package; the product path never calls it.
"""
from .kpm_oracle import *  # noqa: F401,F403
