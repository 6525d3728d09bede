"""CPU oracle for the AFMM product (arXiv 1308.2400, Sec. 2).

Test infrastructure only: the test suite, the package's smoke check and the
benchmark's CPU-baseline leg use it; the product path never does.
"""
from .oracle import *  # noqa: F401,F403
