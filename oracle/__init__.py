"""CPU oracle for the RGF hot path (test infrastructure only).

Plain numpy complex128 restatements of the paper's equations, used to judge the CUDA library.
Only the test suite, the smoke check and the CPU-baseline leg of the benchmark may import
this package; the library itself never does.
"""
from .negf_oracle import *  # noqa: F401,F403
