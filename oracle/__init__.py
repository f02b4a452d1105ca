"""FP64 CPU oracle for the FDAS hot path -- TEST INFRASTRUCTURE ONLY.

Importable only from the tests, the smoke check and the CPU-baseline leg of
the benchmark.  The CUDA product path never imports it.  See fdas_oracle.py
for what it computes and the passages it follows.
"""
from .fdas_oracle import *  # noqa: F401,F403
from .fdas_oracle import build, threads  # noqa: F401
