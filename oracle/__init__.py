"""FP64 CPU oracle for the k-point AFQMC walker step.

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the CPU
baseline leg of the benchmark, never by the product library.
"""
from . import afqmc_kp, dense, fock  # noqa: F401
