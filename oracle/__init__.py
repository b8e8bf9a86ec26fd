"""CPU FP64 oracle of CholeskyQR2 -- TEST INFRASTRUCTURE ONLY.

Only tests/, the package's smoke check and the benchmark's CPU-baseline leg may
import this package; the GPU library neither imports nor links it.
"""
from .cholqr2 import (  # noqa: F401
    NotSPD,
    PassFailed,
    back_substitution,
    cholinv,
    cholinv_depth,
    cqr,
    cqr2,
    lstsq,
    nominal_flops,
    orthogonality,
    panel_cqr2,
    rel_error,
    residual,
    right_solve,
    scqr3,
    shift_of,
    shifted_cqr,
    syrk,
)
from .householder import householder_qr  # noqa: F401
