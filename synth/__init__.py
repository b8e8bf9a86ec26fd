"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This package holds no CholeskyQR arithmetic. It only draws random matrices,
right-hand sides and request streams from counter-based Philox generators, so
that the oracle and the GPU library can be fed the very same bits.
"""
from .matrices import (  # noqa: F401
    ROW_BLOCK,
    gaussian,
    graded_rows,
    scaled_column,
    spiked_column,
    log_sigma,
    random_orthogonal,
    make_matrix,
    make_rhs,
    request_stream,
)
