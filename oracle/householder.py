"""Householder QR written independently of the CholeskyQR2 oracle.

TEST INFRASTRUCTURE ONLY (see oracle/cholqr2.py). It is the brute-force check the
oracle is pinned against: the reduced QR factorization A = QR with positive
diagonal in R is unique for a full-rank A (the problem statement of Section
II-E: Q with orthonormal columns, R upper triangular), so any backward-stable
QR normalised to a positive diagonal must agree with CholeskyQR2 within the
conditioning of the problem.
"""
from __future__ import annotations

import numpy as np


def householder_qr(A: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Reduced QR by Householder reflections, R with a positive diagonal."""
    A = np.array(A, dtype=np.float64, copy=True)
    m, n = A.shape
    if m < n:
        raise ValueError("needs m >= n")
    vs = []
    for k in range(n):
        x = A[k:, k]
        nx = np.linalg.norm(x)
        v = x.copy()
        alpha = -nx if x[0] >= 0 else nx
        v[0] -= alpha
        nv = np.linalg.norm(v)
        if nv > 0:
            v /= nv
            A[k:, k:] -= 2.0 * np.outer(v, v @ A[k:, k:])
        vs.append(v)
    R = np.triu(A[:n, :])
    Q = np.zeros((m, n))
    Q[:n, :n] = np.eye(n)
    for k in range(n - 1, -1, -1):
        v = vs[k]
        Q[k:, :] -= 2.0 * np.outer(v, v @ Q[k:, :])
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d, d[:, None] * R
