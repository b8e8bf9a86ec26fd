"""Closed-form matrices whose Cholesky factor and inverse are known exactly.

Shared by the oracle pins and the GPU parity tests. Nothing here computes a
Cholesky factorization: every value is a formula.
"""
from __future__ import annotations

import os
from math import comb

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def minij(n: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """W = [min(i,j)] (1-based); L = lower all-ones; Y = L^-1 = bidiagonal."""
    i = np.arange(1, n + 1)
    W = np.minimum.outer(i, i).astype(np.float64)
    L = np.tril(np.ones((n, n)))
    Y = np.eye(n) - np.eye(n, k=-1)
    return W, L, Y


def pascal(n: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Symmetric Pascal matrix W = [C(i+j, i)]; L = [C(i, j)];
    L^-1 = [(-1)^(i-j) C(i, j)] (0-based)."""
    W = np.array([[comb(i + j, i) for j in range(n)] for i in range(n)], dtype=np.float64)
    L = np.array([[comb(i, j) if j <= i else 0 for j in range(n)] for i in range(n)], dtype=np.float64)
    Y = np.array([[(-1) ** (i - j) * comb(i, j) if j <= i else 0 for j in range(n)] for i in range(n)],
                 dtype=np.float64)
    return W, L, Y


def read_golden(name: str) -> dict[str, np.ndarray]:
    """Parse a golden fixture: blocks introduced by a line holding one name."""
    blocks: dict[str, list[list[float]]] = {}
    cur = None
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            s = line.strip()
            if not s or s.startswith("#"):
                continue
            if s.isalpha():
                cur = s
                blocks[cur] = []
            else:
                blocks[cur].append([float(x) for x in s.split()])
    return {k: np.array(v) for k, v in blocks.items()}


def upper_with_kappa(n: int, kappa: float, seed: int) -> np.ndarray:
    """Upper-triangular R0 with positive diagonal and condition number about
    kappa: R0 = diag(sigma) + small strictly-upper noise, sigma log-spaced."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 77]))
    sig = np.logspace(0, -np.log10(kappa), n) if n > 1 else np.ones(1)
    R0 = np.diag(sig) + np.triu(rng.standard_normal((n, n)), 1) * (0.1 / n) * sig[None, :]
    return R0
