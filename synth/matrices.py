"""Seeded random test matrices of the shapes the paper factors (Section IV-C).

The paper measures on matrices it generates at random ("we generate random
matrices", Section IV-C) and prints neither their entries nor their
distribution; the recipes below are this project's stand-ins:

* ``gaussian``: iid N(0, 1) entries. A tall Gaussian m x n matrix with m >> n
  has condition number close to (1 + sqrt(n/m)) / (1 - sqrt(n/m)); for
  4096 x 64 that is about 1.3.
* ``make_matrix``: A = G . diag(sigma) . V with G Gaussian, sigma log-spaced
  from 1 down to 1/kappa and V a seeded random orthogonal n x n matrix (the
  sign-normalised Q factor of a Gaussian), so that kappa(A) ~= kappa.

Every random number comes from numpy's Philox4x32-10 bit generator keyed by
(seed, matrix id, row block). Rows are generated in blocks of ``ROW_BLOCK``
with one key per block, so the result does not depend on how many threads
generate it. Matrices are column-major (Fortran order), the LAPACK layout the
library uses.
"""
from __future__ import annotations

import concurrent.futures as _cf
import os

import numpy as np

ROW_BLOCK = 1 << 16

_KEY_V = 0xFFFF_FFFF  # row-block slot reserved for the orthogonal factor V
_KEY_B = 0xFFFF_FFFE  # slot for right-hand sides
_KEY_REQ = 0xFFFF_FFFD  # slot for request-stream parameters


def _gen(seed: int, mid: int, slot: int) -> np.random.Generator:
    key0 = ((int(seed) & 0xFFFF_FFFF) << 32) | (int(mid) & 0xFFFF_FFFF)
    return np.random.Generator(np.random.Philox(key=[key0, int(slot) & 0xFFFF_FFFF_FFFF_FFFF]))


def _threads(threads: int | None) -> int:
    if threads is not None:
        return max(1, int(threads))
    return max(1, min(32, os.cpu_count() or 1))


def _fill_gaussian_block(out: np.ndarray, seed: int, mid: int, b: int, r0: int, r1: int) -> None:
    n = out.shape[1]
    g = _gen(seed, mid, b).standard_normal((n, r1 - r0))
    out[r0:r1, :] = g.T


def gaussian(m: int, n: int, seed: int, mid: int = 0, out: np.ndarray | None = None,
             threads: int | None = None) -> np.ndarray:
    """m x n matrix of iid N(0,1) entries, column-major."""
    if out is None:
        out = np.empty((m, n), dtype=np.float64, order="F")
    nb = (m + ROW_BLOCK - 1) // ROW_BLOCK
    jobs = [(b, b * ROW_BLOCK, min(m, (b + 1) * ROW_BLOCK)) for b in range(nb)]
    nt = _threads(threads)
    if nt == 1 or nb == 1:
        for b, r0, r1 in jobs:
            _fill_gaussian_block(out, seed, mid, b, r0, r1)
    else:
        with _cf.ThreadPoolExecutor(nt) as ex:
            list(ex.map(lambda j: _fill_gaussian_block(out, seed, mid, *j), jobs))
    return out


def log_sigma(n: int, kappa: float) -> np.ndarray:
    """n singular values log-spaced from 1 down to 1/kappa."""
    if n == 1:
        return np.ones(1)
    return np.logspace(0.0, -np.log10(float(kappa)), n)


def random_orthogonal(n: int, seed: int, mid: int = 0) -> np.ndarray:
    """Seeded random orthogonal n x n matrix: Q factor of a Gaussian with R's
    diagonal made positive (LAPACK Householder QR via numpy)."""
    g = _gen(seed, mid, _KEY_V).standard_normal((n, n))
    q, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return np.asfortranarray(q * d)


def make_matrix(m: int, n: int, kappa: float | None, seed: int, mid: int = 0,
                out: np.ndarray | None = None, threads: int | None = None) -> np.ndarray:
    """Column-major m x n FP64 test matrix.

    kappa=None gives iid N(0,1) entries; otherwise A = G . diag(sigma) . V with
    sigma = log_sigma(n, kappa) and V = random_orthogonal(n, seed, mid).
    """
    if kappa is None:
        return gaussian(m, n, seed, mid, out=out, threads=threads)
    if out is None:
        out = np.empty((m, n), dtype=np.float64, order="F")
    sv = (log_sigma(n, kappa)[:, None] * random_orthogonal(n, seed, mid))  # diag(sigma) . V

    def blk(job):
        b, r0, r1 = job
        g = _gen(seed, mid, b).standard_normal((n, r1 - r0))  # G[r0:r1, :]^T
        out[r0:r1, :] = g.T @ sv

    nb = (m + ROW_BLOCK - 1) // ROW_BLOCK
    jobs = [(b, b * ROW_BLOCK, min(m, (b + 1) * ROW_BLOCK)) for b in range(nb)]
    nt = _threads(threads)
    if nt == 1 or nb == 1:
        for j in jobs:
            blk(j)
    else:
        with _cf.ThreadPoolExecutor(nt) as ex:
            list(ex.map(blk, jobs))
    return out


def make_rhs(m: int, seed: int, mid: int = 0) -> np.ndarray:
    """Right-hand side b of length m, iid N(0,1)."""
    return _gen(seed, mid, _KEY_B).standard_normal(m)


def request_stream(count: int, seed: int, rate: float, m_lo: int = 1024, m_hi: int = 262144,
                   n_choices=(16, 32, 64, 128, 256), kappa_lo: float = 1.0,
                   kappa_hi: float = 1e5) -> list[dict]:
    """Least-squares request stream: Poisson arrivals at `rate` per second,
    m uniform in [m_lo, m_hi], n uniform over `n_choices`, kappa log-uniform in
    [kappa_lo, kappa_hi]. Request i's matrix uses seed `seed + i`."""
    g = _gen(seed, 0, _KEY_REQ)
    gaps = g.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps) - gaps[0]
    ms = g.integers(m_lo, m_hi + 1, size=count)
    ns = g.choice(np.asarray(n_choices), size=count)
    ks = np.exp(g.uniform(np.log(kappa_lo), np.log(kappa_hi), size=count))
    return [dict(id=i, t=float(t[i]), m=int(ms[i]), n=int(ns[i]), kappa=float(ks[i]), seed=seed + i)
            for i in range(count)]


# ------------------------------------------------ inputs that stress scaling

def graded_rows(m: int, n: int, kappa: float, seed: int, span: float = 1e6, mid: int = 0) -> np.ndarray:
    """m x n matrix with condition number kappa whose row norms spread over
    about span^2 (12 orders of magnitude for span = 1e6): A = U diag(sigma) V
    with U the orthonormal factor (LAPACK Householder QR via numpy) of D G,
    D = diag(10^u), u uniform in [-log10 span, log10 span] per row, G Gaussian.
    U's rows scale like D, while A keeps the singular values sigma."""
    g = _gen(seed, mid, 0)
    G = g.standard_normal((m, n))
    d = 10.0 ** g.uniform(-np.log10(span), np.log10(span), size=m)
    U, _ = np.linalg.qr(d[:, None] * G)
    A = U @ (log_sigma(n, kappa)[:, None] * random_orthogonal(n, seed, mid))
    return np.asfortranarray(A)


def spiked_column(m: int, n: int, kappa: float | None, seed: int, col: int, ratio: float = 1e8,
                  mid: int = 0) -> np.ndarray:
    """make_matrix(m, n, kappa, seed) with one entry of column `col` (at a
    seeded row) set to `ratio` times the column's median magnitude."""
    A = make_matrix(m, n, kappa, seed, mid)
    row = int(_gen(seed, mid, 1).integers(0, m))
    A[row, col] = ratio * float(np.median(np.abs(A[:, col])))
    return A


def scaled_column(m: int, n: int, kappa: float | None, seed: int, col: int, scale: float = 1e-20,
                  mid: int = 0) -> np.ndarray:
    """make_matrix(m, n, kappa, seed) with column `col` multiplied by `scale`
    (a column of all-tiny entries next to O(1) ones)."""
    A = make_matrix(m, n, kappa, seed, mid)
    A[:, col] *= scale
    return A
