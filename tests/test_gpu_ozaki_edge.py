"""Split-precision path on inputs that stress its column-wise shared exponents.

The split-precision Gram and Q-form give every column of X one shared exponent
(its largest entry), and the Q-form folds those exponents into the rows of
R^-1 so that each output column has one scale. Entries far below their
column's maximum keep fewer significant bits, so the accuracy is normwise. The
inputs here are the ones where that choice shows:

* rows whose norms span twelve orders of magnitude at a fixed kappa
  (synth.graded_rows);
* one entry of a column 1e8 times the column's median (synth.spiked_column);
* a column of entries 1e-20 next to O(1) columns (synth.scaled_column).

A 6-slice plan routes itself to 7 slices on the device when a column's crest
ratio sqrt(m) 2^e_j / ||x_j|| exceeds 16 (in either pass); the test checks
that it did so exactly for the inputs whose crest ratios (of A, and of the
oracle's Q1 for the second pass) exceed 16.

Each runs through CQR2_OZAKI_BF16 (S = 7) and CQR2_OZAKI_BF16_S6 end to end at
ten times the FP64 tolerances (orthogonality <= max(1e-11, 10x the oracle's),
residual <= max(1e-12, 10x the oracle's), R relative <= 1e-11 kappa with kappa
the condition number of A with unit column norms, which a column scaling does
not change for CholeskyQR2), and per step against the elementwise Gram and
Q-form bounds of the split (the same bounds as test_gpu_ozaki).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from gpu_util import EPS, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cq():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_08471_gb300 as m

    return m


def pow2_above(x):
    x = np.abs(np.asarray(x, dtype=np.float64))
    e = np.floor(np.log2(np.where(x > 0, x, 1.0))) + 1
    return 2.0 ** e


def frac_bits(S):
    return 7 + 8 * (S - 1)


def _inputs():
    return {
        "graded_rows_k1e4": lambda: synth.graded_rows(20000, 64, 1e4, seed=71),
        "graded_rows_k1e6": lambda: synth.graded_rows(12000, 128, 1e6, seed=72),
        "spiked_column": lambda: synth.spiked_column(20000, 96, 1e3, seed=73, col=17),
        "spiked_last_column": lambda: synth.spiked_column(8000, 128, 1e4, seed=74, col=127),
        "tiny_column": lambda: synth.scaled_column(20000, 64, 1e4, seed=75, col=5),
        "tiny_and_huge_columns": lambda: synth.scaled_column(
            10000, 128, 1e2, seed=76, col=100, scale=1e-20) * np.where(np.arange(128) == 3, 1e15, 1.0)[None, :],
    }


CASES = sorted(_inputs())


def _max_crest(X):
    """Largest sqrt(m) 2^e_j / ||x_j|| over the columns (2^e_j the power of
    two above the column's largest magnitude)."""
    m = X.shape[0]
    return float(np.max(pow2_above(np.max(np.abs(X), axis=0)) * np.sqrt(m) / np.linalg.norm(X, axis=0)))


def _kappa_equilibrated(A):
    c = np.linalg.norm(A, axis=0)
    return float(np.linalg.cond(A / c[None, :]))


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("case", CASES)
def test_ozaki_edge_cqr2(cq, case, prec):
    A = np.asfortranarray(_inputs()[case]())
    m, n = A.shape
    k = _kappa_equilibrated(A)
    assert k < 1e7
    with cq.Plan(m, n, precision=prec) as p:
        Q, R, info = p.factor(to_dev(A))
        used = p.split_slices()
    assert info.status == 0
    Q, R = to_host(Q), to_host(R)
    Qo, Ro, inter = oracle.cqr2(A, keep=True)
    crest = max(_max_crest(A), _max_crest(inter["Q1"]))
    assert used == (7 if prec == 1 or crest > 16 else 6), (used, crest)
    orth = oracle.orthogonality(Q)
    res = oracle.residual(A, Q, R)
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R) > 0)
    assert orth <= max(1e-11, 10 * oracle.orthogonality(Qo)), orth
    assert res <= max(1e-12, 10 * oracle.residual(A, Qo, Ro)), res
    # R column by column relative to each column's norm (a column scaling
    # multiplies R's column by the same factor, so each column is checked at
    # its own scale)
    col_rel = np.linalg.norm(R - Ro, axis=0) / np.linalg.norm(Ro, axis=0)
    assert float(np.max(col_rel)) <= 1e-11 * k, float(np.max(col_rel))
    assert oracle.rel_error(R, Ro) <= 1e-11 * k


@pytest.mark.parametrize("S,prec", [(7, 1), (6, 2)])
@pytest.mark.parametrize("case", CASES)
def test_ozaki_edge_steps(cq, case, S, prec):
    A = np.asfortranarray(_inputs()[case]())
    m, n = A.shape
    _, _, i1 = oracle.cqr(A)
    Rinv = i1["Rinv"]
    with cq.Plan(m, n, precision=prec) as p:
        Ad = to_dev(A)
        W = to_host(p.syrk(Ad))
        Q = to_host(p.qform(Ad, to_dev(Rinv)))
    absA = np.abs(A)
    ce = pow2_above(np.max(absA, axis=0))
    Wo = oracle.syrk(A)
    wb = m * np.outer(ce, ce) * 2.0 ** (2 - frac_bits(S)) + 2 * m * EPS * (absA.T @ absA)
    assert np.all(np.abs(W - Wo) <= wb), float(np.max(np.abs(W - Wo) / wb))
    Qo = A @ Rinv
    fe = pow2_above(np.max(ce[:, None] * np.abs(np.triu(Rinv)), axis=0))
    qb = n * fe[None, :] * 2.0 ** (2 - frac_bits(S)) + 2 * n * EPS * (absA @ np.abs(Rinv))
    assert np.all(np.abs(Q - Qo) <= qb), float(np.max(np.abs(Q - Qo) / qb))
