"""Split-precision (Ozaki) path: the Gram and Q-forming contractions on the
BF16 tensor cores, checked against the CPU FP64 oracle.

Bounds. Each FP64 entry is rounded once to a fixed-point integer with
7 + 8(S-1) fraction bits relative to 2^e, where 2^e is the smallest power of
two above the largest entry along the contraction (per column of A for the
Gram; per row of A and per column of R^-1 for the Q-form). Products of the
kept slices are exact, and so is their accumulation, so
  |W_oz - W|_ij <= m 2^(e_i + e_j - (7 + 8(S-1)) + 2)
  |Q_oz - Q|_rj <= n 2^(e_r + f_j - (7 + 8(S-1)) + 2)
and the oracle's own FP64 rounding (2 m eps |A|^T|A|, 2 n eps |A||R^-1|) is
added on top. End to end, the target is ten times the FP64 bounds:
||Q^T Q - I||_F <= 1e-11, ||QR - A||_F/||A||_F <= 1e-12,
||R - R_oracle||_F/||R_oracle||_F <= 1e-11 kappa.
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
    """Smallest power of two strictly above each |x| (1 for zero)."""
    x = np.abs(np.asarray(x, dtype=np.float64))
    e = np.floor(np.log2(np.where(x > 0, x, 1.0))) + 1
    return 2.0 ** e


def frac_bits(S):
    return 7 + 8 * (S - 1)


SHAPES = [
    (4096, 64, None),
    (1000, 1, None),
    (64, 64, 10.0),
    (777, 33, 1e3),
    (20000, 128, 1e6),
    (3001, 200, 1e3),
    (2500, 512, 1e4),
]


@pytest.mark.parametrize("S,prec", [(7, 1), (6, 2)])
@pytest.mark.parametrize("m,n,kappa", SHAPES)
def test_ozaki_syrk(cq, m, n, kappa, S, prec):
    A = synth.make_matrix(m, n, kappa, seed=m + n + 1)
    with cq.Plan(m, n, precision=prec) as p:
        W = to_host(p.syrk(to_dev(A)))
    Wo = oracle.syrk(A)
    ce = pow2_above(np.max(np.abs(A), axis=0))
    absA = np.abs(A)
    bound = m * np.outer(ce, ce) * 2.0 ** (2 - frac_bits(S)) + 2 * m * EPS * (absA.T @ absA)
    assert np.array_equal(W, W.T)
    assert np.all(np.abs(W - Wo) <= bound), float(np.max(np.abs(W - Wo) / bound))


@pytest.mark.parametrize("S,prec", [(7, 1), (6, 2)])
@pytest.mark.parametrize("m,n,kappa", SHAPES)
def test_ozaki_qform(cq, m, n, kappa, S, prec):
    A = synth.make_matrix(m, n, kappa, seed=2 * m + n + 1)
    _, _, i1 = oracle.cqr(A)
    Rinv = i1["Rinv"]
    garbage = Rinv + np.tril(np.full((n, n), 3.0), -1)
    with cq.Plan(m, n, precision=prec) as p:
        Q = to_host(p.qform(to_dev(A), to_dev(garbage)))
    Qo = A @ Rinv
    # X enters through its column slices (exponent c_k per column, the Gram's),
    # with 2^c_k folded into row k of R^-1: one exponent f_j per column of the
    # scaled R^-1, and every product's truncation is below 2^(f_j - frac + 1)
    ce = pow2_above(np.max(np.abs(A), axis=0))
    fe = pow2_above(np.max(ce[:, None] * np.abs(np.triu(Rinv)), axis=0))
    bound = n * fe[None, :] * 2.0 ** (2 - frac_bits(S)) + 2 * n * EPS * (np.abs(A) @ np.abs(Rinv))
    assert np.all(np.abs(Q - Qo) <= bound), float(np.max(np.abs(Q - Qo) / bound))


def _check(A, Q, R, kappa):
    Qo, Ro = oracle.cqr2(A)
    k = kappa or 2.0
    orth = oracle.orthogonality(Q)
    res = oracle.residual(A, Q, R)
    rel = oracle.rel_error(R, Ro)
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R) > 0)
    assert orth <= max(1e-11, 10 * oracle.orthogonality(Qo)), orth
    assert res <= max(1e-12, 10 * oracle.residual(A, Qo, Ro)), res
    assert rel <= 1e-11 * k, rel
    return orth, res, rel


@pytest.mark.parametrize("m,n,kappa", SHAPES + [(20000, 96, 1e7), (8192, 256, 1e6), (1500, 1024, 1e2)])
def test_ozaki_cqr2(cq, m, n, kappa):
    A = synth.make_matrix(m, n, kappa, seed=3 * m + n)
    with cq.Plan(m, n, precision=cq.CQR2_OZAKI_BF16) as p:
        Q, R, info = p.factor(to_dev(A))
    assert info.status == 0
    _check(A, to_host(Q), to_host(R), kappa)


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
def test_ozaki_s6_cqr2(cq, kappa):
    m, n = 16384, 128
    A = synth.make_matrix(m, n, kappa, seed=17)
    with cq.Plan(m, n, precision=cq.CQR2_OZAKI_BF16_S6) as p:
        Q, R, info = p.factor(to_dev(A))
        # Gaussian-like columns (crest ratio about 5 to 10): no routing
        assert p.split_slices() == 6
    _check(A, to_host(Q), to_host(R), kappa)
    with cq.Plan(m, n, precision=cq.CQR2_OZAKI_BF16) as p:
        p.factor(to_dev(A))
        assert p.split_slices() == 7
    with cq.Plan(m, n) as p:
        p.factor(to_dev(A))
        assert p.split_slices() == 0


def test_ozaki_deterministic_and_matches_fp64_closely(cq):
    m, n = 30000, 64
    A = to_dev(synth.make_matrix(m, n, 1e5, seed=23))
    with cq.Plan(m, n, precision=cq.CQR2_OZAKI_BF16) as p:
        Q1, R1, _ = p.factor(A)
        Q2, R2, _ = p.factor(A)
    assert bool((Q1 == Q2).all()) and bool((R1 == R2).all())
    with cq.Plan(m, n) as p:
        Qf, Rf, _ = p.factor(A)
    rel = float(((R1 - Rf).norm() / Rf.norm()).item())
    assert rel <= 1e-13 * 1e5


def test_ozaki_nan_reports_not_spd(cq):
    m, n = 2000, 40
    A = synth.make_matrix(m, n, None, seed=5)
    A[100, 7] = np.nan
    with cq.Plan(m, n, precision=cq.CQR2_OZAKI_BF16) as p:
        with pytest.raises(cq.CQR2Error) as e:
            p.factor(to_dev(A))
    assert e.value.status == cq.CQR2_ERR_NOT_SPD and e.value.info.failed_pass == 1


def test_ozaki_rejects_large_n(cq):
    with pytest.raises(cq.CQR2Error) as e:
        cq.Plan(17000, 16385, precision=cq.CQR2_OZAKI_BF16)
    assert e.value.status == cq.CQR2_ERR_UNSUPPORTED


@pytest.mark.parametrize("m,n,kappa", [(8192, 2048, 1e4), (6000, 4100, 1e3)])
def test_ozaki_cqr2_large_n(cq, m, n, kappa):
    # near-square shapes: many Gram tiles per row range, long Q-form contractions
    A = synth.make_matrix(m, n, kappa, seed=m + n)
    with cq.Plan(m, n, precision=cq.CQR2_OZAKI_BF16) as p:
        Q, R, info = p.factor(to_dev(A))
    assert info.status == 0
    _check(A, to_host(Q), to_host(R), kappa)
