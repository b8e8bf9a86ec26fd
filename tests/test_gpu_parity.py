"""GPU parity: every step of CholeskyQR2 through the C ABI against the CPU FP64
oracle, element by element, on seeded inputs spanning several tiles and
ragged tails.

Tolerances (all derived from FP64 rounding, eps = 2^-53):
* Gram W = A^T A: both sides sum the same m products in different orders, so
  |W_gpu - W_oracle| <= 2 m eps (|A|^T |A|) elementwise.
* Q = A R^-1: |Q_gpu - Q_oracle| <= 2 n eps (|A| |R^-1|) elementwise.
* CholInv: bitwise exact on the closed forms (every intermediate an integer);
  otherwise L within 10 n kappa(L) eps of the oracle, Y = L^-1 within
  10 n kappa(L)^2 eps (it inherits L's rounding amplified by kappa(L)), and
  the residuals L Y - I, Y L - I within 10 n kappa(L) eps.
* CholeskyQR2 end to end, FP64, kappa <= 1e6: ||Q^T Q - I||_F <= 1e-12,
  ||QR - A||_F / ||A||_F <= 1e-13, ||R - R_oracle||_F / ||R_oracle||_F <= 1e-12 kappa.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from closed_forms import minij, pascal
from gpu_util import EPS, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cq():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_08471_gb300 as m

    return m


SHAPES = [
    # m, n, kappa
    (4096, 64, None),
    (1000, 1, None),
    (64, 64, 10.0),
    (777, 33, 1e3),
    (3000, 100, 1e6),
    (5000, 128, 1e6),
    (2000, 129, 1e4),
    (4000, 256, 1e4),
    (3001, 300, 1e3),
    (1500, 520, 1e2),
]


@pytest.mark.parametrize("m,n,kappa", SHAPES)
def test_syrk(cq, m, n, kappa):
    A = synth.make_matrix(m, n, kappa, seed=m + n)
    with cq.Plan(m, n) as p:
        W = to_host(p.syrk(to_dev(A)))
    Wo = oracle.syrk(A)
    absA = np.abs(A)
    bound = 2 * m * EPS * (absA.T @ absA)
    assert np.all(np.abs(W - Wo) <= bound + 1e-300)
    assert np.array_equal(W, W.T)


@pytest.mark.parametrize("n", [1, 7, 64, 65, 100, 128, 200, 300, 512])
def test_cholinv_minij_bit_exact(cq, n):
    W, L, Y = minij(n)
    with cq.Plan(n, n) as p:
        Lg, Yg, info = p.cholinv(to_dev(W))
    assert info.status == 0
    np.testing.assert_array_equal(to_host(Lg), L)
    np.testing.assert_array_equal(to_host(Yg), Y)


@pytest.mark.parametrize("n", [2, 9, 16, 28])
def test_cholinv_pascal_bit_exact(cq, n):
    W, L, Y = pascal(n)
    with cq.Plan(n, n) as p:
        Lg, Yg, info = p.cholinv(to_dev(W))
    np.testing.assert_array_equal(to_host(Lg), L)
    np.testing.assert_array_equal(to_host(Yg), Y)


@pytest.mark.parametrize("n", [5, 64, 100, 257, 700])
def test_cholinv_vs_oracle(cq, n):
    A = synth.make_matrix(3 * n + 10, n, 1e3, seed=n)
    W = oracle.syrk(A)
    Lo, Yo = oracle.cholinv(W)
    with cq.Plan(n, n) as p:
        Lg, Yg, info = p.cholinv(to_dev(W))
    Lg, Yg = to_host(Lg), to_host(Yg)
    kl = np.linalg.cond(Lo)
    assert np.array_equal(Lg, np.tril(Lg)) and np.array_equal(Yg, np.tril(Yg))
    assert oracle.rel_error(Lg, Lo) <= 10 * n * kl * EPS
    # Y = L^-1 also inherits L's rounding amplified by kappa(L)
    assert oracle.rel_error(Yg, Yo) <= 10 * n * kl * kl * EPS
    assert np.linalg.norm(Lg @ Lg.T - W) <= 10 * n * EPS * np.linalg.norm(W)
    assert np.linalg.norm(Lg @ Yg - np.eye(n)) <= 10 * n * kl * EPS
    assert np.linalg.norm(Yg @ Lg - np.eye(n)) <= 10 * n * kl * EPS


def test_cholinv_reports_breakdown(cq):
    n = 100
    W = np.eye(n)
    W[70, 70] = -1.0
    with cq.Plan(n, n) as p:
        with pytest.raises(cq.CQR2Error) as e:
            p.cholinv(to_dev(W))
    assert e.value.status == cq.CQR2_ERR_NOT_SPD
    assert e.value.info.failed_pivot == 70 and e.value.info.failed_pass == 1


@pytest.mark.parametrize("m,n,kappa", SHAPES)
def test_qform(cq, m, n, kappa):
    A = synth.make_matrix(m, n, kappa, seed=2 * m + n)
    _, _, i1 = oracle.cqr(A)
    Rinv = i1["Rinv"]
    Rinv_garbage = Rinv + np.tril(np.full((n, n), 7.0), -1)  # lower part must be ignored
    with cq.Plan(m, n) as p:
        Q = to_host(p.qform(to_dev(A), to_dev(Rinv_garbage)))
    Qo = A @ Rinv
    bound = 2 * n * EPS * (np.abs(A) @ np.abs(Rinv))
    assert np.all(np.abs(Q - Qo) <= bound + 1e-300)


@pytest.mark.parametrize("n", [1, 5, 64, 127, 128, 129, 300])
def test_trmm_upper(cq, n):
    rng = np.random.default_rng(n)
    R2 = np.triu(rng.standard_normal((n, n))) + np.tril(np.ones((n, n)), -1) * 3.0  # garbage below
    R1 = np.triu(rng.standard_normal((n, n)))
    with cq.Plan(n, n) as p:
        R = to_host(p.trmm_upper(to_dev(R2), to_dev(R1)))
    Ro = np.triu(R2) @ R1
    assert np.array_equal(R, np.triu(R))
    bound = 2 * n * EPS * (np.abs(np.triu(R2)) @ np.abs(R1))
    assert np.all(np.abs(R - Ro) <= bound + 1e-300)


def _check_cqr2(A, Q, R, kappa):
    Qo, Ro = oracle.cqr2(A)
    k = kappa or 2.0
    orth = oracle.orthogonality(Q)
    res = oracle.residual(A, Q, R)
    rel = oracle.rel_error(R, Ro)
    assert np.array_equal(R, np.triu(R))
    assert np.all(np.diag(R) > 0)
    assert orth <= max(1e-12, 10 * oracle.orthogonality(Qo)), orth
    assert res <= max(1e-13, 10 * oracle.residual(A, Qo, Ro)), res
    assert rel <= 1e-12 * k, rel
    assert np.linalg.norm(Q - Qo) <= 1e-12 * k * np.sqrt(A.shape[1])
    return orth, res, rel


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("m,n,kappa", SHAPES)
def test_cqr2_end_to_end(cq, m, n, kappa, fused):
    A = synth.make_matrix(m, n, kappa, seed=m * 3 + n)
    with cq.Plan(m, n, fused=fused) as p:
        Q, R, info = p.factor(to_dev(A))
    assert info.status == 0 and info.failed_pass == 0
    _check_cqr2(A, to_host(Q), to_host(R), kappa)


def test_cqr2_padded_leading_dimension(cq):
    import torch

    m, n = 1000, 40
    A = synth.make_matrix(m, n, 1e2, seed=99)
    big = np.zeros((m + 13, n))
    big[:m] = A
    Ad = to_dev(big)[:m]
    assert Ad.stride(1) == m + 13
    Qb = cq.empty_colmajor(m + 5, n, device="cuda")[:m]
    Rb = cq.empty_colmajor(n + 3, n, device="cuda")[:n]
    with cq.Plan(m, n) as p:
        p.factor(Ad, Qb, Rb)
    torch.cuda.synchronize()
    _check_cqr2(A, to_host(Qb), to_host(Rb), 1e2)


def test_cqr2_repeated_calls_are_deterministic(cq):
    m, n = 20000, 96
    A = to_dev(synth.make_matrix(m, n, 1e5, seed=5))
    with cq.Plan(m, n, fused=True) as p:
        Q1, R1, _ = p.factor(A)
        Q2, R2, _ = p.factor(A)
    assert bool((Q1 == Q2).all()) and bool((R1 == R2).all())


def test_cqr2_breakdown_zero_column(cq):
    m, n = 500, 12
    A = synth.make_matrix(m, n, None, seed=3)
    A[:, 7] = 0.0
    with cq.Plan(m, n) as p:
        with pytest.raises(cq.CQR2Error) as e:
            p.factor(to_dev(A))
    assert e.value.status == cq.CQR2_ERR_NOT_SPD
    assert e.value.info.failed_pass == 1 and e.value.info.failed_pivot == 7


def test_cqr2_nan_input_reports_not_spd(cq):
    m, n = 300, 10
    A = synth.make_matrix(m, n, None, seed=4)
    A[17, 3] = np.nan
    with cq.Plan(m, n) as p:
        with pytest.raises(cq.CQR2Error) as e:
            p.factor(to_dev(A))
    assert e.value.status == cq.CQR2_ERR_NOT_SPD and e.value.info.failed_pass == 1


def test_plan_survives_breakdown(cq):
    m, n = 400, 16
    bad = synth.make_matrix(m, n, None, seed=1)
    bad[:, 0] = 0.0
    good = synth.make_matrix(m, n, None, seed=2)
    with cq.Plan(m, n) as p:
        with pytest.raises(cq.CQR2Error):
            p.factor(to_dev(bad))
        Q, R, info = p.factor(to_dev(good))
    assert info.status == 0
    _check_cqr2(good, to_host(Q), to_host(R), None)


def test_invalid_arguments(cq):
    import torch

    with pytest.raises(cq.CQR2Error) as e:
        cq.Plan(5, 10)
    assert e.value.status == cq.CQR2_ERR_INVALID_ARG
    with cq.Plan(100, 10) as p:
        A = cq.empty_colmajor(100, 10, device="cuda")
        with pytest.raises(cq.CQR2Error) as e:  # Q aliasing A is rejected
            cq.cqr2_factor(p.handle, 100, 10, A, A, cq.empty_colmajor(10, 10, device="cuda"))
        assert e.value.status == cq.CQR2_ERR_INVALID_ARG
    torch.cuda.synchronize()


@pytest.mark.parametrize("m,n,kappa", [(4096, 64, None), (3000, 100, 1e4), (2500, 256, 1e3), (2000, 300, 1e2)])
def test_lstsq(cq, m, n, kappa):
    A = synth.make_matrix(m, n, kappa, seed=7)
    b = synth.make_rhs(m, seed=7)
    xo = oracle.lstsq(A, b)
    with cq.Plan(m, n) as p:
        x, info = p.lstsq(to_dev(A), to_dev(b))
    x = to_host(x)
    k = kappa or 2.0
    assert np.linalg.norm(x - xo) <= 1e-12 * k * np.linalg.norm(xo)
    # consistent system: b = A x0
    x0 = np.linspace(-1, 1, n)
    with cq.Plan(m, n) as p:
        x, _ = p.lstsq(to_dev(A), to_dev(A @ x0))
    assert np.linalg.norm(to_host(x) - x0) <= 1e-12 * k * np.linalg.norm(x0)
