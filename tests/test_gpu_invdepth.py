"""Inverse depth on the GPU against the oracle's cholinv_depth / right_solve.

At depth d the top d halvings of CholInv leave Y21 unformed and L21 and Q come
from block forward substitution. The GPU splits at multiples of 64 where the
oracle halves exactly, so the inverted blocks differ and the comparison is to
rounding: the bounds of the FP64 parity tests (orthogonality and residual
within ten times the oracle's own, R within 1e-12 kappa of the oracle's).
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


def _check(A, Q, R, kappa, depth):
    n = A.shape[1]
    Qo, Ro = oracle.cqr2(A, inverse_depth=depth)
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R) > 0)
    assert oracle.orthogonality(Q) <= max(100 * n * EPS, 10 * oracle.orthogonality(Qo))
    assert oracle.residual(A, Q, R) <= max(100 * n * EPS, 10 * oracle.residual(A, Qo, Ro))
    assert oracle.rel_error(R, Ro) <= 1e-12 * kappa


@pytest.mark.parametrize("m,n,kappa", [(2000, 300, 1e3), (3000, 520, 1e7), (4100, 1030, 1e5)])
@pytest.mark.parametrize("depth", [1, 2, 4])
def test_inverse_depth_matches_oracle(cq, m, n, kappa, depth):
    A = synth.make_matrix(m, n, kappa, seed=m + n + depth)
    with cq.Plan(m, n) as p:
        p.set_inverse_depth(depth)
        Q, R, info = p.factor(to_dev(A))
    assert info.status == 0
    _check(A, to_host(Q), to_host(R), kappa, depth)


def test_depth_zero_is_the_default_bit_for_bit(cq):
    m, n = 2500, 400
    A = to_dev(synth.make_matrix(m, n, 1e4, seed=8))
    with cq.Plan(m, n) as p:
        Q0, R0, _ = p.factor(A)
        Q0, R0 = to_host(Q0), to_host(R0)
        p.set_inverse_depth(3)
        p.set_inverse_depth(0)
        Q1, R1, _ = p.factor(A)
    assert np.array_equal(Q0, to_host(Q1)) and np.array_equal(R0, to_host(R1))


def test_inverse_depth_host_path_and_rows(cq):
    m, n = 6000, 320
    A = synth.make_matrix(m, n, 1e5, seed=10)
    hQ, hR = np.zeros((m, n), order="F"), np.zeros((n, n), order="F")
    with cq.Plan(m, n) as p:
        p.set_inverse_depth(2)
        p.factor_host(np.asfortranarray(A), hQ, hR)
        _check(A, hQ, hR, 1e5, 2)
        Q, R, info = p.factor_rows(to_dev(A[:4000]))
        assert info.status == 0
        _check(A[:4000], to_host(Q), to_host(R), 1e5, 2)


def test_inverse_depth_shifted(cq):
    from paper_1710_08471_gb300 import _native as N
    import ctypes as C

    m, n = 5000, 300
    A = synth.make_matrix(m, n, 1e11, seed=12)
    h = C.c_void_p()
    N.check(N.load().cqr2_plan_create(C.byref(h), m, n, 0, 0x4, cq._stream_handle()), "create")
    try:
        cq.cqr2_plan_set_inverse_depth(h, 2)
        Q = cq.empty_colmajor(m, n, device="cuda")
        R = cq.empty_colmajor(n, n, device="cuda")
        info = cq.cqr2_factor(h, m, n, to_dev(A), Q, R)
    finally:
        cq.cqr2_plan_destroy(h)
    assert info.status == 0
    Qh, Rh = to_host(Q), to_host(R)
    assert oracle.orthogonality(Qh) <= 100 * n * EPS
    assert oracle.residual(A, Qh, Rh) <= 100 * n * EPS


def test_inverse_depth_refusals(cq):
    with cq.Plan(1000, 64) as p:  # small panel path: whole inverse only
        with pytest.raises(cq.CQR2Error) as e:
            p.set_inverse_depth(1)
        assert e.value.status == cq.CQR2_ERR_UNSUPPORTED
        p.set_inverse_depth(0)
    with cq.Plan(1000, 300, precision=1) as p:  # split precision
        with pytest.raises(cq.CQR2Error) as e:
            p.set_inverse_depth(2)
        assert e.value.status == cq.CQR2_ERR_UNSUPPORTED
    with cq.Plan(1000, 300) as p:
        for bad in (-1, 17):
            with pytest.raises(cq.CQR2Error) as e:
                p.set_inverse_depth(bad)
            assert e.value.status == cq.CQR2_ERR_INVALID_ARG
