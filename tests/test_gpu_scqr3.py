"""Shifted CholeskyQR3 (CQR2_SHIFTED) on the GPU against the oracle's scqr3.

Up to kappa 1e12 the method is unconditionally stable: Q is orthonormal and
QR = A to working accuracy, and R agrees with the oracle's. Tolerances:
orthogonality and residual <= 100 n eps (FP64; x10 for split precision),
R relative <= 1e-12 against the oracle (both backward stable; x10 split).
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


def _shifted_plan(cq, m, n, prec):
    from paper_1710_08471_gb300 import _native as N
    import ctypes as C

    h = C.c_void_p()
    N.check(N.load().cqr2_plan_create(C.byref(h), m, n, prec, 0x4, cq._stream_handle()), "cqr2_plan_create")
    return h


@pytest.mark.parametrize("prec,scale", [(0, 1.0), (1, 10.0)])
@pytest.mark.parametrize("m,n,kappa", [(4096, 48, 1e2), (6000, 64, 1e9), (5000, 128, 1e12), (3001, 300, 1e10),
                                       (777, 33, 1e11)])
def test_scqr3_matches_oracle(cq, m, n, kappa, prec, scale):
    if prec and n > 1024:
        pytest.skip()
    A = synth.make_matrix(m, n, kappa, seed=m + n)
    Qo, Ro = oracle.scqr3(A)
    h = _shifted_plan(cq, m, n, prec)
    try:
        Q = cq.empty_colmajor(m, n, device="cuda")
        R = cq.empty_colmajor(n, n, device="cuda")
        info = cq.cqr2_factor(h, m, n, to_dev(A), Q, R)
    finally:
        cq.cqr2_plan_destroy(h)
    assert info.status == 0
    Qh, Rh = to_host(Q), to_host(R)
    assert np.array_equal(Rh, np.triu(Rh)) and np.all(np.diag(Rh) > 0)
    assert oracle.orthogonality(Qh) <= scale * 100 * n * EPS
    assert oracle.residual(A, Qh, Rh) <= scale * 100 * n * EPS
    assert oracle.rel_error(Rh, Ro) <= scale * 1e-12


def test_cqr2_breaks_down_where_scqr3_does_not(cq):
    m, n = 4000, 40
    A = synth.make_matrix(m, n, 1e10, seed=9)
    with cq.Plan(m, n) as p:
        with pytest.raises(cq.CQR2Error) as e:
            p.factor(to_dev(A))
    assert e.value.status == cq.CQR2_ERR_NOT_SPD
    h = _shifted_plan(cq, m, n, 0)
    try:
        Q = cq.empty_colmajor(m, n, device="cuda")
        R = cq.empty_colmajor(n, n, device="cuda")
        info = cq.cqr2_factor(h, m, n, to_dev(A), Q, R)
    finally:
        cq.cqr2_plan_destroy(h)
    assert info.status == 0 and oracle.orthogonality(to_host(Q)) <= 100 * n * EPS
