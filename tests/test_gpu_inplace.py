"""CQR2_INPLACE (Q written over A) on every path, and least squares with
no Q argument (Q in the plan's own buffer). The in-place result must be the
out-of-place result bit for bit: the same kernels compute the same values,
only the destination differs. Both are also checked against the CPU FP64
oracle with the FP64 (x10 for split precision) tolerances."""
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


CASES = [
    # m, n, precision, fused, shifted, inverse depth, kappa
    (20000, 64, 0, True, False, 0, 1e6),      # fused Q-form + Gram on the panel path
    (20000, 128, 0, False, False, 0, 1e4),    # panel Q-form, not fused
    (6000, 300, 0, False, False, 0, 1e4),     # tiled multiply, Q1 in the workspace
    (6000, 300, 0, False, False, 1, 1e4),     # block forward substitution
    (6000, 300, 0, False, True, 0, 1e10),     # shifted, tiled: Q0 staged and copied over A
    (20000, 100, 0, False, True, 0, 1e10),    # shifted, panel path
    (20000, 128, 1, False, False, 0, 1e6),    # split precision
    (20000, 64, 1, False, True, 0, 1e8),      # split precision, shifted
]


@pytest.mark.parametrize("m,n,prec,fused,shifted,depth,kappa", CASES)
def test_inplace_equals_out_of_place(cq, m, n, prec, fused, shifted, depth, kappa):
    A = synth.make_matrix(m, n, kappa, seed=n + m)
    dA = to_dev(A)
    with cq.Plan(m, n, precision=prec, fused=fused, shifted=shifted, inplace=True) as p:
        if depth:
            p.set_inverse_depth(depth)
        Q0, R0, info0 = p.factor(dA)
        assert info0.status == 0
        W = dA.clone().t().contiguous().t()  # column-major copy, overwritten by Q
        assert W.stride() == (1, m)
        Q1, R1, info1 = p.factor(W, Q=W)
        assert info1.status == 0 and Q1.data_ptr() == W.data_ptr()
    assert bool((W == Q0).all()) and bool((R1 == R0).all())
    scale = 1.0 if prec == 0 else 10.0
    Q, R = to_host(W), to_host(R1)
    if shifted:
        # shifted CholeskyQR3 bounds (as in test_gpu_scqr3)
        Qo, Ro = oracle.scqr3(A)
        assert oracle.orthogonality(Q) <= scale * 100 * n * EPS
        assert oracle.residual(A, Q, R) <= scale * 100 * n * EPS
        assert oracle.rel_error(R, Ro) <= scale * 1e-12
    else:
        Qo, Ro = oracle.cqr2(A)
        assert oracle.orthogonality(Q) <= scale * max(1e-12, 10 * oracle.orthogonality(Qo))
        assert oracle.residual(A, Q, R) <= scale * max(1e-13, 10 * oracle.residual(A, Qo, Ro))
        assert oracle.rel_error(R, Ro) <= scale * 1e-12 * kappa


def test_alias_needs_the_flag(cq):
    m, n = 2000, 32
    dA = to_dev(synth.make_matrix(m, n, 10.0, seed=1))
    with cq.Plan(m, n) as p:
        with pytest.raises(Exception):
            p.factor(dA, Q=dA)
    # same pointer with another leading dimension: rejected even with the flag
    import torch

    buf = torch.zeros((m + 8) * n, dtype=torch.float64, device="cuda")
    A8 = buf.as_strided((m, n), (1, m + 8))
    A8.copy_(dA)
    Qm = buf.as_strided((m, n), (1, m))
    with cq.Plan(m, n, inplace=True) as p:
        with pytest.raises(Exception):
            p.factor(A8, Q=Qm)


@pytest.mark.parametrize("prec", [0, 1])
def test_lstsq_without_q(cq, prec):
    """No Q argument: Q goes to the plan's buffer; x is the same as with a
    caller's Q, over repeated calls and uneven m."""
    n = 48
    with cq.Plan(9000, n, precision=prec) as p:
        for m, kappa in ((9000, 1e4), (3001, 1e2), (9000, 1e3)):
            A = synth.make_matrix(m, n, kappa, seed=m + 7)
            b = synth.make_rhs(m, seed=m)
            dA, db = to_dev(A), to_dev(b)
            x1, info1 = p.lstsq_rows(dA, db)
            x2, info2 = p.lstsq_rows(dA, db, keep_q=False)
            assert info1.status == 0 and info2.status == 0
            assert bool((x1 == x2).all())
            xo = oracle.lstsq(A, b)
            scale = 1.0 if prec == 0 else 10.0
            assert np.linalg.norm(to_host(x2) - xo) <= scale * 1e-12 * kappa * np.linalg.norm(xo)
