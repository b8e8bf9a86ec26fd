"""CholeskyQR2 on column panels (cqr2_plan_set_panel_width), the library's
reading of the subpanel variant named as future work in Section V, against
the oracle's panel_cqr2 on the same inputs.

Tolerances are those of plain native-FP64 CholeskyQR2: orthogonality <=
max(1e-12, 10x the oracle's), residual <= max(1e-13, 10x the oracle's), R
relative to the oracle's <= 1e-12 kappa (R is unique, so it is also held to
the oracle's plain CQR2 R)."""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cq():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_08471_gb300 as m

    return m


def _check(A, Q, R, b, kappa):
    Qo, Ro = oracle.panel_cqr2(A, b)
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R) > 0)
    assert oracle.orthogonality(Q) <= max(1e-12, 10 * oracle.orthogonality(Qo))
    assert oracle.residual(A, Q, R) <= max(1e-13, 10 * oracle.residual(A, Qo, Ro))
    assert oracle.rel_error(R, Ro) <= 1e-12 * kappa
    _, Rc = oracle.cqr2(A)
    assert oracle.rel_error(R, Rc) <= 1e-12 * kappa


@pytest.mark.parametrize("m,n,b,kappa", [(3000, 700, 256, 1e4), (2048, 512, 128, 1e6), (1500, 300, 64, 1e5),
                                         (900, 200, 16, 1e3), (5000, 1100, 512, 1e4), (640, 130, 100, 1e2)])
def test_panels_match_oracle(cq, m, n, b, kappa):
    A = synth.make_matrix(m, n, kappa, seed=m + n + b)
    with cq.Plan(m, n) as p:
        p.set_panel_width(b)
        Q, R, info = p.factor(to_dev(A))
    assert info.status == 0
    _check(A, to_host(Q), to_host(R), b, kappa)


def test_panels_near_square_full_size(cq):
    """8192 x 4096, panels of 512: parity with the oracle and the time against
    plain CholeskyQR2 on the same plan (printed; either may be faster)."""
    import torch

    m, n, b, kappa = 8192, 4096, 512, 1e4
    A = synth.make_matrix(m, n, kappa, seed=61)
    Ad = to_dev(A)
    times = {}
    with cq.Plan(m, n) as p:
        for width in (0, b):
            p.set_panel_width(width)
            Q, R, info = p.factor(Ad)
            assert info.status == 0
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(3):
                p.factor(Ad, Q, R, sync=False)
            torch.cuda.synchronize()
            times[width] = (time.perf_counter() - t0) / 3
    print(f"8192x4096 plain {1e3 * times[0]:.1f} ms, panels of {b}: {1e3 * times[b]:.1f} ms")
    _check(A, to_host(Q), to_host(R), b, kappa)


def test_panels_inplace_and_host_paths_bit_exact(cq):
    m, n, b = 2500, 600, 192
    A = synth.make_matrix(m, n, 1e5, seed=62)
    with cq.Plan(m, n, inplace=True) as p:
        p.set_panel_width(b)
        Ad = to_dev(A)
        Q, R, _ = p.factor(Ad)
        Q, R = to_host(Q), to_host(R)
        A2 = to_dev(A)
        Q2, R2, _ = p.factor(A2, A2)  # Q over A
        np.testing.assert_array_equal(to_host(Q2), Q)
        np.testing.assert_array_equal(to_host(R2), R)
        hQ = np.zeros((m, n), order="F")
        hR = np.zeros((n, n), order="F")
        info = p.factor_host(np.asfortranarray(A), hQ, hR)
        assert info.status == 0
        np.testing.assert_array_equal(hQ, Q)
        np.testing.assert_array_equal(hR, R)


def test_one_panel_is_plain_cqr2(cq):
    m, n = 3000, 300
    A = to_dev(synth.make_matrix(m, n, 1e4, seed=63))
    with cq.Plan(m, n) as p:
        Q0, R0, _ = p.factor(A)
        p.set_panel_width(n)  # b >= n: off
        Q1, R1, _ = p.factor(A)
    assert bool((Q0 == Q1).all()) and bool((R0 == R1).all())


def test_panels_breakdown_reports_column_of_A(cq):
    m, n, b = 1000, 200, 64
    A = synth.make_matrix(m, n, 1e2, seed=53)
    A[:, 150] = 0.0
    with cq.Plan(m, n) as p:
        p.set_panel_width(b)
        with pytest.raises(cq.CQR2Error) as e:
            p.factor(to_dev(A))
    assert e.value.status == cq.CQR2_ERR_NOT_SPD
    assert e.value.info.failed_pass == 1 and e.value.info.failed_pivot == 150


def test_panels_least_squares(cq):
    m, n, b = 4000, 500, 128
    A = synth.make_matrix(m, n, 1e3, seed=64)
    bvec = synth.make_rhs(m, seed=64)
    with cq.Plan(m, n) as p:
        p.set_panel_width(b)
        x, info = p.lstsq(to_dev(A), to_dev(bvec))
    xo = oracle.lstsq(A, bvec)
    assert np.linalg.norm(to_host(x) - xo) <= 1e-12 * 1e3 * np.linalg.norm(xo)


def test_panels_unsupported_combinations(cq):
    with cq.Plan(2000, 300, precision=cq.CQR2_OZAKI_BF16) as p:
        with pytest.raises(cq.CQR2Error) as e:
            p.set_panel_width(64)
        assert e.value.status == cq.CQR2_ERR_UNSUPPORTED
    with cq.Plan(2000, 300, shifted=True) as p:
        with pytest.raises(cq.CQR2Error) as e:
            p.set_panel_width(64)
        assert e.value.status == cq.CQR2_ERR_UNSUPPORTED
    with cq.Plan(2000, 300) as p:
        with pytest.raises(cq.CQR2Error) as e:
            p.set_panel_width(-1)
        assert e.value.status == cq.CQR2_ERR_INVALID_ARG
