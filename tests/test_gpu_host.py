"""cqr2_factor_host: host buffers in and out, copies overlapped with the work.

A arrives in row blocks on a copy stream while the pass-1 Gram consumes them,
and Q leaves block by block as the last Q-form writes it. The results must
satisfy the same bounds as the device-buffer path, for every variant (FP64
fused and unfused, n above the small-panel limit, split precision, shifted
CholeskyQR3), with leading dimensions larger than m and with row counts that
leave some blocks empty.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from gpu_util import EPS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cq():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_08471_gb300 as m

    return m


def _run(cq, m, n, kappa, precision=0, fused=True, flags=0, pad=0, reps=2):
    from paper_1710_08471_gb300 import _native as N
    import ctypes as C

    A = synth.make_matrix(m, n, kappa, seed=m + 3 * n)
    hA = np.zeros((m + pad, n), order="F")
    hA[:m] = A
    hQ = np.full((m + pad, n), np.nan, order="F")
    hR = np.full((n, n), np.nan, order="F")
    h = C.c_void_p()
    fl = flags | (N.CQR2_FUSED if fused else 0)
    N.check(N.load().cqr2_plan_create(C.byref(h), m, n, precision, fl, cq._stream_handle()), "cqr2_plan_create")
    try:
        for _ in range(reps):
            info = N.Info()
            st = N.load().cqr2_factor_host(h, hA.ctypes.data, hA.shape[0], hQ.ctypes.data, hQ.shape[0],
                                           hR.ctypes.data, n, C.byref(info))
            N.check(st, "cqr2_factor_host", info)
    finally:
        cq.cqr2_plan_destroy(h)
    assert np.array_equal(hA[:m], A)  # input untouched
    if pad:
        assert np.all(np.isnan(hQ[m:]))  # rows beyond m of the host Q are not written
    return A, np.asfortranarray(hQ[:m]), hR


def _check(A, Q, R, kappa, scale=1.0):
    n = A.shape[1]
    Qo, Ro = oracle.cqr2(A)
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R) > 0)
    assert oracle.orthogonality(Q) <= scale * max(100 * n * EPS, 10 * oracle.orthogonality(Qo))
    assert oracle.residual(A, Q, R) <= scale * max(100 * n * EPS, 10 * oracle.residual(A, Qo, Ro))
    assert oracle.rel_error(R, Ro) <= scale * 1e-12 * kappa


@pytest.mark.parametrize("m,n,kappa,fused,pad", [(200003, 64, 1e4, True, 0), (200003, 64, 1e4, False, 5),
                                                 (5000, 128, 1e6, True, 0), (300, 40, 1e2, True, 3),
                                                 (20000, 300, 1e5, False, 0)])
def test_factor_host_fp64(cq, m, n, kappa, fused, pad):
    A, Q, R = _run(cq, m, n, kappa, fused=fused, pad=pad)
    _check(A, Q, R, kappa)


def test_factor_host_matches_device_path_closely(cq):
    # the blocked pass-1 Gram sums in another order, so agreement is to rounding
    from gpu_util import to_dev, to_host

    m, n = 100000, 96
    A, Q, R = _run(cq, m, n, 1e3)
    with cq.Plan(m, n) as p:
        Qd, Rd, info = p.factor(to_dev(A))
    assert np.max(np.abs(to_host(Qd) - Q)) <= 1e-12
    assert oracle.rel_error(R, to_host(Rd)) <= 1e-13


def test_factor_host_split_precision(cq):
    A, Q, R = _run(cq, 50000, 128, 1e6, precision=1, fused=False)
    _check(A, Q, R, 1e6, scale=10.0)


def test_factor_host_shifted(cq):
    # shifted CholeskyQR3 through the host path: kappa beyond plain CQR2's reach
    A, Q, R = _run(cq, 30000, 48, 1e10, flags=0x4, fused=False)
    Qo, Ro = oracle.scqr3(A)
    assert oracle.orthogonality(Q) <= 100 * 48 * EPS
    assert oracle.residual(A, Q, R) <= 100 * 48 * EPS
    assert oracle.rel_error(R, Ro) <= 1e-12


def test_factor_host_stage_times(cq):
    m, n = 65536, 64
    A = synth.make_matrix(m, n, 1e2, seed=5)
    hA, hQ, hR = np.asfortranarray(A), np.zeros((m, n), order="F"), np.zeros((n, n), order="F")
    with cq.Plan(m, n) as p:
        p.factor_host(hA, hQ, hR)
        p.set_profiling(True)
        p.factor_host(hA, hQ, hR)
        st = p.stage_times()
        p.set_profiling(False)
    assert st["h2d"][1] == 1 and st["h2d"][0] > 0
    assert st["d2h"][1] >= 1 and st["d2h"][0] > 0
    _check(A, hQ, hR, 1e2)
