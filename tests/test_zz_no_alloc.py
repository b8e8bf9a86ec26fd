"""The allocation-free Gram entry point, cqr2_syrk_noalloc.

Some callers cannot allocate device memory (a host that gives all of it to
its own pool allocator, or code where a cudaMalloc could fail or stall in the
middle of a job). For them cqr2_syrk_noalloc computes W = A^T A with its
partial sums in a fixed scratch array inside the library. This file checks,
through the C ABI, that two calls in a row give the same Gram as the plan-based
entry point cqr2_syrk and as the CPU oracle's Syrk, within the Gram tolerance
the other tests use (|W - W_ref| <= 2 m eps (|A|^T |A|) elementwise), and
that pointers the kernels could not read on this device are refused before
anything is launched. The file is named so that pytest collects it last.
"""
from __future__ import annotations

import ctypes

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


def _noalloc_raw(cq, m, n, A, W):
    """Call the C entry point directly through ctypes."""
    import torch

    from paper_1710_08471_gb300 import _native

    lib = _native.load()
    st = lib.cqr2_syrk_noalloc(ctypes.c_void_p(A.data_ptr()), m, n, A.stride(1) if n > 1 else m,
                               ctypes.c_void_p(W.data_ptr()), W.stride(1) if n > 1 else n,
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st


@pytest.mark.parametrize("m,n,kappa", [(20000, 128, 1e6), (3001, 300, 1e3), (777, 33, None), (5000, 1, None),
                                       (1 << 20, 64, 1e4)])
def test_noalloc_matches_plan_syrk_twice(cq, m, n, kappa):
    import torch

    A = synth.make_matrix(m, n, kappa, seed=m + 7 * n)
    Ad = to_dev(A)
    with cq.Plan(m, n) as p:
        W_plan = to_host(p.syrk(Ad))
    W_oracle = oracle.syrk(A)
    absA = np.abs(A)
    bound = 2 * m * EPS * (absA.T @ absA)
    outs = []
    for call in range(2):
        W = cq.empty_colmajor(n, n, device="cuda")
        W.fill_(float("nan"))
        if call == 0:
            assert _noalloc_raw(cq, m, n, Ad, W) == cq.CQR2_OK
        else:  # the public Python wrapper over the same entry point
            cq.cqr2_syrk_noalloc(m, n, Ad, W, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        Wh = to_host(W)
        assert np.all(np.abs(Wh - W_plan) <= bound + 1e-300)
        assert np.all(np.abs(Wh - W_oracle) <= bound + 1e-300)
        assert np.array_equal(Wh, Wh.T)
        outs.append(Wh)
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_after_different_shape_reuses_scratch(cq):
    """A small call after a large one must not see the large call's leftovers."""
    import torch

    big = to_dev(synth.make_matrix(50000, 256, 1e3, seed=1))
    Wb = cq.empty_colmajor(256, 256, device="cuda")
    assert _noalloc_raw(cq, 50000, 256, big, Wb) == cq.CQR2_OK
    A = synth.make_matrix(300, 40, 10.0, seed=2)
    W = cq.empty_colmajor(40, 40, device="cuda")
    assert _noalloc_raw(cq, 300, 40, to_dev(A), W) == cq.CQR2_OK
    torch.cuda.synchronize()
    absA = np.abs(A)
    assert np.all(np.abs(to_host(W) - A.T @ A) <= 2 * 300 * EPS * (absA.T @ absA) + 1e-300)


def test_noalloc_rejects_sizes_beyond_maximum(cq):
    from paper_1710_08471_gb300 import _native

    lib = _native.load()
    n = 2817  # one more than CQR2_NOALLOC_MAX_N
    p = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    assert lib.cqr2_syrk_noalloc(p, n, n, n, p, n, None) == cq.CQR2_ERR_UNSUPPORTED
    assert lib.cqr2_syrk_noalloc(p, 10, 20, 10, p, 20, None) == cq.CQR2_ERR_INVALID_ARG
    assert lib.cqr2_syrk_noalloc(None, 10, 5, 10, p, 5, None) == cq.CQR2_ERR_INVALID_ARG


def test_noalloc_rejects_host_pointers(cq):
    """A host array (pageable or pinned) is refused with INVALID_ARG before any
    kernel is launched."""
    import torch

    from paper_1710_08471_gb300 import _native

    lib = _native.load()
    m, n = 256, 8
    hA = np.asfortranarray(synth.make_matrix(m, n, None, seed=3))
    W = cq.empty_colmajor(n, n, device="cuda")
    Wp = ctypes.c_void_p(W.data_ptr())
    assert lib.cqr2_syrk_noalloc(ctypes.c_void_p(hA.ctypes.data), m, n, m, Wp, n, None) == cq.CQR2_ERR_INVALID_ARG
    pinned = torch.empty((n, m), dtype=torch.float64, pin_memory=True)
    assert lib.cqr2_syrk_noalloc(ctypes.c_void_p(pinned.data_ptr()), m, n, m, Wp, n, None) == cq.CQR2_ERR_INVALID_ARG
    Ad = to_dev(hA)
    hW = np.zeros((n, n), order="F")
    assert lib.cqr2_syrk_noalloc(ctypes.c_void_p(Ad.data_ptr()), m, n, m, ctypes.c_void_p(hW.ctypes.data), n,
                                 None) == cq.CQR2_ERR_INVALID_ARG
    # and the device pair still works afterwards
    assert lib.cqr2_syrk_noalloc(ctypes.c_void_p(Ad.data_ptr()), m, n, m, Wp, n, None) == cq.CQR2_OK
    torch.cuda.synchronize()
    absA = np.abs(hA)
    assert np.all(np.abs(to_host(W) - oracle.syrk(hA)) <= 2 * m * EPS * (absA.T @ absA) + 1e-300)
