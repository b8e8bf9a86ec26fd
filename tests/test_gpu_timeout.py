"""The bounded-wait timeout path, made to run out on purpose without a fault:
a wait on an mbarrier that nothing arrives at gives up after its poll limit,
the status word says CQR2_ERR_TIMEOUT, and the context keeps working."""
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


def test_wait_runs_out_and_reports_timeout(cq):
    from paper_1710_08471_gb300 import _native as N

    lib = N.load()
    assert lib.cqr2_selftest_wait_timeout(1 << 14, cq._stream_handle()) == cq.CQR2_ERR_TIMEOUT
    for bad in (0, -1, (1 << 24) + 1):
        assert lib.cqr2_selftest_wait_timeout(bad, cq._stream_handle()) == cq.CQR2_ERR_INVALID_ARG
    # the context is intact: a split-precision factorization (the kernel whose waits these are) still works
    m, n = 5000, 96
    A = synth.make_matrix(m, n, 1e4, seed=3)
    with cq.Plan(m, n, precision=cq.CQR2_OZAKI_BF16) as p:
        Q, R, info = p.factor(to_dev(A))
    assert info.status == 0
    assert oracle.orthogonality(to_host(Q)) <= 100 * n * EPS
