"""Full-size parity, in the launch configuration bench.py times.

Workloads (seeded, synth.make_matrix):
  tall     m = 2^23, n = 128, kappa = 1e6 (the benchmark's default workload)
  wide512  m = 2^21, n = 512, kappa in {1e2, 1e4, 1e6, 1e7} (split precision)
  square   m = 65536, n = 8192, kappa = 1e4 (FP64, recursive CholInv)

R is compared with the CPU FP64 oracle's R in full; Q on a sample of rows
(Q = A R^-1 acts row by row, so the oracle's rows are exact counterparts);
orthogonality and the residual are measured over the whole Q on the device.
Tolerances: FP64 as in test_gpu_parity (orthogonality <= 1e-12 or 10x the
oracle's own, residual <= 1e-13, R relative <= 1e-12 kappa); split precision
ten times those.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_dev, to_host

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def cq():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_08471_gb300 as m

    return m


def device_metrics(A_d, Q, R):
    """||Q^T Q - I||_F and ||QR - A||_F / ||A||_F over the whole matrices."""
    import torch

    n = Q.shape[1]
    G = Q.t() @ Q
    G -= torch.eye(n, dtype=G.dtype, device=G.device)
    orth = float(torch.linalg.norm(G).item())
    num = 0.0
    den = 0.0
    for r0 in range(0, Q.shape[0], 1 << 21):
        a = A_d[r0:r0 + (1 << 21)]
        d = Q[r0:r0 + (1 << 21)] @ R - a
        num += float((d * d).sum().item())
        den += float((a * a).sum().item())
    return orth, (num / den) ** 0.5


def sampled_rows(m, k=4096, seed=0):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(m, size=min(k, m), replace=False))


def check_full(cq, A, Qo, Ro, prec, fused, kappa, scale, oracle_orth, oracle_res):
    import torch

    m, n = A.shape
    A_d = to_dev(A)
    with cq.Plan(m, n, precision=prec, fused=fused) as p:
        Q, R, info = p.factor(A_d)
    assert info.status == 0
    Rh = to_host(R)
    assert np.array_equal(Rh, np.triu(Rh)) and np.all(np.diag(Rh) > 0)
    assert oracle.rel_error(Rh, Ro) <= scale * 1e-12 * kappa
    rows = sampled_rows(m)
    Qs = to_host(Q[torch.from_numpy(rows).cuda()])
    Qos = Qo[rows]
    assert np.linalg.norm(Qs - Qos) <= scale * 1e-12 * kappa * np.linalg.norm(Qos)
    orth, res = device_metrics(A_d, Q, R)
    assert orth <= scale * max(1e-12, 10 * oracle_orth), orth
    assert res <= scale * max(1e-13, 10 * oracle_res), res
    del Q, R, A_d
    torch.cuda.empty_cache()


@pytest.fixture(scope="module")
def tall():
    A = synth.make_matrix(1 << 23, 128, 1e6, seed=1)
    Qo, Ro = oracle.cqr2(A)
    return A, Qo, Ro, oracle.orthogonality(Qo), oracle.residual(A, Qo, Ro)


@pytest.mark.parametrize("prec,fused,scale", [(0, True, 1.0), (0, False, 1.0), (1, False, 10.0)])
def test_tall_full_size(cq, tall, prec, fused, scale):
    A, Qo, Ro, oo, orr = tall
    check_full(cq, A, Qo, Ro, prec, fused, 1e6, scale, oo, orr)


@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6, 1e7])
def test_wide512_ozaki_kappa_sweep(cq, kappa):
    A = synth.make_matrix(1 << 21, 512, kappa, seed=3 + int(np.log10(kappa)))
    Qo, Ro = oracle.cqr2(A)
    check_full(cq, A, Qo, Ro, 1, False, kappa, 10.0, oracle.orthogonality(Qo), oracle.residual(A, Qo, Ro))


def test_square_fp64_full_size(cq):
    A = synth.make_matrix(65536, 8192, 1e4, seed=2)
    Qo, Ro = oracle.cqr2(A)
    check_full(cq, A, Qo, Ro, 0, False, 1e4, 1.0, oracle.orthogonality(Qo), oracle.residual(A, Qo, Ro))
