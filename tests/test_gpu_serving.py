"""The continuous-batching least-squares server: every request is answered,
every result matches the CPU FP64 oracle, and each result is bit-for-bit the
same whether the request was served alone (the only request the server saw)
or overlapped with the others (eight slots, small requests grouped)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from gpu_util import to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1710_08471_gb300 as cq
    from paper_1710_08471_gb300 import serving

    m_max = 24000
    pool = serving.InputPool(m_max, (16, 32, 64, 128), seed=300)  # kappa grid 1 .. 1e5, four per decade
    stream = synth.request_stream(40, seed=300, rate=2000.0, m_lo=1024, m_hi=m_max, n_choices=(16, 32, 64, 128))
    return cq, serving, pool, stream, m_max


def _serve(env, slots, precision=0, budget=8e9, realtime=False, group_max=64):
    cq, serving, pool, stream, m_max = env
    reqs = [pool.request(r["id"], r["t"], r["m"], r["n"], r["kappa"]) for r in stream]
    srv = serving.Server(budget, slots=slots, precision=precision, m_max=m_max, n_values=(16, 32, 64, 128),
                         group_max=group_max)
    try:
        stats = srv.run(reqs, realtime=realtime)
    finally:
        srv.close()
    return reqs, stats


@pytest.mark.parametrize("precision,tol,group_max", [(0, 1e-12, 64), (1, 1e-11, 64), (0, 1e-12, 1)])
def test_serving_matches_oracle(env, precision, tol, group_max):
    cq, serving, pool, stream, m_max = env
    reqs, stats = _serve(env, slots=6, precision=precision, group_max=group_max)
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    # small requests (n <= 64, m n^2 <= 2^24) ran in grouped launches
    small = sum(1 for r in reqs if r.n <= 64 and r.m * r.n * r.n <= 1 << 24)
    assert small > 0 and stats["grouped_requests"] == (small if group_max > 1 else 0)
    kappa_of = {q["id"]: pool.kappa_of(q["kappa"]) for q in stream}
    for r in reqs:
        A = to_host(r.A_src)
        b = to_host(r.b_src)
        xo = oracle.lstsq(A, b)
        assert np.linalg.norm(to_host(r.x) - xo) <= tol * kappa_of[r.id] * np.linalg.norm(xo), r.id


def test_same_result_alone_and_in_the_mix(env):
    cq, serving, pool, stream, m_max = env
    mixed, st = _serve(env, slots=8)
    assert st["completed"] == len(mixed) and st["grouped_requests"] > 0
    # each request served on its own: the server sees no other request
    srv = serving.Server(8e9, slots=1, m_max=m_max, n_values=(16, 32, 64, 128))
    try:
        for q, b in zip(stream, mixed):
            a = pool.request(q["id"], q["t"], q["m"], q["n"], q["kappa"])
            st1 = srv.run([a], realtime=False)
            assert st1["completed"] == 1 and a.status == 0
            assert a.id == b.id
            assert bool((a.x == b.x).all()), a.id
    finally:
        srv.close()


def test_realtime_admission_under_small_budget(env):
    cq, serving, pool, stream, m_max = env
    # room for the plans plus about two of the largest requests at a time
    reqs = [pool.request(r["id"], r["t"], r["m"], r["n"], r["kappa"]) for r in stream[:20]]
    srv = serving.Server(1e12, slots=4, m_max=m_max, n_values=(16, 32, 64, 128))
    try:
        srv.budget = srv.workspace_bytes + 2 * 8 * (2 * m_max * 128 + 128 * 128 + m_max + 128)
        stats = srv.run(reqs, realtime=True)
    finally:
        srv.close()
    assert stats["completed"] == 20 and stats["failed"] == 0
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    for r in reqs:
        assert r.t_done >= r.t_admit >= r.t_arrival - 1e-9


def test_request_larger_than_budget_is_rejected(env):
    cq, serving, pool, stream, m_max = env
    reqs = [pool.request(0, 0.0, m_max, 128, 10.0), pool.request(1, 0.0, 2000, 16, 10.0)]
    srv = serving.Server(1e12, slots=2, m_max=m_max, n_values=(16, 128))
    try:
        srv.budget = srv.workspace_bytes + reqs[1].bytes + 1
        stats = srv.run(reqs, realtime=False)
    finally:
        srv.close()
    assert reqs[0].status == cq.CQR2_ERR_OOM and reqs[1].status == 0
    assert stats["completed"] == 2 and stats["failed"] == 1
