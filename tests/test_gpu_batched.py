"""Variable-m plans, CUDA-graph replay, grouped batches and the autotuner,
each checked against the CPU FP64 oracle with the FP64 tolerances of
test_gpu_parity (orthogonality <= 1e-12, residual <= 1e-13, R relative
<= 1e-12 kappa) and, where a result must not depend on how it was scheduled,
bit for bit."""
from __future__ import annotations

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


def check(A, Q, R, kappa, scale=1.0):
    Qo, Ro = oracle.cqr2(A)
    k = kappa or 2.0
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R) > 0)
    assert oracle.orthogonality(Q) <= scale * max(1e-12, 10 * oracle.orthogonality(Qo))
    assert oracle.residual(A, Q, R) <= scale * max(1e-13, 10 * oracle.residual(A, Qo, Ro))
    assert oracle.rel_error(R, Ro) <= scale * 1e-12 * k


@pytest.mark.parametrize("prec,scale", [(0, 1.0), (1, 10.0)])
def test_factor_rows_uneven_m(cq, prec, scale):
    n = 64
    with cq.Plan(6000, n, precision=prec) as p:
        for m, kappa in [(6000, 1e4), (64, 10.0), (777, 1e3), (3001, None), (6000, 1e2)]:
            A = synth.make_matrix(m, n, kappa, seed=m)
            Q, R, info = p.factor_rows(to_dev(A))
            assert info.status == 0
            check(A, to_host(Q), to_host(R), kappa, scale)


@pytest.mark.parametrize("prec,scale", [(0, 1.0), (1, 10.0)])
@pytest.mark.parametrize("n", [16, 64])
def test_factor_rows_more_ranges_than_full_size(cq, prec, scale, n):
    # Row counts just above a multiple of the CTA target round to shorter (and
    # so more) Gram row ranges than the plan's full size does; the partial
    # buffers must hold them (n = 16: 38900 rows make 304 ranges against 293
    # at 2^18 rows on the split-precision path).
    with cq.Plan(1 << 18, n, precision=prec) as p:
        for m in (38900, 38913, 77801, 155000, 155701, (1 << 18) - 1):
            A = synth.make_matrix(m, n, 1e3, seed=m)
            Q, R, info = p.factor_rows(to_dev(A))
            assert info.status == 0
            check(A, to_host(Q), to_host(R), 1e3, scale)


def test_lstsq_rows(cq):
    n = 32
    with cq.Plan(5000, n) as p:
        for m in (5000, 100, 2047):
            A = synth.make_matrix(m, n, 1e3, seed=m + 1)
            b = synth.make_rhs(m, seed=m)
            x, info = p.lstsq_rows(to_dev(A), to_dev(b))
            xo = oracle.lstsq(A, b)
            assert np.linalg.norm(to_host(x) - xo) <= 1e-12 * 1e3 * np.linalg.norm(xo)


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_matches_direct(cq, prec):
    import torch

    m, n = 8000, 96
    A1 = to_dev(synth.make_matrix(m, n, 1e5, seed=1))
    A2 = to_dev(synth.make_matrix(m, n, 1e3, seed=2))
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with cq.Plan(m, n, precision=prec) as p:
        Qd, Rd, _ = p.factor(A1)
        Qd2, Rd2, _ = p.factor(A2)
    with cq.Plan(m, n, precision=prec, stream=s, graph=True) as p:
        Q = cq.empty_colmajor(m, n, device="cuda")
        R = cq.empty_colmajor(n, n, device="cuda")
        counts = []
        for _ in range(3):  # capture, then replay twice
            l0 = cq.cqr2_launch_count()
            p.factor(A1, Q, R)
            counts.append(cq.cqr2_launch_count() - l0)
            torch.cuda.synchronize()
            assert bool((Q == Qd).all()) and bool((R == Rd).all())
        assert counts[0] > 10 and counts[1] == counts[0] == counts[2]  # a replay counts the graph's kernels
        p.factor(A2, Q, R)  # new arguments: a new capture
        torch.cuda.synchronize()
        assert bool((Q == Qd2).all()) and bool((R == Rd2).all())


def _problems(cq, shapes, seed0=0):
    mats, probs = [], []
    for i, (m, n, kappa) in enumerate(shapes):
        A = synth.make_matrix(m, n, kappa, seed=seed0 + i)
        mats.append(A)
        probs.append((to_dev(A), cq.empty_colmajor(m, n, device="cuda"), cq.empty_colmajor(n, n, device="cuda")))
    return mats, probs


SMALL = [(64, 1, None), (100, 8, 10.0), (4096, 64, None), (777, 33, 1e3), (2000, 64, 1e5), (65, 64, 1e2),
         (31, 17, None), (5000, 48, 1e4)]
MIXED = SMALL + [(20000, 128, 1e6), (3001, 200, 1e3), (30000, 64, 1e4), (1500, 300, 1e2)]


def test_batch_grouped_kernel(cq):
    mats, probs = _problems(cq, SMALL * 4, seed0=10)
    with cq.Batch(len(probs), small_work_limit=1 << 40) as b:
        infos = b.factor(probs)
    for A, (_, Q, R), inf, (m, n, kappa) in zip(mats, probs, infos, SMALL * 4):
        assert inf.status == 0
        check(A, to_host(Q), to_host(R), kappa)


@pytest.mark.parametrize("prec,scale", [(0, 1.0), (1, 10.0)])
def test_batch_mixed_routing(cq, prec, scale):
    mats, probs = _problems(cq, MIXED, seed0=50)
    with cq.Batch(len(probs), precision=prec) as b:
        infos = b.factor(probs)
    for A, (_, Q, R), inf, (m, n, kappa) in zip(mats, probs, infos, MIXED):
        assert inf.status == 0
        # small problems run in the FP64 grouped kernel whatever the precision
        check(A, to_host(Q), to_host(R), kappa, scale)


def test_batch_breakdown_is_per_problem(cq):
    shapes = [(500, 16, None), (600, 16, None), (700, 128, None), (800, 128, None)]
    mats, probs = _problems(cq, shapes, seed0=90)
    bad = [1, 3]
    for i in bad:
        mats[i][:, 5] = 0.0
        probs[i][0].copy_(to_dev(mats[i]))
    with cq.Batch(len(probs)) as b:
        infos = b.factor(probs)
    for i, inf in enumerate(infos):
        if i in bad:
            assert inf.status == cq.CQR2_ERR_NOT_SPD and inf.failed_pass == 1 and inf.failed_pivot == 5
        else:
            assert inf.status == 0
            check(mats[i], to_host(probs[i][1]), to_host(probs[i][2]), None)


def test_batch_result_same_alone_and_in_mix(cq):
    """A problem's result does not depend on what else is in its batch."""
    mats, probs = _problems(cq, MIXED, seed0=200)
    with cq.Batch(len(probs)) as b:
        b.factor(probs)
        mixed = [(to_host(Q), to_host(R)) for _, Q, R in probs]
        for i, pr in enumerate(probs):
            b.factor([pr])
            Q, R = to_host(pr[1]), to_host(pr[2])
            assert np.array_equal(Q, mixed[i][0]) and np.array_equal(R, mixed[i][1]), i


def _lstsq_problems(cq, shapes, seed0=0):
    import torch

    mats, rhs, probs = [], [], []
    for i, (m, n, kappa) in enumerate(shapes):
        A = synth.make_matrix(m, n, kappa, seed=seed0 + i)
        b = synth.make_rhs(m, seed=seed0 + 1000 + i)
        mats.append(A)
        rhs.append(b)
        probs.append((to_dev(A), cq.empty_colmajor(m, n, device="cuda"), cq.empty_colmajor(n, n, device="cuda"),
                      to_dev(b), torch.empty(n, dtype=torch.float64, device="cuda")))
    return mats, rhs, probs


def check_x(A, b, x, kappa, scale=1.0):
    xo = oracle.lstsq(A, b)
    k = kappa or 2.0
    assert np.linalg.norm(x - xo) <= scale * 1e-12 * k * np.linalg.norm(xo)


@pytest.mark.parametrize("limit", [1 << 40, None])
def test_batch_lstsq(cq, limit):
    """Least squares through the batch: the grouped kernel's tail (c = Q^T b
    while the final Q is formed, back substitution in one warp) and, with the
    default routing, the planned problems' cqr2_lstsq_rows."""
    shapes = MIXED if limit is None else SMALL * 2
    mats, rhs, probs = _lstsq_problems(cq, shapes, seed0=400)
    kw = {} if limit is None else {"small_work_limit": limit}
    with cq.Batch(len(probs), **kw) as b:
        infos = b.factor(probs)
    for A, bv, pr, inf, (m, n, kappa) in zip(mats, rhs, probs, infos, shapes):
        assert inf.status == 0
        check(A, to_host(pr[1]), to_host(pr[2]), kappa)
        check_x(A, bv, to_host(pr[4]), kappa)


def test_batch_lstsq_ragged_and_extremes(cq):
    # n = 1, n = 64 with m = n, row counts off the 32-row panel, and a
    # right-hand side in the range of A (zero residual): x = the generating
    # coefficients
    shapes = [(1, 1, None), (64, 64, 10.0), (65, 63, 1e2), (33, 32, None), (4097, 64, 1e3), (31, 31, 1e1)]
    mats, rhs, probs = _lstsq_problems(cq, shapes, seed0=500)
    xs = []
    for i, (A, (m, n, _)) in enumerate(zip(mats, shapes)):
        xt = np.random.default_rng(i).standard_normal(n)
        rhs[i] = A @ xt
        xs.append(xt)
        probs[i][3].copy_(to_dev(rhs[i]))
    with cq.Batch(len(probs), small_work_limit=1 << 40) as b:
        infos = b.factor(probs)
    for A, bv, pr, inf, xt, (m, n, kappa) in zip(mats, rhs, probs, infos, xs, shapes):
        assert inf.status == 0
        x = to_host(pr[4])
        check_x(A, bv, x, kappa)
        assert np.linalg.norm(x - xt) <= 1e-12 * (kappa or 2.0) * np.linalg.norm(xt)


def test_batch_async_info_and_reuse(cq):
    """factor(sync=False) then info(): the same outcomes as the synchronous
    form; a second call on the batch waits for the first."""
    shapes = [(500, 16, None), (600, 16, None), (3000, 128, 1e3), (800, 64, 1e2)]
    mats, rhs, probs = _lstsq_problems(cq, shapes, seed0=600)
    mats[1][:, 3] = 0.0
    probs[1][0].copy_(to_dev(mats[1]))
    with cq.Batch(len(probs)) as b:
        assert b.factor(probs, sync=False) is None
        infos = b.info()
        assert [i.status for i in infos] == [0, cq.CQR2_ERR_NOT_SPD, 0, 0]
        assert infos[1].failed_pass == 1 and infos[1].failed_pivot == 3
        x0 = [to_host(p[4]) for p in probs]
        b.factor(probs[:3], sync=False)
        b.factor(probs[:3], sync=False)  # reuses the descriptors after the first finished
        infos = b.info()
        assert len(infos) == 3 and infos[1].status == cq.CQR2_ERR_NOT_SPD
    for i in (0, 2):
        assert np.array_equal(to_host(probs[i][4]), x0[i])
        check_x(mats[i], rhs[i], x0[i], shapes[i][2])


def test_batch_lstsq_same_alone_and_in_mix(cq):
    mats, rhs, probs = _lstsq_problems(cq, MIXED, seed0=700)
    with cq.Batch(len(probs)) as b:
        b.factor(probs)
        mixed = [to_host(p[4]) for p in probs]
        for i, pr in enumerate(probs):
            b.factor([pr])
            assert np.array_equal(to_host(pr[4]), mixed[i]), i


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_graph_replay(cq, prec):
    """cfg.graph: the first call runs eagerly, the repeat is captured, later
    repeats replay the graph. Every call gives the eager batch's results bit
    for bit, a replay recomputes from the inputs' current contents (A scaled
    by 2 gives the same Q and 2 R exactly), and a new list runs eagerly."""
    import torch

    shapes = MIXED[:6] + MIXED[-4:]
    mats, rhs, probs = _lstsq_problems(cq, shapes, seed0=800)
    with cq.Batch(len(probs), precision=prec) as b:
        assert all(i.status == 0 for i in b.factor(probs))
        ref = [(to_host(p[1]), to_host(p[2]), to_host(p[4])) for p in probs]
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with cq.Batch(len(probs), precision=prec, stream=s, graph=True) as b:
        for call in range(4):
            for p in probs:
                p[1].zero_(), p[2].zero_(), p[4].zero_()
            torch.cuda.synchronize()
            infos = b.factor(probs)
            assert all(i.status == 0 for i in infos), call
            for i, p in enumerate(probs):
                assert np.array_equal(to_host(p[1]), ref[i][0]), (call, i)
                assert np.array_equal(to_host(p[2]), ref[i][1]), (call, i)
                assert np.array_equal(to_host(p[4]), ref[i][2]), (call, i)
        for p in probs:
            p[0].mul_(2.0)
        torch.cuda.synchronize()
        l0 = cq.cqr2_launch_count()
        b.factor(probs)  # replay on the new contents
        assert cq.cqr2_launch_count() - l0 >= 1 + 4 * 10  # the grouped launch and the planned problems' kernels
        for i, p in enumerate(probs):
            assert np.array_equal(to_host(p[1]), ref[i][0]), i
            assert np.array_equal(to_host(p[2]), 2.0 * ref[i][1]), i
        for p in probs:
            p[0].mul_(0.5)
        torch.cuda.synchronize()
        # a different list: eager again, still correct
        sub = probs[::2]
        infos = b.factor(sub)
        for (A, bv, pr, (m, n, kappa)), inf in zip(list(zip(mats, rhs, probs, shapes))[::2], infos):
            assert inf.status == 0
            check(A, to_host(pr[1]), to_host(pr[2]), kappa, 1.0 if prec == 0 else 10.0)
            check_x(A, bv, to_host(pr[4]), kappa, 1.0 if prec == 0 else 10.0)


def test_autotune_records_table(cq):
    res = cq.cqr2_autotune(50000, 128)
    assert res["candidates"] >= 4 and res["gram_ctas"] in (1, 2, 4, 8) and res["ms"] > 0
    table = cq.cqr2_tune_table()
    assert "128:15:0" in table and "small_work_limit=" in table
    # plans accept the tuned knobs
    with cq.Plan(50000, 128, fused=True) as p:
        p.set_gram_ctas(res["gram_ctas"])
        p.set_fused(res["fused"])
        A = synth.make_matrix(50000, 128, 1e4, seed=3)
        Q, R, _ = p.factor(to_dev(A))
    check(A, to_host(Q), to_host(R), 1e4)


def test_autotune_batch_routing_limit(cq):
    """The batch routing autotuner measures the grouped kernel against plans
    and sets the limit later batches use (restored afterwards)."""
    try:
        lim = cq.cqr2_autotune_batch(32, 152)
        assert lim >= 0 and lim % (32 * 32) == 0
        assert f"small_work_limit={lim}" in cq.cqr2_tune_table()
        # a batch created now routes by the tuned limit, and still factors correctly
        shapes = [(max(64, lim // (32 * 32)), 32, 1e3), (64, 32, 10.0), (4 * max(64, lim // (32 * 32)) + 1, 32, 1e2)]
        mats, probs = _problems(cq, shapes, seed0=900)
        with cq.Batch(len(probs)) as b:
            infos = b.factor(probs)
        for A, (_, Q, R), inf, (m, n, kappa) in zip(mats, probs, infos, shapes):
            assert inf.status == 0
            check(A, to_host(Q), to_host(R), kappa)
    finally:
        cq.cqr2_tune_set_small_limit(32768 * 64 * 64)
