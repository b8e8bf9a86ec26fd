"""The serving scheduler on the CPU, with a fake executor and a deterministic
clock: FIFO admission, the HBM budget, continuous admission while other
requests run, rejection of requests larger than the budget, and latency
percentiles."""
from __future__ import annotations

import pytest

from paper_1710_08471_gb300 import serving


class FakeClock:
    def __init__(self, tick=1e-4):
        self.t = 0.0
        self.tick = tick

    def __call__(self):
        self.t += self.tick
        return self.t

    def sleep(self, dt):
        self.t += dt


class FakeExecutor:
    """Completes a request `service(r)` seconds of fake time after submission."""

    def __init__(self, clock, slots=2, service=lambda r: r.m * r.n * 1e-7):
        self.clock = clock
        self._slots = slots
        self.service = service
        self.workspace_bytes = 1000
        self.concurrent = 0
        self.max_concurrent = 0

    @property
    def slots(self):
        return self._slots

    def sync(self):
        pass

    def submit(self, r, slot):
        self.concurrent += 1
        self.max_concurrent = max(self.max_concurrent, self.concurrent)
        return {"done": self.clock.t + self.service(r)}

    def poll(self, h):
        return self.clock.t >= h["done"]

    def finish(self, r, h):
        self.concurrent -= 1
        r.status = 0

    def close(self):
        pass


def req(i, t, m, n):
    return serving.Request(id=i, t_arrival=t, m=m, n=n, A_src=None, b_src=None)


def make(budget, slots=2, service=None):
    clk = FakeClock()
    ex = FakeExecutor(clk, slots=slots, **({"service": service} if service else {}))
    return serving.Server(budget, executor=ex, clock=clk, sleep=clk.sleep), ex


def test_fifo_and_completion():
    srv, ex = make(1e12, slots=3)
    reqs = [req(i, 0.001 * i, 1000 + 10 * i, 16) for i in range(20)]
    st = srv.run(reqs, realtime=True)
    assert st["completed"] == 20 and st["failed"] == 0
    assert srv.admitted == list(range(20))
    assert ex.max_concurrent <= 3
    for r in reqs:
        assert r.t_arrival <= r.t_admit + 1e-12 <= r.t_done + 1e-12


def test_budget_is_never_exceeded():
    big = req(0, 0.0, 5000, 64).bytes
    srv, ex = make(1000 + 2.5 * big, slots=8)
    reqs = [req(i, 0.0, 5000, 64) for i in range(10)]
    st = srv.run(reqs, realtime=False)
    assert st["completed"] == 10
    assert srv.peak_inflight_bytes <= 2.5 * big
    assert ex.max_concurrent == 2  # only two fit at a time


def test_continuous_admission_while_others_run():
    # one long request, then short ones arriving later: they start on the
    # free slot long before the long one finishes
    srv, ex = make(1e12, slots=2, service=lambda r: 1.0 if r.id == 0 else 0.01)
    reqs = [req(0, 0.0, 100, 8)] + [req(i, 0.05 * i, 100, 8) for i in range(1, 6)]
    srv.run(reqs, realtime=True)
    long_done = reqs[0].t_done
    assert all(r.t_done < long_done for r in reqs[1:])
    assert all(r.t_admit - r.t_arrival < 0.02 for r in reqs[1:])


def test_oversized_request_rejected_others_served():
    small = req(1, 0.0, 1000, 16)
    huge = req(0, 0.0, 10 ** 7, 256)
    srv, ex = make(1000 + 10 * small.bytes, slots=2)
    st = srv.run([huge, small], realtime=False)
    assert huge.status == serving.N.CQR2_ERR_OOM and small.status == 0
    assert st["completed"] == 2 and st["failed"] == 1


def test_percentile():
    v = list(range(101))
    assert serving.percentile(v, 50) == 50
    assert serving.percentile(v, 99) == 99
    assert serving.percentile([3.0], 99) == 3.0
    assert serving.percentile([], 50) != serving.percentile([], 50)  # nan


class FakeGroupExecutor(FakeExecutor):
    """FakeExecutor that also runs groups of small requests (n <= 64 and
    m n^2 <= limit) as one unit of work taking the longest member's time."""

    def __init__(self, clock, slots=2, group_max=4, limit=10 ** 7, **kw):
        super().__init__(clock, slots=slots, **kw)
        self.group_max = group_max
        self.limit = limit
        self.groups = []

    def groupable(self, m, n):
        return self.group_max > 1 and n <= 64 and m * n * n <= self.limit

    def submit_group(self, reqs, slot):
        assert all(self.groupable(r.m, r.n) for r in reqs) and len(reqs) <= self.group_max
        self.groups.append([r.id for r in reqs])
        self.concurrent += 1
        self.max_concurrent = max(self.max_concurrent, self.concurrent)
        return {"done": self.clock.t + max(self.service(r) for r in reqs)}

    def finish_group(self, reqs, h):
        self.concurrent -= 1
        for r in reqs:
            r.status = 0


def make_grouped(budget, slots=1, group_max=4, limit=10 ** 7):
    clk = FakeClock()
    ex = FakeGroupExecutor(clk, slots=slots, group_max=group_max, limit=limit)
    return serving.Server(budget, executor=ex, clock=clk, sleep=clk.sleep), ex


def test_small_requests_grouped_behind_a_small_head():
    # queue: small, large, small, small, small, small (all at t = 0), one slot,
    # groups of at most 4: the head takes the next three small ones with it;
    # the large one runs alone next; the last small one after that
    shapes = [(1000, 16), (100000, 128), (2000, 32), (3000, 16), (1500, 64), (1200, 8)]
    reqs = [req(i, 0.0, m, n) for i, (m, n) in enumerate(shapes)]
    srv, ex = make_grouped(1e12, slots=1, group_max=4)
    st = srv.run(reqs, realtime=False)
    assert st["completed"] == 6 and st["failed"] == 0
    assert ex.groups == [[0, 2, 3, 4], [5]]
    assert srv.admitted == [0, 2, 3, 4, 1, 5]
    assert st["group_launches"] == 2 and st["grouped_requests"] == 5
    # a group completes together
    assert len({reqs[i].t_done for i in (0, 2, 3, 4)}) == 1


def test_large_head_runs_alone_and_limit_routes_by_shape():
    # m n^2 above the limit is not grouped even with n <= 64
    reqs = [req(0, 0.0, 10 ** 6, 64), req(1, 0.0, 1000, 16), req(2, 0.0, 1000, 16)]
    srv, ex = make_grouped(1e12, slots=1, group_max=8, limit=10 ** 7)
    srv.run(reqs, realtime=False)
    assert ex.groups == [[1, 2]]
    assert srv.admitted == [0, 1, 2]


def test_group_respects_budget():
    r0 = req(0, 0.0, 1000, 16)
    budget = 1000 + 2.5 * r0.bytes  # room for two at a time
    reqs = [req(i, 0.0, 1000, 16) for i in range(5)]
    srv, ex = make_grouped(budget, slots=2, group_max=8)
    st = srv.run(reqs, realtime=False)
    assert st["completed"] == 5
    assert all(len(g) <= 2 for g in ex.groups)
    assert srv.peak_inflight_bytes <= 2.5 * r0.bytes
    assert sorted(i for g in ex.groups for i in g) == list(range(5))


def test_grouping_off_with_group_max_one():
    reqs = [req(i, 0.0, 1000, 16) for i in range(4)]
    srv, ex = make_grouped(1e12, slots=2, group_max=1)
    st = srv.run(reqs, realtime=False)
    assert ex.groups == [] and st["group_launches"] == 0 and st["completed"] == 4
