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
