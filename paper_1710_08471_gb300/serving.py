"""Continuous-batching least-squares server over the CholeskyQR2 C ABI.

Requests (m x n least-squares solves, x = R^-1 Q^T b through CholeskyQR2)
arrive over time. The server:

* queues arrivals in order;
* admits the head of the queue when a slot (a CUDA stream with its own
  plans) is free and the request's device memory -- A, Q, R, b, x -- fits in
  the HBM budget next to what is already in flight;
* enqueues the request's copy-in and cqr2_lstsq_rows on the slot's stream, so
  requests that arrive while others run overlap on the device, and keeps A,
  Q and R on the device until the request completes;
* batches small requests: when the head of the queue is small (n <= 64 and
  m n^2 <= group_work_limit), the slot takes it together with the other
  small requests waiting in the queue (up to group_max, within the budget)
  and runs them as one launch of the persistent grouped kernel, least-squares
  tail included (cqr2_batch_factor with right-hand sides);
* polls completion events, frees the memory, and admits more work.

Plans are created per (slot, n) for the largest m the server accepts and are
reused for every request of that n (cqr2_lstsq_rows takes the request's m).
Whether a request runs grouped depends on its shape alone, so its result is
the same bit for bit whatever else is in flight. Every computation runs in
libcqr2's kernels; this module only schedules.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import time

import paper_1710_08471_gb300 as cq
from . import _native as N


@dataclasses.dataclass
class Request:
    id: int
    t_arrival: float          # seconds since the start of the run
    m: int
    n: int
    A_src: object             # device tensor (m x n, column-major) to copy in
    b_src: object             # device vector (m)
    # filled by the server
    t_admit: float = math.nan
    t_done: float = math.nan
    status: int = -1
    x: object = None
    R: object = None
    Q: object = None
    slot: int = -1

    @property
    def bytes(self) -> int:
        return 8 * (2 * self.m * self.n + self.n * self.n + self.m + self.n)


GROUP_MAX_N = 64  # the grouped kernel's largest n


class CudaExecutor:
    """Runs requests on CUDA stream slots through cqr2_lstsq_rows, one plan
    per (slot, n) sized for the largest m, and groups of small requests
    through one grouped launch per slot (a cqr2 batch on the slot's stream).
    group_max = 1 turns grouping off."""

    def __init__(self, slots: int, precision: int, m_max: int, n_values, keep_outputs: bool = False,
                 group_max: int = 64, group_work_limit: int = 1 << 24):
        import torch

        self.torch = torch
        self.precision = precision
        self.m_max = int(m_max)
        self.keep = keep_outputs
        self.group_max = int(group_max)
        self.group_work_limit = int(group_work_limit)
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.plans = [dict() for _ in range(slots)]
        self.batches = []
        self.workspace_bytes = 0
        for s in range(slots):
            for n in n_values:
                if not self.groupable(self.m_max, n):
                    self._plan(s, n)
        if self.group_max > 1:
            # the batch routes by the same rule (n <= 64, m n^2 <= the limit)
            self.batches = [cq.Batch(self.group_max, small_work_limit=self.group_work_limit, streams=1,
                                     stream=self.streams[s]) for s in range(slots)]

    def groupable(self, m: int, n: int) -> bool:
        return self.group_max > 1 and n <= GROUP_MAX_N and m * n * n <= self.group_work_limit

    @property
    def slots(self) -> int:
        return len(self.streams)

    def _plan(self, slot: int, n: int):
        p = self.plans[slot].get(n)
        if p is None:
            prec = self.precision if n <= 1024 else cq.CQR2_FP64
            p = cq.Plan(self.m_max, n, precision=prec, stream=self.streams[slot])
            self.plans[slot][n] = p
            self.workspace_bytes += p.workspace_bytes
        return p

    def sync(self) -> None:
        self.torch.cuda.synchronize()

    def submit(self, r: Request, slot: int):
        """Enqueue the copy-in and the solve on the slot's stream; returns a
        handle that keeps the request's buffers alive."""
        torch = self.torch
        s = self.streams[slot]
        with torch.cuda.stream(s):
            A = cq.empty_colmajor(r.m, r.n, device="cuda")
            A.copy_(r.A_src)
            b = r.b_src.clone()
            Q = cq.empty_colmajor(r.m, r.n, device="cuda")
            R = cq.empty_colmajor(r.n, r.n, device="cuda")
            x = torch.empty(r.n, dtype=torch.float64, device="cuda")
            plan = self._plan(slot, r.n)
            cq.cqr2_lstsq_rows(plan.handle, r.m, r.n, A, b, x, Q, R, sync=False)
            ev = torch.cuda.Event()
            ev.record(s)
        return (ev, (A, b, Q, R, x), plan)

    def submit_group(self, reqs: list, slot: int):
        """Enqueue the copy-in of every request of the group and one grouped
        launch (factorization and least-squares tail) on the slot's stream."""
        torch = self.torch
        s = self.streams[slot]
        bufs = []
        with torch.cuda.stream(s):
            for r in reqs:
                A = cq.empty_colmajor(r.m, r.n, device="cuda")
                A.copy_(r.A_src)
                b = r.b_src.clone()
                Q = cq.empty_colmajor(r.m, r.n, device="cuda")
                R = cq.empty_colmajor(r.n, r.n, device="cuda")
                x = torch.empty(r.n, dtype=torch.float64, device="cuda")
                bufs.append((A, Q, R, b, x))
            batch = self.batches[slot]
            batch.factor(bufs, sync=False)
            ev = torch.cuda.Event()
            ev.record(s)
        return (ev, bufs, batch)

    def poll(self, handle) -> bool:
        return handle[0].query()

    def finish(self, r: Request, handle) -> None:
        ev, (A, b, Q, R, x), plan = handle
        info = N.Info()
        # status word of the plan's last call: the slot's stream has finished it
        N.load().cqr2_plan_info(plan.handle, info)
        r.status = info.status
        r.x = x
        if self.keep:
            r.Q, r.R = Q, R

    def finish_group(self, reqs: list, handle) -> None:
        ev, bufs, batch = handle
        infos = batch.info()  # the slot's stream has finished: no wait
        for r, (A, Q, R, b, x), inf in zip(reqs, bufs, infos):
            r.status = inf.status
            r.x = x
            if self.keep:
                r.Q, r.R = Q, R

    def close(self) -> None:
        for d in self.plans:
            for p in d.values():
                p.close()
        self.plans = []
        for b in self.batches:
            b.close()
        self.batches = []


class Server:
    """Continuous-batching scheduler: FIFO queue, admission against an HBM
    budget into free slots, completion by polling. The executor runs the
    requests (CudaExecutor by default); clock and sleep can be replaced for
    deterministic tests."""

    def __init__(self, budget_bytes: float, slots: int = 8, precision: int = cq.CQR2_FP64, m_max: int = 262144,
                 n_values=(16, 32, 64, 128, 256), keep_outputs: bool = False, executor=None, clock=None,
                 sleep=None, group_max: int = 64, group_work_limit: int = 1 << 24):
        self.exec = executor if executor is not None else CudaExecutor(slots, precision, m_max, n_values,
                                                                       keep_outputs, group_max, group_work_limit)
        self.clock = clock or time.perf_counter
        self.sleep = sleep or time.sleep
        self.budget = float(budget_bytes)
        self.busy = [None] * self.exec.slots  # (requests, handle, grouped)
        self.inflight_bytes = 0
        self.peak_inflight_bytes = 0
        self.admitted: list[int] = []
        self.group_launches = 0
        self.grouped_requests = 0

    @property
    def workspace_bytes(self) -> int:
        return self.exec.workspace_bytes

    def _groupable(self, r: Request) -> bool:
        g = getattr(self.exec, "groupable", None)
        return g is not None and g(r.m, r.n)

    def _submit(self, reqs: list, slot: int, t0: float):
        grouped = self._groupable(reqs[0])
        handle = self.exec.submit_group(reqs, slot) if grouped else self.exec.submit(reqs[0], slot)
        t = self.clock() - t0
        for r in reqs:
            r.t_admit = t
            r.slot = slot
            self.inflight_bytes += r.bytes
            self.admitted.append(r.id)
        self.busy[slot] = (reqs, handle, grouped)
        self.peak_inflight_bytes = max(self.peak_inflight_bytes, self.inflight_bytes)
        if grouped:
            self.group_launches += 1
            self.grouped_requests += len(reqs)

    def _retire(self, slot: int, t0: float):
        reqs, handle, grouped = self.busy[slot]
        t = self.clock() - t0
        for r in reqs:
            r.t_done = t
        if grouped:
            self.exec.finish_group(reqs, handle)
        else:
            self.exec.finish(reqs[0], handle)
        self.busy[slot] = None
        for r in reqs:
            self.inflight_bytes -= r.bytes

    def _take(self, queue, limit: float):
        """The head of the queue and, if it is small, the other small requests
        waiting behind it (in queue order, up to the group size, within the
        budget)."""
        head = queue.popleft()
        reqs = [head]
        if not self._groupable(head):
            return reqs
        room = limit - self.inflight_bytes - head.bytes
        gmax = self.exec.group_max
        keep = collections.deque()
        while queue and len(reqs) < gmax:
            r = queue.popleft()
            if self._groupable(r) and r.bytes <= room:
                reqs.append(r)
                room -= r.bytes
            else:
                keep.append(r)
        keep.extend(queue)
        queue.clear()
        queue.extend(keep)
        return reqs

    def run(self, requests: list[Request], realtime: bool = True) -> dict:
        """Serve `requests`. With realtime, a request is not admitted before
        its arrival time; otherwise all are available at time 0."""
        queue = collections.deque()
        pending = collections.deque(sorted(requests, key=lambda r: r.t_arrival))
        done = []
        self.exec.sync()
        t0 = self.clock()
        slots = len(self.busy)
        limit = self.budget - self.workspace_bytes
        while pending or queue or any(b is not None for b in self.busy):
            now = self.clock() - t0
            while pending and (not realtime or pending[0].t_arrival <= now):
                queue.append(pending.popleft())
            for s in range(slots):
                if self.busy[s] is not None and self.exec.poll(self.busy[s][1]):
                    done.extend(self.busy[s][0])
                    self._retire(s, t0)
            while queue and queue[0].bytes > limit:
                # larger than the whole budget: it can never be admitted
                r = queue.popleft()
                r.status = N.CQR2_ERR_OOM
                r.t_done = self.clock() - t0
                done.append(r)
            for s in range(slots):
                if not queue:
                    break
                if self.busy[s] is None and self.inflight_bytes + queue[0].bytes <= limit:
                    self._submit(self._take(queue, limit), s, t0)
            if not queue and pending and realtime:
                # idle until the next arrival
                wait = pending[0].t_arrival - (self.clock() - t0)
                if wait > 0 and all(b is None for b in self.busy):
                    self.sleep(min(wait, 0.001))
        t_end = self.clock() - t0
        lat = sorted((r.t_done - r.t_arrival) for r in done) if realtime else sorted(r.t_done for r in done)
        return {
            "completed": len(done),
            "failed": sum(1 for r in done if r.status != 0),
            "seconds": t_end,
            "qr_per_s": len(done) / t_end if t_end > 0 else float("nan"),
            "p50_ms": 1e3 * percentile(lat, 50),
            "p99_ms": 1e3 * percentile(lat, 99),
            "mean_ms": 1e3 * sum(lat) / max(1, len(lat)),
            "workspace_bytes": self.workspace_bytes,
            "peak_inflight_gb": self.peak_inflight_bytes / 1e9,
            "group_launches": self.group_launches,
            "grouped_requests": self.grouped_requests,
        }

    def close(self):
        self.exec.close()


def percentile(sorted_vals, q: float) -> float:
    if not sorted_vals:
        return float("nan")
    k = (len(sorted_vals) - 1) * q / 100.0
    f = math.floor(k)
    c = min(f + 1, len(sorted_vals) - 1)
    return sorted_vals[f] + (sorted_vals[c] - sorted_vals[f]) * (k - f)


def run_workload(count: int, rate: float, seed: int = 100, precision: int = cq.CQR2_FP64, slots: int = 8,
                 budget: float = 64e9, m_max: int = 262144, n_values=(16, 32, 64, 128, 256),
                 realtime: bool = True, pool: "InputPool | None" = None, group_max: int = 64,
                 group_work_limit: int = 1 << 24) -> dict:
    """Serve a seeded least-squares request stream (synth.request_stream:
    Poisson arrivals at `rate`, m uniform in [1024, m_max], n uniform over
    n_values, kappa log-uniform in [1, 1e5]) and return latency/throughput."""
    import synth

    stream = synth.request_stream(count, seed=seed, rate=rate, m_lo=1024, m_hi=m_max, n_choices=tuple(n_values))
    pool = pool or InputPool(m_max, n_values, seed=seed)
    reqs = [pool.request(r["id"], r["t"], r["m"], r["n"], r["kappa"]) for r in stream]
    srv = Server(budget, slots=slots, precision=precision, m_max=m_max, n_values=n_values, group_max=group_max,
                 group_work_limit=group_work_limit)
    try:
        stats = srv.run(reqs, realtime=realtime)
    finally:
        srv.close()
    done = [r for r in reqs if r.status == 0]
    flops = sum(4.0 * r.m * r.n * r.n + 5.0 * r.n ** 3 / 3.0 + 2.0 * r.m * r.n for r in done)
    stats["tflops"] = flops / stats["seconds"] / 1e12 if stats["seconds"] > 0 else float("nan")
    stats.update({"requests": count, "rate_per_s": rate, "slots": slots, "precision": precision,
                  "budget_gb": budget / 1e9, "m_max": m_max, "n_values": list(n_values), "group_max": group_max,
                  "group_work_limit": group_work_limit})
    return stats


def main(argv=None) -> None:
    import argparse
    import json

    ap = argparse.ArgumentParser(description="least-squares serving benchmark over CholeskyQR2")
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--budget-gb", type=float, default=64.0)
    ap.add_argument("--precision", type=int, default=cq.CQR2_OZAKI_BF16)
    ap.add_argument("--seed", type=int, default=100)
    ap.add_argument("--group-max", type=int, default=64, help="small requests per grouped launch (1 = no grouping)")
    ap.add_argument("--group-work-limit", type=int, default=1 << 24, help="grouped when n <= 64 and m n^2 <= this")
    args = ap.parse_args(argv)
    pool = InputPool(262144, (16, 32, 64, 128, 256), seed=args.seed)
    # warm-up (not reported): first device allocations and kernel loads
    run_workload(min(300, args.requests), args.rate, args.seed + 1, args.precision, args.slots, args.budget_gb * 1e9,
                 pool=pool)
    out = {"continuous": run_workload(args.requests, args.rate, args.seed, args.precision, args.slots,
                                      args.budget_gb * 1e9, pool=pool, group_max=args.group_max,
                                      group_work_limit=args.group_work_limit),
           "one_at_a_time": run_workload(args.requests, args.rate, args.seed, args.precision, 1,
                                         args.budget_gb * 1e9, pool=pool, group_max=1)}
    print(json.dumps(out))


def kappa_grid(lo: float = 1.0, hi: float = 1e5, per_decade: int = 4) -> list[float]:
    """Condition numbers log-spaced from lo to hi, per_decade per decade."""
    k = max(1, round(per_decade * math.log10(hi / lo)))
    return [lo * (hi / lo) ** (i / k) for i in range(k + 1)]


class InputPool:
    """Device-resident synthetic inputs for request streams: for every n and
    every condition number of a log-spaced grid (by default 1 .. 1e5 at four
    per decade, 21 values), one m_max x n matrix A = G diag(sigma) V built by
    the seeded generator (synth.make_matrix) on the host and copied to the
    device once; a request of m rows uses the first m rows. A request's kappa,
    drawn log-uniform per request, is served by the nearest grid value, within
    a factor 10^(1/8) ~ 1.33 at the default grid (the inputs cannot be formed
    per request without putting an m x n x n product of the generator on the
    GPU next to the work being timed)."""

    def __init__(self, m_max: int, n_values, kappas=None, seed: int = 100):
        import numpy as np
        import torch

        import synth

        self.kappas = list(kappas) if kappas is not None else kappa_grid()
        self.A = {}
        for n in n_values:
            for i, k in enumerate(self.kappas):
                h = synth.make_matrix(m_max, n, k, seed=seed, mid=1000 * n + i)
                t = torch.from_numpy(np.ascontiguousarray(h.T)).cuda().t()
                self.A[(n, i)] = t
        self.b = torch.from_numpy(synth.make_rhs(m_max, seed=seed)).cuda()

    def bucket(self, kappa: float) -> int:
        lk = math.log10(max(kappa, 1.0))
        return min(range(len(self.kappas)), key=lambda i: abs(math.log10(self.kappas[i]) - lk))

    def kappa_of(self, kappa: float) -> float:
        """The grid condition number a request drawn with `kappa` is served with."""
        return self.kappas[self.bucket(kappa)]

    def request(self, rid: int, t: float, m: int, n: int, kappa: float) -> Request:
        i = self.bucket(kappa)
        return Request(id=rid, t_arrival=t, m=m, n=n, A_src=self.A[(n, i)][:m], b_src=self.b[:m])


if __name__ == "__main__":
    main()
