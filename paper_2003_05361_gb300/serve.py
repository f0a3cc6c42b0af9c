"""Continuous-batching serving loop for RAS solves.

Requests (2D Poisson systems of different grid sides) arrive over time. The
loop admits an arrived request when its estimated device footprint fits the
HBM budget and enough subdomain slots are free, sets it up (host maps and GPU
factorisation, in worker threads so it overlaps the running steps), starts it
with ras_solve_begin, and advances every admitted system together with
ras_batch_step: one persistent launch per turn in which the subdomains of all
active systems run side by side. Finished systems retire immediately and their
slots and memory go to the next arrivals.

Everything numeric runs in the library's kernels; this module only schedules.
"""
from __future__ import annotations

import math
import statistics
import threading
import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import (RAS_ASYNC, RAS_ENOTSUP, RAS_FP32, RAS_LOCAL_BANDCHOL, ras_batch_step,
               ras_destroy, ras_get_info, ras_partition_regular2d, ras_setup, ras_solve_begin)


@dataclass
class Request:
    rid: int
    side: int
    arrival: float  # seconds after the stream starts
    seed: int       # right-hand-side seed


@dataclass
class Record:
    rid: int
    side: int
    n: int
    arrival: float
    admitted: float
    started: float
    finished: float
    status: int
    iterations: int
    relres: float
    device_bytes: int
    rejected: bool = False  # could never fit the slots or the budget (status RAS_ENOTSUP)

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


def request_stream(num: int, rate: float, seed: int = 5, side_min: int = 64,
                   side_max: int = 512, rhs_seed0: int = 1000):
    """Seeded open-loop stream: exponential inter-arrival gaps (a Poisson
    process of `rate` requests per second) and sides uniform in
    [side_min, side_max], both from SplitMix64(seed); request i solves with the
    right-hand side of seed rhs_seed0 + i."""
    import problems

    u = problems.uniform01(seed, 2 * num)
    gaps = -np.log1p(-u[:num]) / rate
    arrivals = np.cumsum(gaps)
    sides = side_min + np.floor(u[num:] * (side_max - side_min + 1)).astype(int)
    return [Request(i, int(sides[i]), float(arrivals[i]), rhs_seed0 + i) for i in range(num)]


@dataclass
class _Active:
    req: Request
    ctx: object
    b: object
    x: object
    n: int
    parts: int
    nbytes: int
    admitted: float
    started: float


@dataclass
class Server:
    """Serving configuration. step_limit: local updates per subdomain (async)
    or iterations (sync) per batched launch; max_parts: subdomain slots shared
    by the active systems; budget_bytes: HBM budget for active contexts
    (default 0.8 x free device memory). A request that needs more slots or
    bytes than these limits allow even alone is rejected on arrival (record
    status RAS_ENOTSUP), never queued."""

    mode: int = RAS_ASYNC
    prec: int = RAS_FP32
    kind: int = RAS_LOCAL_BANDCHOL
    overlap: int = 2
    block: int = 64
    tol: float = 1e-8
    step_limit: int = 20
    max_parts: int = 600
    budget_bytes: int = 0
    workers: int = 2
    keep_solutions: bool = False
    bytes_per_unknown: float = 1200.0  # initial estimate, raised by measurements
    records: list = field(default_factory=list)
    solutions: dict = field(default_factory=dict)

    def _estimate(self, side: int) -> int:
        return int(self.bytes_per_unknown * side * side) + 3 * 8 * side * side

    def _prepare(self, req: Request, stream, t0: float):
        import torch

        import problems

        A = problems.poisson2d(req.side)
        b = problems.rhs_uniform(A.n, req.seed)
        px = math.ceil(req.side / self.block)
        part = ras_partition_regular2d(req.side, req.side, px, px)
        with torch.cuda.stream(stream):
            ctx = ras_setup(A, part, px * px, self.overlap, self.kind, self.prec, 10, stream=stream)
            bd = torch.tensor(b, device="cuda")
            x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
            ras_solve_begin(ctx, bd, x, self.tol)
        nbytes = ras_get_info(ctx)["device_bytes"] + 3 * 8 * A.n
        return _Active(req, ctx, bd, x, A.n, px * px, nbytes, 0.0, time.perf_counter() - t0)

    # device-facing steps of the loop (the scheduler below only calls these)
    def _default_stream(self):
        import torch

        return torch.cuda.current_stream()

    def _free_device_bytes(self) -> int:
        import torch

        return torch.cuda.mem_get_info()[0]

    def _step(self, ctxs):
        return ras_batch_step(ctxs, self.mode, self.step_limit)

    def _release(self, a: _Active) -> None:
        ras_destroy(a.ctx)

    def _solution(self, a: _Active):
        return a.x.cpu().numpy()

    def run(self, requests, stream=None):
        """Serves `requests` (sorted by arrival) in real time; returns summary stats."""
        if stream is None:
            stream = self._default_stream()
        if self.budget_bytes <= 0:
            self.budget_bytes = int(0.8 * self._free_device_bytes())
        pending = deque(sorted(requests, key=lambda r: r.arrival))
        inflight = deque()  # futures of setups in progress
        active: list[_Active] = []
        used_bytes = 0
        used_parts = 0
        lock = threading.Lock()
        t0 = time.perf_counter()
        pool = ThreadPoolExecutor(self.workers)
        steps = 0
        try:
            while pending or inflight or active:
                now = time.perf_counter() - t0
                while pending and pending[0].arrival <= now:
                    r = pending[0]
                    px = math.ceil(r.side / self.block)
                    est = self._estimate(r.side)
                    if px * px > self.max_parts or est > self.budget_bytes:
                        # can never fit, even alone: reject it rather than
                        # block the queue behind it
                        pending.popleft()
                        self.records.append(Record(r.rid, r.side, r.side * r.side, r.arrival,
                                                   now, now, now, RAS_ENOTSUP, 0, float("nan"),
                                                   est, rejected=True))
                        continue
                    if used_parts + px * px > self.max_parts or used_bytes + est > self.budget_bytes:
                        break
                    pending.popleft()
                    used_parts += px * px
                    used_bytes += est
                    fut = pool.submit(self._prepare, r, stream, t0)
                    inflight.append((fut, est, now))
                while inflight and inflight[0][0].done():
                    fut, est, adm = inflight.popleft()
                    a = fut.result()
                    a.admitted = adm
                    with lock:
                        used_bytes += a.nbytes - est
                        self.bytes_per_unknown = max(self.bytes_per_unknown,
                                                     (a.nbytes - 24 * a.n) / a.n)
                    active.append(a)
                if not active:
                    if inflight:
                        inflight[0][0].result()
                    elif pending:
                        time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
                    continue
                done, infos = self._step([a.ctx for a in active])
                steps += 1
                tnow = time.perf_counter() - t0
                keep = []
                for a, d, info in zip(active, done, infos):
                    if not d:
                        keep.append(a)
                        continue
                    self.records.append(Record(a.req.rid, a.req.side, a.n, a.req.arrival,
                                               a.admitted, a.started, tnow, info.status,
                                               info.iterations, info.relres, a.nbytes))
                    if self.keep_solutions:
                        self.solutions[a.req.rid] = self._solution(a)
                    self._release(a)
                    used_bytes -= a.nbytes
                    used_parts -= a.parts
                active = keep
        finally:
            pool.shutdown(wait=True)
        wall = time.perf_counter() - t0
        return self.summary(wall, steps)

    def summary(self, wall: float, steps: int) -> dict:
        rejected = sum(1 for r in self.records if r.rejected)
        served = [r for r in self.records if not r.rejected]
        lat = sorted(r.latency for r in served)
        if not lat:
            return {"completed": 0, "rejected": rejected}

        def pct(q):
            return lat[min(len(lat) - 1, int(math.ceil(q * len(lat))) - 1)]

        first = min(r.arrival for r in served)
        last = max(r.finished for r in served)
        wait = [r.admitted - r.arrival for r in served]
        setup = [r.started - r.admitted for r in served]
        run = [r.finished - r.started for r in served]
        return {
            "completed": len(lat),
            "rejected": rejected,
            "failed": sum(1 for r in served if r.status != 0),
            "p50_ms": 1e3 * pct(0.50),
            "p99_ms": 1e3 * pct(0.99),
            "mean_ms": 1e3 * statistics.fmean(lat),
            "solves_per_s": len(lat) / max(last - first, 1e-9),
            "wall_s": wall,
            "steps": steps,
            "max_relres": max(r.relres for r in served),
            # where a request's latency goes: waiting for admission, host and
            # device setup (maps, factorisation), and solving in the batch
            "admission_wait_ms_mean": 1e3 * statistics.fmean(wait),
            "setup_ms_mean": 1e3 * statistics.fmean(setup),
            "solve_ms_mean": 1e3 * statistics.fmean(run),
        }
