"""The serving scheduler's host logic on CPU (no GPU): a fake backend stands
in for setup, batched steps and teardown, so admission by free subdomain
slots and device footprint, FIFO order, retirement and the latency summary
are checked without device work."""
import time
from dataclasses import dataclass

import pytest

import paper_2003_05361_gb300 as ras
from paper_2003_05361_gb300.serve import Request, Server, _Active, request_stream


@dataclass
class _Info:
    status: int
    iterations: int
    relres: float


class _FakeCtx:
    def __init__(self, req, turns, nbytes=0):
        self.req = req
        self.left = turns
        self.turns = 0
        self.nbytes = nbytes


class FakeServer(Server):
    """Setup returns a context that finishes after side // 128 + 1 turns;
    every batched turn is checked against the slot and byte limits."""

    def __init__(self, *args, over=0.9, **kwargs):
        super().__init__(*args, **kwargs)
        self.turn_log = []
        self.bytes_log = []  # device footprint of the active systems, per turn
        self.over = over     # true footprint / the estimate at admission

    def _default_stream(self):
        return None

    def _free_device_bytes(self):
        return 10 ** 12

    def _prepare(self, req, stream, t0):
        time.sleep(0.001)  # setup takes a little while (worker thread)
        px = -(-req.side // self.block)
        n = req.side * req.side
        nbytes = int(self.over * Server._estimate(Server(), req.side))
        return _Active(req, _FakeCtx(req, req.side // 128 + 1, nbytes), None, None, n, px * px,
                       nbytes, 0.0, time.perf_counter() - t0)

    def _step(self, ctxs):
        time.sleep(0.002)  # a batched turn takes longer than a setup
        parts = sum((-(-c.req.side // self.block)) ** 2 for c in ctxs)
        self.turn_log.append((len(ctxs), parts))
        self.bytes_log.append(sum(c.nbytes for c in ctxs))
        done, infos = [], []
        for c in ctxs:
            c.left -= 1
            c.turns += 1
            done.append(c.left == 0)
            infos.append(_Info(0, c.turns * self.step_limit, 1e-9))
        return done, infos

    def _release(self, a):
        a.ctx.left = -1  # released exactly once

    def _solution(self, a):
        return a.req.rid


@pytest.mark.parametrize("max_parts,budget_mb", [(600, 0), (40, 0), (20, 200)])
def test_scheduler_limits_order_and_completion(max_parts, budget_mb):
    reqs = request_stream(60, rate=2000.0, seed=5)
    srv = FakeServer(max_parts=max_parts, budget_bytes=budget_mb * 2 ** 20, workers=2,
                     keep_solutions=True)
    stats = srv.run(reqs)
    budget = srv.budget_bytes
    never = {r.rid for r in reqs
             if (-(-r.side // 64)) ** 2 > max_parts or srv._estimate(r.side) > budget}
    if max_parts < 64 or budget_mb:
        assert never  # the stream has requests that can never fit these limits
    assert stats["rejected"] == len(never) and stats["failed"] == 0
    assert stats["completed"] == 60 - len(never)
    assert {r.rid for r in srv.records if r.rejected} == never
    assert all(r.status == ras.RAS_ENOTSUP for r in srv.records if r.rejected)
    assert srv.solutions == {r: r for r in range(60) if r not in never}
    # every batched turn respects the shared subdomain slots and the byte budget
    assert all(parts <= max_parts for _, parts in srv.turn_log)
    assert all(nb <= budget for nb in srv.bytes_log)
    assert max(n for n, _ in srv.turn_log) >= 2  # systems really run side by side
    # admission is first come, first served, and never before arrival
    served = sorted((r for r in srv.records if not r.rejected), key=lambda r: r.rid)
    adm = [r.admitted for r in served]
    assert all(a <= b for a, b in zip(adm, adm[1:]))
    assert all(r.admitted >= r.arrival - 1e-9 and r.finished >= r.started for r in served)
    assert stats["p50_ms"] <= stats["p99_ms"]
    assert stats["admission_wait_ms_mean"] >= 0.0


def test_scheduler_waits_for_future_arrivals():
    reqs = [Request(0, 64, 0.0, 1000), Request(1, 128, 0.05, 1001)]
    srv = FakeServer()
    t0 = time.perf_counter()
    stats = srv.run(reqs)
    assert stats["completed"] == 2 and stats["rejected"] == 0
    assert time.perf_counter() - t0 >= 0.05
    r1 = next(r for r in srv.records if r.rid == 1)
    assert r1.admitted >= 0.05


def test_footprint_budget_limits_concurrency():
    # room for two 256^2 systems at a time: never more than two in a turn
    srv = FakeServer(budget_bytes=0)
    srv.budget_bytes = int(2.5 * srv._estimate(256))
    reqs = [Request(i, 256, 0.0, 1000 + i) for i in range(6)]
    stats = srv.run(reqs)
    assert stats["completed"] == 6 and stats["rejected"] == 0
    assert max(n for n, _ in srv.turn_log) == 2


def test_footprint_budget_is_never_exceeded_when_estimates_are_high():
    # the true footprint below the estimate (0.9 x): every turn stays within
    # the budget
    srv = FakeServer(budget_bytes=0)
    srv.budget_bytes = int(2.5 * srv._estimate(256))
    reqs = [Request(i, 256, 0.0, 1000 + i) for i in range(6)]
    srv.run(reqs)
    assert srv.bytes_log and all(nb <= srv.budget_bytes for nb in srv.bytes_log)


def test_footprint_correction_when_estimates_are_low():
    # the true footprint 1.4 x the initial estimate: the systems admitted on
    # the first estimate may overshoot the budget, the measured footprint then
    # raises the per-unknown estimate, and later admissions keep the budget
    est0 = Server()._estimate(256)
    srv = FakeServer(budget_bytes=0, over=1.4, workers=1)
    srv.budget_bytes = int(2.5 * est0)
    reqs = [Request(i, 256, 0.01 * i, 1000 + i) for i in range(8)]
    stats = srv.run(reqs)
    assert stats["completed"] == 8 and stats["rejected"] == 0
    true_bpu = (int(1.4 * est0) - 24 * 256 * 256) / (256 * 256)
    assert abs(srv.bytes_per_unknown - true_bpu) < 1e-6
    # at most the first wave (two systems admitted on the low estimate)
    # overshoots, and by no more than their underestimate
    over_first_wave = 2 * (int(1.4 * est0) - est0)
    assert all(nb <= srv.budget_bytes + over_first_wave for nb in srv.bytes_log)
    # once the estimate is right, no turn holds more than fits the budget
    assert max(n for n, _ in srv.turn_log[-3:]) <= 2
