"""Continuous batching: a request's result must be the same alone and in the
mix. Sync FP64: bitwise equal (every system reduces its residual in a fixed
order that does not depend on the batch). Async: both results meet the
tolerance and differ by at most 2 kappa tol relative (each is within
kappa * relres of the exact solution)."""
import math

import numpy as np
import pytest

import oracle
import paper_2003_05361_gb300 as ras
import problems
from paper_2003_05361_gb300.serve import Request, Server, request_stream

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def solve_alone(side, seed, mode, prec, tol):
    A = problems.poisson2d(side)
    b = problems.rhs_uniform(A.n, seed)
    px = math.ceil(side / 64)
    part = ras.ras_partition_regular2d(side, side, px, px)
    ctx = ras.ras_setup(A, part, px * px, 2, ras.RAS_LOCAL_BANDCHOL, prec)
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    info = ras.ras_solve(ctx, torch.tensor(b, device="cuda"), x, tol, mode)
    assert info.status == 0
    ras.ras_destroy(ctx)
    return A, b, x.cpu().numpy()


def requests_small():
    # arrivals spread over ~0.2 s so that several overlap on the GPU
    sides = [64, 150, 97, 200, 64, 128, 180]
    return [Request(i, s, 0.03 * i, 1000 + i) for i, s in enumerate(sides)]


def test_serving_sync_fp64_bitwise_equal_to_alone():
    srv = Server(mode=ras.RAS_SYNC, prec=ras.RAS_FP64, step_limit=25, keep_solutions=True)
    stats = srv.run(requests_small())
    assert stats["completed"] == 7 and stats["failed"] == 0
    # requests overlapped: at least one was admitted before another finished
    recs = sorted(srv.records, key=lambda r: r.arrival)
    assert any(recs[i + 1].admitted < recs[i].finished for i in range(len(recs) - 1))
    for r in srv.records:
        A, b, x = solve_alone(r.side, 1000 + r.rid, ras.RAS_SYNC, ras.RAS_FP64, 1e-8)
        assert np.array_equal(srv.solutions[r.rid], x), r.rid


def test_serving_async_mixed_within_tolerance_of_alone():
    tol = 1e-8
    srv = Server(mode=ras.RAS_ASYNC, prec=ras.RAS_FP32, step_limit=15, keep_solutions=True,
                 tol=tol)
    stats = srv.run(requests_small())
    assert stats["completed"] == 7 and stats["failed"] == 0
    for r in srv.records:
        A, b, x = solve_alone(r.side, 1000 + r.rid, ras.RAS_ASYNC, ras.RAS_FP32, tol)
        xm = srv.solutions[r.rid]
        for v in (x, xm):
            _, rn = oracle.residual(A, b, v)
            assert rn / np.linalg.norm(b) < tol
        h = 1.0 / (r.side + 1)
        kappa = 1.0 / math.sin(math.pi * h / 2) ** 2  # lam_max / lam_min bound of the 5-point matrix
        assert np.linalg.norm(xm - x) <= 2 * kappa * tol * np.linalg.norm(x)


def test_request_stream_is_seeded_and_in_range():
    a = request_stream(200, rate=50.0, seed=5)
    b = request_stream(200, rate=50.0, seed=5)
    assert [(r.side, r.arrival) for r in a] == [(r.side, r.arrival) for r in b]
    assert all(64 <= r.side <= 512 for r in a)
    assert all(a[i].arrival < a[i + 1].arrival for i in range(len(a) - 1))
    # mean inter-arrival ~ 1/rate
    gaps = np.diff([0.0] + [r.arrival for r in a])
    assert 0.7 / 50 < gaps.mean() < 1.3 / 50
