"""GPU parity tests for general (nonsymmetric) systems: the banded LU and
GMRES local solvers (Sec. 4.1 names LU and GMRES as the local solvers of a
generic system) on the upwind convection-diffusion matrix, through the C ABI
against the CPU oracle.

Bars: synchronous FP64 iterates equal to the oracle's up to rounding (1e-12
relative for banded LU, whose blocked substitutions only reorder sums; 1e-9
for GMRES, whose classical Gram-Schmidt applied twice reorders the modified
Gram-Schmidt of the oracle); FP32 iterates within a few times the FP32
rounding the oracle itself shows against FP64; every converged result has a
true FP64 relative residual below the tolerance and an error against the
direct solution within the bound the residual implies."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
import paper_2003_05361_gb300 as ras
import problems

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

LU, GM = ras.RAS_LOCAL_BANDLU, ras.RAS_LOCAL_GMRES
F64, F32, BF16 = ras.RAS_FP64, ras.RAS_FP32, ras.RAS_BF16_STORE
OR_KIND = {LU: oracle.BANDLU, GM: oracle.GMRES}
OR_PREC = {F64: oracle.FP64, F32: oracle.FP32, BF16: oracle.BF16}


def gpu_solve(A, b, part, P, gamma, kind, prec=F64, m=20, mode=ras.RAS_SYNC, tol=1e-8,
              max_updates=0, ctx=None):
    own = ctx is None
    if own:
        ctx = ras.ras_setup(A, part, P, gamma, kind, prec, m)
    bd = torch.tensor(b, device="cuda")
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    info = ras.ras_solve(ctx, bd, x, tol, mode, max_updates)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    if own:
        ras.ras_destroy(ctx)
    return xh, info


def true_relres(A, b, x):
    _, rn = oracle.residual(A, b, x)
    return rn / np.linalg.norm(b)


@pytest.mark.parametrize("kind,m,rtol", [(LU, 1, 1e-12), (GM, 8, 1e-9), (GM, 20, 1e-9)])
def test_sync_trajectory_matches_oracle(kind, m, rtol):
    # ragged grid (45 = 15 * 3, rows split 23 / 22): several 32-row tiles per
    # subdomain and a partial last tile; strong convection
    NX = 45
    A = problems.convdiff2d(NX, 1.5, -0.7)
    b = problems.rhs_uniform(A.n, 21)
    part = ras.ras_partition_regular2d(NX, NX, 3, 2)
    ctx = ras.ras_setup(A, part, 6, 2, kind, F64, m)
    assert ras.ras_get_launch(ctx)["kernel_variant"] == (0 if kind == LU else 4)
    for k in (1, 2, 5):
        x, info = gpu_solve(A, b, part, 6, 2, kind, F64, m, max_updates=k, ctx=ctx)
        assert info.status == ras.RAS_ENOCONV and info.iterations == k
        xo = oracle.ras_sync(A, b, part, 6, 2, OR_KIND[kind], oracle.FP64, m, tol=0.0, max_iter=k,
                             allow_noconv=True)[0]
        assert np.abs(x - xo).max() <= rtol * np.abs(xo).max(), k
    ras.ras_destroy(ctx)


@pytest.mark.parametrize("kind,m", [(LU, 1), (GM, 20)])
def test_fp32_iterates_match_oracle_fp32(kind, m):
    # FP32 local solves (factors rounded to FP32 / FP32 Arnoldi): the GPU and
    # the oracle round differently, so each sits within the FP32 rounding
    # distance of the FP64 iterate; their gap is bounded by a few times the
    # oracle's own FP32-vs-FP64 gap
    NX = 45
    A = problems.convdiff2d(NX, 0.9, 0.4)
    b = problems.rhs_uniform(A.n, 22)
    part = ras.ras_partition_regular2d(NX, NX, 3, 2)
    ctx = ras.ras_setup(A, part, 6, 2, kind, F32, m)
    for k in (1, 3):
        x, info = gpu_solve(A, b, part, 6, 2, kind, F32, m, max_updates=k, ctx=ctx)
        assert info.iterations == k
        xo32 = oracle.ras_sync(A, b, part, 6, 2, OR_KIND[kind], oracle.FP32, m, tol=0.0,
                               max_iter=k, allow_noconv=True)[0]
        xo64 = oracle.ras_sync(A, b, part, 6, 2, OR_KIND[kind], oracle.FP64, m, tol=0.0,
                               max_iter=k, allow_noconv=True)[0]
        gap = np.abs(xo32 - xo64).max()
        assert 0.0 < gap <= 1e-4 * np.abs(xo64).max()
        assert np.abs(x - xo32).max() <= 4.0 * gap + 1e-7 * np.abs(xo64).max(), k
    ras.ras_destroy(ctx)


@pytest.mark.parametrize("kind", [LU, GM])
def test_sync_converged_matches_oracle_bfs_partition(kind):
    N = 60
    A = problems.convdiff2d(N, -1.2, 0.8)
    b = problems.rhs_uniform(A.n, 23)
    part = ras.ras_partition_bfs(A, 5, 2)
    x, info = gpu_solve(A, b, part, 5, 3, kind, F64, 12)
    xo, it, _ = oracle.ras_sync(A, b, part, 5, 3, OR_KIND[kind], oracle.FP64, 12, tol=1e-8)
    # GMRES makes the outer iteration non-linear in x: a different rounding
    # order may move the step where the threshold is crossed
    slack = 1 if kind == LU else max(2, int(0.01 * it))
    assert info.status == 0 and abs(info.iterations - it) <= slack
    assert true_relres(A, b, x) < 1e-8
    assert np.abs(x - xo).max() <= 1e-7 * np.abs(xo).max()


def test_band_lu_eigenvector_closed_form():
    # b = lam u with the closed-form lowest mode u: the exact solution is u
    N = 96
    A = problems.convdiff2d(N, 0.5, 0.5)
    b, u, lam = problems.rhs_eigen_convdiff2d(N, 0.5, 0.5)
    part = ras.ras_partition_regular2d(N, N, 2, 2)
    x, info = gpu_solve(A, b, part, 4, 2, LU, F64, tol=1e-10)
    xo, it, _ = oracle.ras_sync(A, b, part, 4, 2, oracle.BANDLU, oracle.FP64, 1, tol=1e-10)
    assert info.status == 0 and abs(info.iterations - it) <= 1
    rr = true_relres(A, b, x)
    assert rr < 1e-10
    assert np.linalg.norm(x - u) / np.linalg.norm(u) <= 1e-6
    assert np.abs(x - xo).max() <= 1e-10 * np.abs(xo).max()


@pytest.mark.parametrize("kind,prec", [(LU, F32), (LU, BF16), (GM, F32)])
def test_mixed_precision_reaches_fp64_accuracy(kind, prec):
    N = 64
    A = problems.convdiff2d(N, 1.0, -0.5)
    b = problems.rhs_uniform(A.n, 24)
    part = ras.ras_partition_regular2d(N, N, 2, 2)
    x, info = gpu_solve(A, b, part, 4, 2, kind, prec, 16, tol=1e-10)
    assert info.status == 0
    assert true_relres(A, b, x) < 1e-10
    xs = spla.spsolve(A.to_scipy().tocsc(), b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-7
    _, it, _ = oracle.ras_sync(A, b, part, 4, 2, OR_KIND[kind], OR_PREC[prec], 16, tol=1e-10)
    assert abs(info.iterations - it) <= max(3, 0.1 * it)


@pytest.mark.parametrize("kind,prec,mode", [(LU, F32, ras.RAS_ASYNC), (LU, F64, ras.RAS_ASYNC),
                                            (GM, F32, ras.RAS_ASYNC),
                                            (LU, F32, ras.RAS_ASYNC_DECENTRAL),
                                            (GM, F32, ras.RAS_ASYNC_DECENTRAL)])
def test_async_converges_to_direct_solution(kind, prec, mode):
    N = 64
    A = problems.convdiff2d(N, 2.0, 1.0)
    b = problems.rhs_uniform(A.n, 25)
    part = ras.ras_partition_regular2d(N, N, 4, 4)
    xs = spla.spsolve(A.to_scipy().tocsc(), b)
    ctx = ras.ras_setup(A, part, 16, 2, kind, prec, 10)
    for rep in range(3):
        x, info = gpu_solve(A, b, part, 16, 2, kind, prec, 10, mode=mode, tol=1e-9, ctx=ctx)
        assert info.status == 0, info.as_dict()
        assert true_relres(A, b, x) < 1e-9
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-6
    ras.ras_destroy(ctx)


def test_single_subdomain_is_direct_solve():
    # P = 1: one banded-LU update is the exact solve; GMRES with more steps
    # than its 32 limit allows is not exact, so only LU is checked exactly
    N = 40
    A = problems.convdiff2d(N, 0.7, -0.3)
    b = problems.rhs_uniform(A.n, 26)
    part = np.zeros(A.n, dtype=np.int32)
    x, info = gpu_solve(A, b, part, 1, 1, LU, F64, tol=1e-12)
    assert info.status == 0 and info.iterations == 1
    xs = spla.spsolve(A.to_scipy().tocsc(), b)
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)


def test_gmres_exact_on_tiny_subdomains():
    # subdomains of at most 24 rows and 32 GMRES steps: the steps stop at the
    # subdomain size (the Krylov space is then the whole local space), so
    # every local solve is exact and the iterates equal banded LU's
    N = 12
    A = problems.convdiff2d(N, 0.6, 1.1)
    b = problems.rhs_uniform(A.n, 27)
    part = ras.ras_partition_regular2d(N, N, 3, 2)
    for k in (1, 4):
        xg, ig = gpu_solve(A, b, part, 6, 0, GM, F64, 32, max_updates=k)
        xl, il = gpu_solve(A, b, part, 6, 0, LU, F64, max_updates=k)
        assert ig.iterations == il.iterations == k
        assert np.linalg.norm(xg - xl) <= 1e-11 * np.linalg.norm(xl)


def test_zero_pivot_reports_enotspd():
    # [[0, 1], [1, 0]]: LU without pivoting meets u_00 = 0 during setup
    A = problems.CSR(2, np.array([0, 2, 4], np.int32), np.array([0, 1, 0, 1], np.int32),
                     np.array([0.0, 1.0, 1.0, 0.0]))
    with pytest.raises(ras.RasError) as e:
        ras.ras_setup(A, np.zeros(2, np.int32), 1, 0, LU, F64)
    assert e.value.status == ras.RAS_ENOTSPD


def test_batch_equals_solo_sync_bitwise():
    ctxs, bs, xs, solo = [], [], [], []
    for N, bx in ((40, 0.5), (52, -1.0)):
        A = problems.convdiff2d(N, bx, 0.3)
        b = problems.rhs_uniform(A.n, N)
        part = ras.ras_partition_regular2d(N, N, 2, 2)
        ctx = ras.ras_setup(A, part, 4, 2, GM, F64, 10)
        x1, info1 = gpu_solve(A, b, part, 4, 2, GM, F64, 10, ctx=ctx)
        solo.append((x1, info1.iterations))
        ctxs.append(ctx)
        bs.append(torch.tensor(b, device="cuda"))
        xs.append(torch.zeros(A.n, dtype=torch.float64, device="cuda"))
    infos = ras.ras_solve_batch(ctxs, bs, xs, 1e-8, ras.RAS_SYNC)
    for (x1, it1), x, info in zip(solo, xs, infos):
        assert info.status == 0 and info.iterations == it1
        assert np.array_equal(x.cpu().numpy(), x1)
    for c in ctxs:
        ras.ras_destroy(c)


@pytest.mark.parametrize("kind,prec", [(LU, F32), (GM, F32)])
def test_autotune_then_solve(kind, prec):
    N = 128
    A = problems.convdiff2d(N, 1.0, 1.0)
    b = problems.rhs_uniform(A.n, 28)
    part = ras.ras_partition_regular2d(N, N, 3, 3)
    ctx = ras.ras_setup(A, part, 9, 2, kind, prec, 12)
    xs = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    r = ras.ras_autotune(ctx, xs, ras.RAS_SYNC, 20, True)
    assert r.candidates >= 1 and r.inner_iters <= 12
    x, info = gpu_solve(A, b, part, 9, 2, kind, prec, 12, ctx=ctx)
    assert info.status == 0 and true_relres(A, b, x) < 1e-8
    ras.ras_destroy(ctx)
