"""Pins for the oracle's synchronous RAS iteration (Sec. 2.1, Algorithm 1),
against closed forms, special cases that reduce to textbook methods, and the
explicit iteration matrix on tiny systems."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
import problems


def dense(A):
    return A.to_scipy().toarray()


def iterate(A, b, part, P, gamma, k, **kw):
    """x^k of the oracle (k RAS updates from x^0 = 0)."""
    x, it, hist = oracle.ras_sync(A, b, part, P, gamma, tol=0.0, max_iter=k, allow_noconv=True, **kw)
    assert it == k
    return x, hist


def test_single_subdomain_is_direct_solve():
    # P = 1: Omega = everything, one update is the exact solve
    A = problems.poisson2d(20)
    b = problems.rhs_uniform(A.n, 1)
    x, it, hist = oracle.ras_sync(A, b, np.zeros(A.n, np.int32), 1, 2, tol=1e-8)
    assert it == 1
    assert hist[1] < 1e-13
    xs = spla.spsolve(A.to_scipy().tocsc(), b)
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)


def block_jacobi(S, b, part, P, k):
    """Textbook block Jacobi: x <- x + D^{-1} (b - S x), D = diag blocks of the partition."""
    x = np.zeros_like(b)
    blocks = [np.nonzero(part == p)[0] for p in range(P)]
    for _ in range(k):
        r = b - S @ x
        xn = x.copy()
        for idx in blocks:
            xn[idx] = x[idx] + np.linalg.solve(S[np.ix_(idx, idx)], r[idx])
        x = xn
    return x


@pytest.mark.parametrize("kind", [oracle.BANDCHOL, oracle.CG])
def test_zero_overlap_is_block_jacobi(kind):
    N = 12
    A = problems.poisson2d(N)
    S = dense(A)
    b = problems.rhs_uniform(A.n, 2)
    part = oracle.partition_regular2d(N, N, 3, 2)
    for k in (1, 2, 7):
        # CG with m >= block size is an exact local solve (finite termination)
        x, _ = iterate(A, b, part, 6, 0, k, kind=kind, m=60)
        xj = block_jacobi(S, b, part, 6, k)
        assert np.linalg.norm(x - xj) <= 1e-11 * max(np.linalg.norm(xj), 1.0)


def ras_operators(S, part, P, gamma, A):
    """Explicit RAS operators: returns (T, c_op) with x^{k+1} = T x^k + c_op b,
    T = I - sum_p Rt_p^T A_p^{-1} R_p S (Rt_p: restriction to owned points)."""
    n = S.shape[0]
    M = np.zeros((n, n))
    G = np.zeros((n, n), bool)
    for i in range(n):
        G[i, A.col[A.row_ptr[i]:A.row_ptr[i + 1]]] = True
    for p in range(P):
        # Omega_p by gamma rounds of graph growth (independent of the oracle)
        inside = part == p
        for _ in range(gamma):
            inside = inside | G[inside].any(0)
        om = np.nonzero(inside)[0]
        R = np.zeros((om.size, n))
        R[np.arange(om.size), om] = 1.0
        Rt = R.copy()
        Rt[part[om] != p] = 0.0
        Ap = S[np.ix_(om, om)]
        M += Rt.T @ np.linalg.solve(Ap, R)
    return np.eye(n) - M @ S, M


@pytest.mark.parametrize("N,px,py,gamma", [(6, 2, 2, 1), (8, 2, 2, 2), (7, 3, 1, 1)])
def test_iteration_matrix(N, px, py, gamma):
    A = problems.poisson2d(N)
    S = dense(A)
    b = problems.rhs_uniform(A.n, 3)
    P = px * py
    part = oracle.partition_regular2d(N, N, px, py)
    T, M = ras_operators(S, part, P, gamma, A)
    assert np.max(np.abs(np.linalg.eigvals(T))) < 1.0
    xk = np.zeros(A.n)
    for k in range(1, 6):
        xk = T @ xk + M @ b
        x, _ = iterate(A, b, part, P, gamma, k)
        assert np.linalg.norm(x - xk) <= 1e-12 * np.linalg.norm(xk)


def test_iteration_matrix_bfs_partition():
    A = problems.poisson3d(4)
    S = dense(A)
    b = problems.rhs_uniform(A.n, 4)
    part = oracle.partition_bfs(A, 3, 1)
    T, M = ras_operators(S, part, 3, 1, A)
    xk = np.zeros(A.n)
    for k in range(1, 4):
        xk = T @ xk + M @ b
        x, _ = iterate(A, b, part, 3, 1, k)
        assert np.linalg.norm(x - xk) <= 1e-12 * np.linalg.norm(xk)


def test_eigenvector_closed_form_config1():
    # b = lam_min u with u the lowest mode: ||x - u|| / ||u|| <= ||r|| / ||b||
    N = 128
    A = problems.poisson2d(N)
    b, u, lam = problems.rhs_eigen2d(N)
    part = oracle.partition_regular2d(N, N, 2, 2)
    x, it, hist = oracle.ras_sync(A, b, part, 4, 2, tol=1e-8)
    err = np.linalg.norm(x - u) / np.linalg.norm(u)
    assert hist[-1] < 1e-8 <= hist[-2]
    assert err <= hist[-1] * (1 + 1e-6)
    assert 200 <= it <= 320


def test_dense_lu_16x16():
    N = 16
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 5)
    xd = oracle.dense_lu_solve(dense(A), b)
    assert np.allclose(xd, np.linalg.solve(dense(A), b), rtol=1e-12)
    part = oracle.partition_regular2d(N, N, 2, 2)
    x, it, hist = oracle.ras_sync(A, b, part, 4, 2, tol=1e-10)
    kappa = np.linalg.cond(dense(A))
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= kappa * hist[-1]
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-8


def test_history_is_true_residual():
    N = 24
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 7)
    part = oracle.partition_regular2d(N, N, 2, 3)
    x, hist = iterate(A, b, part, 6, 2, 9)
    r = b - A.to_scipy() @ x
    assert abs(hist[-1] - np.linalg.norm(r) / np.linalg.norm(b)) <= 1e-14


def test_overlap_reduces_iterations():
    # Sec. 4.3: larger overlap -> faster information propagation, fewer iterations
    N = 48
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 1)
    part = oracle.partition_regular2d(N, N, 3, 2)
    its = []
    for g in (0, 1, 2, 4):
        _, it, _ = oracle.ras_sync(A, b, part, 6, g, tol=1e-8)
        its.append(it)
    assert its == sorted(its, reverse=True) and its[0] > its[-1]


def test_regular1d_information_propagation():
    # Sec. 3.2.1: with regular1d, information needs P-1 solves to travel from
    # the first strip to the last. A right-hand side supported in strip 0
    # leaves strip P-1 untouched for the first P-2 updates (overlap 0).
    N, P = 16, 5
    A = problems.poisson2d(N)
    part = oracle.partition_regular2d(N, N, 1, P)
    b = np.where(part == 0, 1.0, 0.0)
    for k in range(1, P + 1):
        x, _ = iterate(A, b, part, P, 0, k)
        last = np.abs(x[part == P - 1]).max()
        if k <= P - 1:
            assert last == 0.0
        else:
            assert last > 0.0


@pytest.mark.parametrize("prec", [oracle.FP32, oracle.BF16])
def test_mixed_precision_reaches_fp64_accuracy(prec):
    # correction form: FP32/BF16 local factors, FP64 residual and update
    N = 64
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 1)
    part = oracle.partition_regular2d(N, N, 2, 2)
    x64, it64, _ = oracle.ras_sync(A, b, part, 4, 2, tol=1e-10)
    x, it, hist = oracle.ras_sync(A, b, part, 4, 2, prec=prec, tol=1e-10)
    assert hist[-1] < 1e-10
    xs = spla.spsolve(A.to_scipy().tocsc(), b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= 1e-7
    if prec == oracle.FP32:
        assert abs(it - it64) <= 2
    else:
        assert it >= it64


def test_local_solver_variants_converge():
    N = 40
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 3)
    part = oracle.partition_regular2d(N, N, 2, 2)
    xs = spla.spsolve(A.to_scipy().tocsc(), b)
    for kind, prec in [(oracle.CG, oracle.FP64), (oracle.CG, oracle.FP32),
                       (oracle.ILU0_CG, oracle.FP64), (oracle.ILU0_CG, oracle.FP32)]:
        x, it, hist = oracle.ras_sync(A, b, part, 4, 2, kind=kind, prec=prec, m=10, tol=1e-9)
        assert hist[-1] < 1e-9
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-6


def test_cg_with_many_steps_equals_direct_local_solve():
    N = 14
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 9)
    part = oracle.partition_regular2d(N, N, 2, 2)
    xd, _ = iterate(A, b, part, 4, 1, 6)
    xc, _ = iterate(A, b, part, 4, 1, 6, kind=oracle.CG, m=200)
    assert np.linalg.norm(xd - xc) <= 1e-10 * np.linalg.norm(xd)


def test_openmp_threads_same_result():
    N = 32
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 3)
    part = oracle.partition_regular2d(N, N, 4, 4)
    x1, it1, h1 = oracle.ras_sync(A, b, part, 16, 2, nthreads=1)
    x4, it4, h4 = oracle.ras_sync(A, b, part, 16, 2, nthreads=4)
    assert it1 == it4 and np.array_equal(x1, x4) and np.array_equal(h1, h4)


def test_invalid_inputs():
    A = problems.poisson2d(4)
    b = np.ones(16)
    with pytest.raises(oracle.OracleError):
        oracle.ras_sync(A, b, np.full(16, 3, np.int32), 2, 1)
    with pytest.raises(oracle.OracleError):
        oracle.ras_sync(A, b, np.zeros(16, np.int32), 1, -1)
    with pytest.raises(oracle.OracleError):
        oracle.ras_sync(A, b, np.zeros(16, np.int32), 1, 1, kind=oracle.CG, prec=oracle.BF16)
    with pytest.raises(oracle.OracleError):
        oracle.ras_sync(A, b, np.zeros(16, np.int32), 1, 1, kind=oracle.GMRES, prec=oracle.BF16)
    with pytest.raises(oracle.OracleError):
        oracle.ras_sync(A, b, np.zeros(16, np.int32), 1, 1, kind=5)


# ---------------------------------------------------------------- nonsymmetric systems (Sec. 4.1:
# a generic system with LU or GMRES local solves)

def test_single_subdomain_nonsymmetric_is_direct_solve():
    A = problems.convdiff2d(16, 1.0, -0.5)
    b = problems.rhs_uniform(A.n, 1)
    xs = spla.spsolve(A.to_scipy().tocsc(), b)
    for kind, m in ((oracle.BANDLU, 1), (oracle.GMRES, A.n)):
        x, it, hist = oracle.ras_sync(A, b, np.zeros(A.n, np.int32), 1, 2, kind=kind, m=m, tol=1e-8)
        assert it == 1 and hist[1] < 1e-12
        assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)


@pytest.mark.parametrize("kind", [oracle.BANDLU, oracle.GMRES])
def test_zero_overlap_nonsymmetric_is_block_jacobi(kind):
    N = 12
    A = problems.convdiff2d(N, 0.6, 1.1)
    S = dense(A)
    b = problems.rhs_uniform(A.n, 2)
    part = oracle.partition_regular2d(N, N, 3, 2)
    for k in (1, 2, 7):
        # GMRES over the whole local space (24 rows) is an exact local solve
        x, _ = iterate(A, b, part, 6, 0, k, kind=kind, m=24)
        xj = block_jacobi(S, b, part, 6, k)
        assert np.linalg.norm(x - xj) <= 1e-11 * max(np.linalg.norm(xj), 1.0)


@pytest.mark.parametrize("N,px,py,gamma,bx,by", [(6, 2, 2, 1, 0.8, -0.3), (8, 2, 2, 2, -2.0, 1.0),
                                                 (7, 3, 1, 1, 4.0, 0.0)])
def test_iteration_matrix_nonsymmetric(N, px, py, gamma, bx, by):
    # RAS on an M-matrix converges (rho(T) < 1 for a nonsymmetric M-matrix too)
    A = problems.convdiff2d(N, bx, by)
    S = dense(A)
    b = problems.rhs_uniform(A.n, 3)
    P = px * py
    part = oracle.partition_regular2d(N, N, px, py)
    T, M = ras_operators(S, part, P, gamma, A)
    assert np.max(np.abs(np.linalg.eigvals(T))) < 1.0
    xk = np.zeros(A.n)
    for k in range(1, 6):
        xk = T @ xk + M @ b
        x, _ = iterate(A, b, part, P, gamma, k, kind=oracle.BANDLU)
        assert np.linalg.norm(x - xk) <= 1e-12 * np.linalg.norm(xk)


def test_nonsymmetric_converges_to_direct_solution():
    N = 40
    A = problems.convdiff2d(N, 1.5, -0.8)
    b = problems.rhs_uniform(A.n, 4)
    part = oracle.partition_regular2d(N, N, 2, 2)
    xs = spla.spsolve(A.to_scipy().tocsc(), b)
    its = {}
    for kind, prec, m in [(oracle.BANDLU, oracle.FP64, 1), (oracle.BANDLU, oracle.FP32, 1),
                          (oracle.BANDLU, oracle.BF16, 1), (oracle.GMRES, oracle.FP64, 20),
                          (oracle.GMRES, oracle.FP32, 20)]:
        x, it, hist = oracle.ras_sync(A, b, part, 4, 2, kind=kind, prec=prec, m=m, tol=1e-9)
        assert hist[-1] < 1e-9
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-7
        its[(kind, prec)] = it
    # FP32 factors: the correction form keeps the FP64 iteration count
    assert abs(its[(oracle.BANDLU, oracle.FP32)] - its[(oracle.BANDLU, oracle.FP64)]) <= 2


def test_gmres_with_full_local_space_equals_lu():
    N = 14
    A = problems.convdiff2d(N, -0.7, 0.9)
    b = problems.rhs_uniform(A.n, 9)
    part = oracle.partition_regular2d(N, N, 2, 2)
    xd, _ = iterate(A, b, part, 4, 1, 6, kind=oracle.BANDLU)
    xg, _ = iterate(A, b, part, 4, 1, 6, kind=oracle.GMRES, m=200)
    assert np.linalg.norm(xd - xg) <= 1e-10 * np.linalg.norm(xd)


def test_convdiff_eigenvector_rhs_error_bound():
    # b = lam u with u the closed-form lowest mode: x* = u exactly
    N = 48
    A = problems.convdiff2d(N, 0.5, 0.5)
    b, u, lam = problems.rhs_eigen_convdiff2d(N, 0.5, 0.5)
    part = oracle.partition_regular2d(N, N, 2, 2)
    x, it, hist = oracle.ras_sync(A, b, part, 4, 2, kind=oracle.BANDLU, tol=1e-10)
    kappa = np.linalg.cond(dense(A))
    assert np.linalg.norm(x - u) / np.linalg.norm(u) <= kappa * hist[-1]
    assert np.linalg.norm(x - u) / np.linalg.norm(u) <= 1e-7


# ---------------------------------------------------------------- optimized local matrices (ORAS)

def oras_operators(S, part, P, gamma, A, alpha):
    """Explicit operators with optimized local matrices, built from the dense
    matrix: A~_p = S[om, om] + alpha * diag(S[om, outside] row sums)."""
    n = S.shape[0]
    M = np.zeros((n, n))
    G = np.zeros((n, n), bool)
    for i in range(n):
        G[i, A.col[A.row_ptr[i]:A.row_ptr[i + 1]]] = True
    for p in range(P):
        inside = part == p
        for _ in range(gamma):
            inside = inside | G[inside].any(0)
        om = np.nonzero(inside)[0]
        Ap = S[np.ix_(om, om)] + alpha * np.diag(S[np.ix_(om, np.nonzero(~inside)[0])].sum(1))
        R = np.zeros((om.size, n))
        R[np.arange(om.size), om] = 1.0
        Rt = R.copy()
        Rt[part[om] != p] = 0.0
        M += Rt.T @ np.linalg.solve(Ap, R)
    return np.eye(n) - M @ S, M


def test_oras_alpha_zero_is_ras_bitwise():
    A = problems.poisson2d(24)
    b = problems.rhs_uniform(A.n, 7)
    part = oracle.partition_regular2d(24, 24, 2, 3)
    x0, h0 = iterate(A, b, part, 6, 2, 9)
    x1, h1 = iterate(A, b, part, 6, 2, 9, oras_alpha=0.0)
    assert np.array_equal(x0, x1) and np.array_equal(h0, h1)


@pytest.mark.parametrize("case,kind,alpha", [("poisson", oracle.BANDCHOL, 0.6),
                                             ("poisson", oracle.BANDCHOL, -0.4),
                                             ("convdiff", oracle.BANDLU, 0.5),
                                             ("diffusion", oracle.BANDCHOL, 0.7)])
def test_oras_iteration_matrix(case, kind, alpha):
    N = 8
    if case == "poisson":
        A = problems.poisson2d(N)
    elif case == "convdiff":
        A = problems.convdiff2d(N, 1.0, -0.5)
    else:
        A = problems.diffusion2d(N, problems.grf_coefficient(N, 5))
    S = dense(A)
    b = problems.rhs_uniform(A.n, 3)
    part = oracle.partition_regular2d(N, N, 2, 2)
    T, M = oras_operators(S, part, 4, 1, A, alpha)
    xk = np.zeros(A.n)
    for k in range(1, 6):
        xk = T @ xk + M @ b
        x, _ = iterate(A, b, part, 4, 1, k, kind=kind, oras_alpha=alpha)
        assert np.linalg.norm(x - xk) <= 1e-12 * np.linalg.norm(xk)


def test_oras_fixed_point_and_robin_speedup():
    # the residual stays that of A, so the limit is A^-1 b; a Robin-type
    # condition (alpha toward 1: p = (2/h)(1-alpha)/(1+alpha) on the Laplacian)
    # cuts the iteration count at overlap 2 and 4
    N = 64
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 1)
    part = oracle.partition_regular2d(N, N, 4, 4)
    xs = spla.spsolve(A.to_scipy().tocsc(), b)
    for gamma in (2, 4):
        its = []
        for alpha in (0.0, 0.5, 0.8):
            x, it, hist = oracle.ras_sync(A, b, part, 16, gamma, tol=1e-9, oras_alpha=alpha)
            assert hist[-1] < 1e-9
            assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-7
            its.append(it)
        assert its[0] > its[1] > its[2]
        assert its[2] < 0.6 * its[0]


def test_oras_cg_with_many_steps_equals_band():
    N = 14
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 9)
    part = oracle.partition_regular2d(N, N, 2, 2)
    xd, _ = iterate(A, b, part, 4, 1, 6, oras_alpha=0.5)
    xc, _ = iterate(A, b, part, 4, 1, 6, kind=oracle.CG, m=200, oras_alpha=0.5)
    xi, _ = iterate(A, b, part, 4, 1, 6, kind=oracle.GMRES, m=200, oras_alpha=0.5)
    assert np.linalg.norm(xd - xc) <= 1e-10 * np.linalg.norm(xd)
    assert np.linalg.norm(xd - xi) <= 1e-10 * np.linalg.norm(xd)
    with pytest.raises(oracle.OracleError):
        oracle.ras_sync(A, b, part, 4, 1, oras_alpha=float("nan"))
