"""Pins for the synthetic input generators (matrices and right-hand sides)."""
import numpy as np
import pytest

import problems


def test_splitmix64_published_vector(golden):
    want = [int(v, 16) for v in golden("splitmix64_seed0.txt")]
    got = [int(v) for v in problems.splitmix64(0, 3)]
    assert got == want


def test_uniform_range_and_moments():
    u = problems.uniform01(123, 200000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3
    assert abs(u.var() - 1.0 / 12.0) < 2e-3
    b = problems.rhs_uniform(1000, 1)
    assert b.min() >= -1.0 and b.max() < 1.0


def test_normals_moments():
    z = problems.normals(5, 200001)
    assert z.size == 200001
    assert abs(z.mean()) < 1e-2
    assert abs(z.std() - 1.0) < 1e-2


@pytest.mark.parametrize("N", [1, 2, 5, 16])
def test_poisson2d_structure(N):
    A = problems.poisson2d(N)
    S = A.to_scipy().toarray()
    assert A.n == N * N
    assert np.array_equal(S, S.T)
    assert np.all(np.diag(S) == 4.0)
    # row sum = 4 - (number of interior neighbours); corners 2, edges 1, interior 0
    rs = S.sum(1).reshape(N, N)
    want = np.zeros((N, N))
    for y in range(N):
        for x in range(N):
            want[y, x] = (x == 0) + (x == N - 1) + (y == 0) + (y == N - 1)
    assert np.array_equal(rs, want)
    # offsets {-N, -1, 0, 1, N} of Sec. 4.1, cut at the row ends
    for i in range(A.n):
        cols = A.col[A.row_ptr[i]:A.row_ptr[i + 1]]
        assert np.all(np.diff(cols) > 0)
        for c in cols:
            d = c - i
            assert d in (-N, -1, 0, 1, N)
            if abs(d) == 1:
                assert c // N == i // N


def test_poisson3d_structure():
    N = 4
    A = problems.poisson3d(N)
    S = A.to_scipy().toarray()
    assert np.array_equal(S, S.T)
    assert np.all(np.diag(S) == 6.0)
    assert A.nnz == N ** 3 + 2 * 3 * N * N * (N - 1)


@pytest.mark.parametrize("N", [8, 33])
def test_eigenvector_rhs(N):
    A = problems.poisson2d(N)
    b, u, lam = problems.rhs_eigen2d(N)
    Au = A.matvec(u)
    assert np.linalg.norm(Au - lam * u) <= 1e-14 * np.linalg.norm(lam * u) * 10
    # it is the smallest eigenvalue of the dense matrix
    if N <= 8:
        ev = np.linalg.eigvalsh(A.to_scipy().toarray())
        assert abs(ev[0] - lam) < 1e-12


def test_eigenvector_rhs3d():
    N = 6
    A = problems.poisson3d(N)
    b, u, lam = problems.rhs_eigen3d(N)
    assert np.linalg.norm(A.matvec(u) - lam * u) <= 1e-13 * np.linalg.norm(b)


def test_diffusion_constant_k_is_poisson():
    N = 7
    A = problems.diffusion2d(N, np.ones((N, N)))
    P = problems.poisson2d(N)
    assert np.allclose(A.to_scipy().toarray(), P.to_scipy().toarray(), atol=0, rtol=0)


def test_diffusion_structure():
    N = 9
    k = problems.grf_coefficient(N, seed=4)
    A = problems.diffusion2d(N, k)
    S = A.to_scipy().toarray()
    assert np.allclose(S, S.T, rtol=0, atol=0)
    # row sums are the boundary-face coefficients (interior faces cancel)
    want = np.zeros((N, N))
    want[:, 0] += k[:, 0]
    want[:, -1] += k[:, -1]
    want[0, :] += k[0, :]
    want[-1, :] += k[-1, :]
    assert np.allclose(S.sum(1), want.ravel(), rtol=1e-12, atol=1e-12)
    # harmonic-mean face between nodes (0,0) and (0,1)
    kf = 2 * k[0, 0] * k[0, 1] / (k[0, 0] + k[0, 1])
    assert abs(S[0, 1] + kf) < 1e-14 * kf
    assert np.all(np.linalg.eigvalsh(S) > 0)


def test_grf_statistics():
    N = 256
    g = np.log(problems.grf_coefficient(N, seed=4))
    assert abs(g.mean()) < 0.2
    assert 0.7 < g.std() < 1.3
    # correlation at lag ~ ell (h = 1/257, ell = 1/32 -> 8 nodes): exp(-1/2)
    lag = 8
    c = np.mean(g[:, :-lag] * g[:, lag:]) / g.var()
    assert 0.45 < c < 0.75
    assert np.array_equal(g, np.log(problems.grf_coefficient(N, seed=4)))


@pytest.mark.parametrize("N,bx,by", [(5, 0.5, -0.3), (9, -1.2, 0.0), (16, 2.0, 3.0)])
def test_convdiff_structure(N, bx, by):
    A = problems.convdiff2d(N, bx, by)
    S = A.to_scipy().toarray()
    # flow reversal is the transpose; no convection is the Poisson matrix
    assert np.array_equal(S.T, problems.convdiff2d(N, -bx, -by).to_scipy().toarray())
    assert np.array_equal(problems.convdiff2d(N, 0.0, 0.0).to_scipy().toarray(),
                          problems.poisson2d(N).to_scipy().toarray())
    # M-matrix rows: positive diagonal, non-positive off-diagonal, zero row sum
    # away from the boundary (upwinding adds |b| to the diagonal and to one side)
    assert np.all(np.diag(S) == 4.0 + abs(bx) + abs(by))
    off = S - np.diag(np.diag(S))
    assert np.all(off <= 0.0)
    rs = S.sum(1).reshape(N, N)
    if N > 2:
        assert np.allclose(rs[1:-1, 1:-1], 0.0, atol=1e-14)
    assert np.all(rs >= -1e-14)
    # west neighbour of (x, y) carries -(1 + max(bx, 0))
    i = 1 * N + 1 if N > 2 else 1
    assert S[i, i - 1] == -1.0 - max(bx, 0.0) and S[i, i + 1] == -1.0 - max(-bx, 0.0)
    if bx or by:
        assert not np.array_equal(S, S.T)


@pytest.mark.parametrize("N,bx,by", [(8, 0.5, -0.3), (33, 1.5, 0.25), (20, 0.0, 0.0)])
def test_convdiff_eigenvector_closed_form(N, bx, by):
    A = problems.convdiff2d(N, bx, by)
    b, u, lam = problems.rhs_eigen_convdiff2d(N, bx, by)
    assert np.linalg.norm(A.matvec(u) - lam * u) <= 1e-13 * np.linalg.norm(u) * lam
    assert np.array_equal(b, lam * u)
    if bx == 0.0 and by == 0.0:
        b2, u2, lam2 = problems.rhs_eigen2d(N)
        assert np.allclose(u, u2, rtol=1e-14) and abs(lam - lam2) <= 1e-15
    # the smallest eigenvalue of the nonsymmetric matrix (all eigenvalues are real)
    ev = np.linalg.eigvals(A.to_scipy().toarray())
    assert abs(np.min(ev.real) - lam) <= 1e-10 and np.max(np.abs(ev.imag)) <= 1e-8
