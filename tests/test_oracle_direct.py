"""Pins of the oracle's global direct solves and of its set-up / iterate split.

The direct solves give x* = A^{-1} b, the fixed point of RAS (Sec. 2.1), which
the errors of the CUDA path are stated against. They are pinned here against
textbook routines (numpy's dense solve, the oracle's dense LU with partial
pivoting), the closed-form eigenvector solution of the Sec. 4.1 Laplacian and
the residual of the full-size solve.
"""
import numpy as np
import pytest

import oracle
import problems


def _dense(A):
    return A.to_scipy().toarray()


@pytest.mark.parametrize("N", [1, 2, 4, 7, 12])
def test_poisson2d_direct_vs_dense_lu(N):
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 3 + N)
    x = oracle.poisson2d_direct(N, b)
    xl = oracle.dense_lu_solve(_dense(A), b)
    xn = np.linalg.solve(_dense(A), b)
    assert np.abs(x - xl).max() <= 1e-13 * np.abs(xl).max()
    assert np.abs(x - xn).max() <= 1e-13 * np.abs(xn).max()


@pytest.mark.parametrize("N", [1, 3, 5])
def test_poisson3d_direct_vs_dense_lu(N):
    A = problems.poisson3d(N)
    b = problems.rhs_uniform(A.n, 7 + N)
    x = oracle.poisson3d_direct(N, b)
    xl = oracle.dense_lu_solve(_dense(A), b)
    assert np.abs(x - xl).max() <= 1e-13 * np.abs(xl).max()


def test_poisson2d_direct_anisotropic_rhs_orientation():
    # a right-hand side that is not symmetric in x <-> y catches a transposed
    # operand (S B S vs S B^T S)
    N = 9
    A = problems.poisson2d(N)
    b = np.zeros(A.n)
    b[0 * N + 3] = 1.0  # y = 0, x = 3
    b[5 * N + 1] = -2.0
    x = oracle.poisson2d_direct(N, b)
    assert np.abs(A.matvec(x) - b).max() <= 1e-13


def test_poisson_direct_eigenvector_closed_form():
    # b = lambda u with u the lowest discrete eigenvector: x* = u exactly
    for N in (16, 64):
        A = problems.poisson2d(N)
        b, u, lam = problems.rhs_eigen2d(N)
        x = oracle.poisson2d_direct(N, b)
        assert np.abs(x - u).max() <= 1e-12 * np.abs(u).max()
    N = 12
    b, u, lam = problems.rhs_eigen3d(N)
    x = oracle.poisson3d_direct(N, b)
    assert np.abs(x - u).max() <= 1e-12 * np.abs(u).max()


def test_poisson2d_direct_full_size_residual():
    # the 1024^2 benchmark system: ||b - A x*|| / ||b|| at FP64 rounding level
    N = 1024
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 1)
    x = oracle.poisson2d_direct(N, b)
    _, rn = oracle.residual(A, b, x)
    assert rn <= 1e-11 * np.linalg.norm(b)


@pytest.mark.parametrize("case", ["poisson", "diffusion"])
def test_band_direct_solve(case):
    N = 11
    A = problems.poisson2d(N) if case == "poisson" else \
        problems.diffusion2d(N, problems.grf_coefficient(N, 2))
    b = problems.rhs_uniform(A.n, 5)
    x = oracle.band_direct_solve(A, b)
    xl = oracle.dense_lu_solve(_dense(A), b)
    assert np.abs(x - xl).max() <= 1e-12 * np.abs(xl).max()
    if case == "poisson":
        xp = oracle.poisson2d_direct(N, b)
        assert np.abs(x - xp).max() <= 1e-13 * np.abs(xp).max()


def test_band_direct_solve_matches_closed_form_at_64():
    N = 64
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 9)
    x = oracle.band_direct_solve(A, b)
    xp = oracle.poisson2d_direct(N, b)
    assert np.abs(x - xp).max() <= 1e-12 * np.abs(xp).max()


# ---------------------------------------------------------------- set-up / iterate split

@pytest.mark.parametrize("kind,prec", [(oracle.BANDCHOL, oracle.FP64), (oracle.CG, oracle.FP32),
                                       (oracle.ILU0_CG, oracle.FP64)])
def test_setup_iterate_split_equals_ras_sync(kind, prec):
    N = 20
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 2)
    part = oracle.partition_regular2d(N, N, 2, 2)
    xr, kr, hr = oracle.ras_sync(A, b, part, 4, 2, kind, prec, 5, tol=0.0, max_iter=6,
                                 allow_noconv=True)
    h = oracle.RasSetup(A, part, 4, 2, kind, prec, 5)
    assert h.setup_s > 0.0
    x = np.zeros(A.n)
    k1, h1 = h.iterate(b, x, max_iter=2)
    k2, h2 = h.iterate(b, x, max_iter=4, nthreads=3)
    assert (k1, k2, kr) == (2, 4, 6)
    assert np.array_equal(x, xr)  # same bits: iterations continue from x
    assert np.array_equal(np.concatenate([h1[:2], h2]), hr)
    h.close()


def test_setup_iterate_converges_to_direct_solution():
    N = 24
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 4)
    part = oracle.partition_regular2d(N, N, 3, 2)
    h = oracle.RasSetup(A, part, 6, 2)
    x = np.zeros(A.n)
    k, hist = h.iterate(b, x, tol=1e-11, max_iter=5000, allow_noconv=False)
    assert hist[-1] < 1e-11
    xs = oracle.poisson2d_direct(N, b)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
