"""Direct solves of the global system A x = b for the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring): these give the FP64
reference solution x* = A^{-1} b that the RAS iterates converge to (the fixed
point of the RAS iteration, Sec. 2.1), against which errors are stated.

* poisson2d_direct / poisson3d_direct: the 5-point (7-point) Dirichlet
  Laplacian of Sec. 4.1 (diagonal 4 (6), off-diagonal -1, no h^2 scaling) is
  the Kronecker sum of the 1D operator T = tridiag(-1, 2, -1) along each grid
  axis. T = S diag(lam) S with the discrete sine transform matrix
  S[j, k] = sqrt(2/(N+1)) sin(pi (j+1)(k+1)/(N+1)) (symmetric and orthogonal)
  and lam[k] = 2 - 2 cos(pi (k+1)/(N+1)); so A^{-1} b is: transform b with S
  along every axis, divide entry (i, j[, k]) by lam[i] + lam[j] (+ lam[k]),
  transform back. Dense matrix products (numpy), exact up to FP64 rounding.
* band_direct_solve: banded Cholesky of the whole matrix in natural order
  (the oracle's or_band_cholesky / or_band_solve on A itself, i.e. RAS with
  one subdomain), for any SPD matrix whose band fits in memory.
"""
from __future__ import annotations

import numpy as np


def _sine_basis(N: int):
    k = np.arange(1, N + 1, dtype=np.float64)
    S = np.sqrt(2.0 / (N + 1)) * np.sin(np.pi * np.outer(k, k) / (N + 1))
    lam = 2.0 - 2.0 * np.cos(np.pi * k / (N + 1))
    return S, lam


def poisson2d_direct(N: int, b: np.ndarray) -> np.ndarray:
    """x = A^{-1} b for the N x N 5-point Laplacian (index y*N + x)."""
    S, lam = _sine_basis(N)
    B = np.asarray(b, dtype=np.float64).reshape(N, N)  # B[y, x]
    Bh = S @ B @ S
    Yh = Bh / (lam[:, None] + lam[None, :])
    return (S @ Yh @ S).reshape(-1)


def poisson3d_direct(N: int, b: np.ndarray) -> np.ndarray:
    """x = A^{-1} b for the N^3 7-point Laplacian (index (z*N + y)*N + x)."""
    S, lam = _sine_basis(N)
    B = np.asarray(b, dtype=np.float64).reshape(N, N, N)  # B[z, y, x]

    def transform(X):
        X = np.tensordot(S, X, axes=([1], [0]))  # along z
        X = np.einsum("jb,abc->ajc", S, X)  # along y
        X = np.einsum("kc,abc->abk", S, X)  # along x
        return X

    Bh = transform(B)
    Yh = Bh / (lam[:, None, None] + lam[None, :, None] + lam[None, None, :])
    return transform(Yh).reshape(-1)


def band_direct_solve(A, b: np.ndarray) -> np.ndarray:
    """x = A^{-1} b by banded Cholesky of the whole SPD matrix A in natural
    order (half-bandwidth w = max |i - j| over the nonzeros; band storage
    n (w + 1) doubles)."""
    from . import band_cholesky, band_solve

    n = A.n
    rows = np.repeat(np.arange(n), np.diff(A.row_ptr))
    lower = A.col <= rows
    w = int(np.max(rows - A.col)) if A.nnz else 0
    band = np.zeros((n, w + 1))
    band[rows[lower], A.col[lower] - rows[lower] + w] = A.val[lower]
    L = band_cholesky(band, w)
    return band_solve(L, w, np.asarray(b, dtype=np.float64))
