"""Matrix and right-hand-side generators (numpy only).

Conventions shared by every consumer:

* 2D grids have N x N interior unknowns, index i = y*N + x (x fastest).
  3D grids: i = (z*N + y)*N + x.
* Dirichlet couplings to the boundary and across row ends are dropped, so the
  Sec. 4.1 stencil offsets {-N,-1,0,1,N} are the standard 5-point Laplacian
  with no h^2 scaling.
* CSR arrays: row_ptr int32[n+1], col int32[nnz] (ascending within a row),
  val float64[nnz].
* Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014): output k (k = 0,1,...) of a
  stream with seed s mixes the state s + (k+1)*0x9E3779B97F4A7C15 (mod 2^64).
  Uniform doubles are (z >> 11) * 2^-53.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


@dataclass
class CSR:
    """Host CSR matrix (int32 indices, float64 values)."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_scipy(self):
        import scipy.sparse as sp

        return sp.csr_matrix((self.val, self.col, self.row_ptr), shape=(self.n, self.n))

    def matvec(self, x: np.ndarray) -> np.ndarray:
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        return np.bincount(rows, weights=self.val * x[self.col], minlength=self.n)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream for `seed`."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits each."""
    z = splitmix64(seed, count, start)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normals(seed: int, count: int) -> np.ndarray:
    """Standard normals by the Box-Muller transform over SplitMix64 pairs."""
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def _assemble(n: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray) -> CSR:
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    return CSR(n, row_ptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64))


def _grid_stencil(shape, diag: float) -> CSR:
    """Constant-coefficient (2*dim+1)-point Laplacian on a tensor grid."""
    dims = len(shape)
    n = int(np.prod(shape))
    idx = np.arange(n).reshape(shape[::-1])  # [z][y][x] / [y][x]
    rows = [np.arange(n)]
    cols = [np.arange(n)]
    vals = [np.full(n, diag)]
    for axis in range(dims):
        # axis counted from the fastest index
        ax = dims - 1 - axis
        sl_lo = [slice(None)] * dims
        sl_hi = [slice(None)] * dims
        sl_lo[ax] = slice(0, -1)
        sl_hi[ax] = slice(1, None)
        a = idx[tuple(sl_lo)].ravel()
        b = idx[tuple(sl_hi)].ravel()
        rows += [a, b]
        cols += [b, a]
        vals += [np.full(a.size, -1.0), np.full(b.size, -1.0)]
    return _assemble(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def poisson2d(N: int) -> CSR:
    """2D 5-point Poisson matrix, N x N unknowns, diagonal 4, neighbours -1."""
    return _grid_stencil((N, N), 4.0)


def poisson3d(N: int) -> CSR:
    """3D 7-point Poisson matrix, N^3 unknowns, diagonal 6, neighbours -1."""
    return _grid_stencil((N, N, N), 6.0)


def diffusion2d(N: int, k: np.ndarray) -> CSR:
    """Node-centred -div(k grad u) on N x N interior nodes (no h^2 scaling).

    k has shape (N, N) indexed [y, x]. The face coefficient between two
    interior nodes is the harmonic mean 2 k_a k_b / (k_a + k_b); a face to the
    Dirichlet boundary (u = 0 outside) uses the interior node's k. Row i is
    sum_f k_f (u_i - u_nb).
    """
    k = np.asarray(k, dtype=np.float64)
    assert k.shape == (N, N)
    n = N * N
    idx = np.arange(n).reshape(N, N)
    diag = np.zeros((N, N))
    rows, cols, vals = [], [], []
    # x-faces between (y, x) and (y, x+1)
    kf = 2.0 * k[:, :-1] * k[:, 1:] / (k[:, :-1] + k[:, 1:])
    a, b = idx[:, :-1].ravel(), idx[:, 1:].ravel()
    rows += [a, b]
    cols += [b, a]
    vals += [-kf.ravel(), -kf.ravel()]
    diag[:, :-1] += kf
    diag[:, 1:] += kf
    # y-faces between (y, x) and (y+1, x)
    kf = 2.0 * k[:-1, :] * k[1:, :] / (k[:-1, :] + k[1:, :])
    a, b = idx[:-1, :].ravel(), idx[1:, :].ravel()
    rows += [a, b]
    cols += [b, a]
    vals += [-kf.ravel(), -kf.ravel()]
    diag[:-1, :] += kf
    diag[1:, :] += kf
    # boundary faces
    diag[:, 0] += k[:, 0]
    diag[:, -1] += k[:, -1]
    diag[0, :] += k[0, :]
    diag[-1, :] += k[-1, :]
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag.ravel())
    return _assemble(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def convdiff2d(N: int, bx: float, by: float) -> CSR:
    """Upwind convection-diffusion -Laplace(u) + beta . grad(u) on N x N
    interior nodes, unscaled (a nonsymmetric M-matrix).

    bx, by are the velocity components times the mesh width h. With first-order
    upwinding the row of node (x, y) is (4 + |bx| + |by|) u - (1 + max(bx, 0))
    u_west - (1 + max(-bx, 0)) u_east - (1 + max(by, 0)) u_south
    - (1 + max(-by, 0)) u_north; couplings to the Dirichlet boundary are
    dropped as for the Poisson matrix. bx = by = 0 gives poisson2d(N); the
    transpose of convdiff2d(N, bx, by) is convdiff2d(N, -bx, -by).
    """
    n = N * N
    idx = np.arange(n).reshape(N, N)
    rows = [np.arange(n)]
    cols = [np.arange(n)]
    vals = [np.full(n, 4.0 + abs(bx) + abs(by))]
    # (lower node, upper node, coefficient of the upper row on the lower node,
    #  coefficient of the lower row on the upper node)
    for lo, hi, c_up, c_dn in (
        (idx[:, :-1].ravel(), idx[:, 1:].ravel(), -1.0 - max(bx, 0.0), -1.0 - max(-bx, 0.0)),
        (idx[:-1, :].ravel(), idx[1:, :].ravel(), -1.0 - max(by, 0.0), -1.0 - max(-by, 0.0)),
    ):
        rows += [hi, lo]
        cols += [lo, hi]
        vals += [np.full(hi.size, c_up), np.full(lo.size, c_dn)]
    return _assemble(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def rhs_eigen_convdiff2d(N: int, bx: float, by: float):
    """Closed-form eigenvector right-hand side for convdiff2d(N, bx, by).

    The matrix is I (x) T_x + T_y (x) I with tridiagonal Toeplitz T = tridiag(s,
    d, t) per direction (s: coefficient on the lower neighbour, t: on the upper
    one, d = 2 + |b|). Its eigenvector of lowest frequency is v_j = (s/t)^(j/2)
    sin(j pi h), j = 1..N, h = 1/(N+1), with eigenvalue d - 2 sqrt(s t) cos(pi h).
    Returns (b, u, lam) with u the 2D product vector and b = lam u.
    """
    h = 1.0 / (N + 1)
    j = np.arange(1, N + 1)

    def mode(bd):
        s, t, d = -1.0 - max(bd, 0.0), -1.0 - max(-bd, 0.0), 2.0 + abs(bd)
        v = (s / t) ** (j / 2.0) * np.sin(j * np.pi * h)
        return v, d - 2.0 * np.sqrt(s * t) * np.cos(np.pi * h)

    vx, lx = mode(bx)
    vy, ly = mode(by)
    u = np.outer(vy, vx).ravel()
    lam = lx + ly
    return lam * u, u, lam


def grf_coefficient(N: int, seed: int, sigma: float = 1.0, ell: float = 1.0 / 32.0) -> np.ndarray:
    """k = exp(sigma * g) on the N x N interior nodes, g a unit Gaussian field.

    g has zero mean, unit variance and covariance exp(-r^2 / (2 ell^2)) in
    unit-square coordinates (node spacing h = 1/(N+1)). It is sampled by
    circulant embedding on a 2N x 2N periodic grid (FFT spectral method) and
    cropped to N x N. The complex white noise uses Box-Muller normals over
    SplitMix64(seed): real parts first, then imaginary parts.
    """
    M = 2 * N
    h = 1.0 / (N + 1)
    j = np.arange(M)
    d = np.minimum(j, M - j) * h
    r2 = d[:, None] ** 2 + d[None, :] ** 2
    c = np.exp(-r2 / (2.0 * ell * ell))
    lam = np.fft.fft2(c).real
    lam = np.maximum(lam, 0.0)
    z = normals(seed, 2 * M * M)
    xi = z[: M * M].reshape(M, M) + 1j * z[M * M:].reshape(M, M)
    w = np.fft.fft2(np.sqrt(lam / (M * M)) * xi)
    g = w.real[:N, :N]
    return np.exp(sigma * g)


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """b_i = 2u_i - 1, u_i uniform in [0,1) from SplitMix64(seed), index order."""
    return 2.0 * uniform01(seed, n) - 1.0


def rhs_eigen2d(N: int):
    """Eigenvector right-hand side for the 2D 5-point matrix.

    u_{x,y} = sin(pi (x+1) h) sin(pi (y+1) h), h = 1/(N+1), is an eigenvector
    with eigenvalue lam = 8 sin^2(pi h / 2); b = lam * u so that the exact
    discrete solution is u. Returns (b, u, lam).
    """
    h = 1.0 / (N + 1)
    s = np.sin(np.pi * (np.arange(N) + 1) * h)
    u = np.outer(s, s).ravel()
    lam = 8.0 * np.sin(np.pi * h / 2.0) ** 2
    return lam * u, u, lam


def rhs_eigen3d(N: int):
    """3D analogue of rhs_eigen2d: lam = 12 sin^2(pi h / 2)."""
    h = 1.0 / (N + 1)
    s = np.sin(np.pi * (np.arange(N) + 1) * h)
    u = (s[:, None, None] * s[None, :, None] * s[None, None, :]).ravel()
    lam = 12.0 * np.sin(np.pi * h / 2.0) ** 2
    return lam * u, u, lam
