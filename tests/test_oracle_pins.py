"""Pins for the oracle's building blocks, each against something other than
the oracle itself: library routines (numpy/scipy/networkx), closed forms,
hand-worked fixtures and brute force on tiny inputs."""
from collections import deque

import networkx as nx
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import oracle
import problems


def dense(A):
    return A.to_scipy().toarray()


# ---------------------------------------------------------------- generators

def test_splitmix64_published_vector(golden):
    want = [int(v, 16) for v in golden("splitmix64_seed0.txt")]
    assert [oracle.splitmix64(0, k) for k in range(3)] == want


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-8, 8, 20000),
                        [1.0, -1.0, 1.00390625, 1.01171875, 3.0e-30]])
    # torch rounds float32 -> bf16 with ties to even; feed values exact in fp32
    v32 = v.astype(np.float32).astype(np.float64)
    want = torch.tensor(v32, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.round_bf16(x) for x in v32])
    assert np.array_equal(got, want)
    # ties: 1 + 2^-8 sits halfway between 1 and 1 + 2^-7 -> even (1.0)
    assert oracle.round_bf16(1.0 + 2.0 ** -8) == 1.0
    assert oracle.round_bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2 * 2.0 ** -7


# ---------------------------------------------------------------- partitions

@pytest.mark.parametrize("nx_,ny_,px,py", [(8, 8, 2, 2), (10, 7, 3, 2), (16, 16, 1, 4), (5, 5, 5, 5)])
def test_regular2d_blocks(nx_, ny_, px, py):
    part = oracle.partition_regular2d(nx_, ny_, px, py).reshape(ny_, nx_)
    assert set(np.unique(part)) == set(range(px * py))
    # each part is one axis-aligned rectangle; widths differ by at most one
    widths, heights = set(), set()
    for p in range(px * py):
        ys, xs = np.nonzero(part == p)
        h, w = ys.max() - ys.min() + 1, xs.max() - xs.min() + 1
        assert h * w == ys.size
        widths.add(w)
        heights.add(h)
        # numbering: block row major
        assert p == (p // px) * px + (p % px)
    assert max(widths) - min(widths) <= 1 and max(heights) - min(heights) <= 1
    # block ids increase along x then y
    assert np.all(np.diff(part, axis=1) >= 0) and np.all(np.diff(part, axis=0) >= 0)


def bfs_partition_reference(A, P, seed):
    """Second, independent implementation of the BFS-growth partitioner."""
    n = A.n
    nbrs = [list(A.col[A.row_ptr[i]:A.row_ptr[i + 1]]) for i in range(n)]
    u = problems.uniform01(seed, 2 * P)
    w = [1.0 + 0.3 * (2.0 * u[p] - 1.0) for p in range(P)]
    W = 0.0
    for p in range(P):
        W += w[p]
    target = [int(np.floor(float(n) * w[p] / W)) for p in range(P)]
    rem = n - sum(target)
    p = 0
    while rem > 0:
        target[p] += 1
        rem -= 1
        p = (p + 1) % P
    p = 0
    while rem < 0:
        if target[p] > 0:
            target[p] -= 1
            rem += 1
        p = (p + 1) % P
    part = [-1] * n
    size = [0] * P
    queues = [deque() for _ in range(P)]
    pos = [0] * n
    for p in range(P):
        v = min(int(np.floor(u[P + p] * n)), n - 1)
        while part[v] != -1:
            v = (v + 1) % n
        part[v] = p
        size[p] = 1
        queues[p].append(v)
    while True:
        claimed = False
        for p in range(P):
            if size[p] >= target[p]:
                continue
            q = queues[p]
            while q:
                f = q[0]
                hit = None
                while pos[f] < len(nbrs[f]):
                    j = nbrs[f][pos[f]]
                    pos[f] += 1
                    if part[j] == -1:
                        hit = j
                        break
                if hit is None:
                    q.popleft()
                    continue
                part[hit] = p
                size[p] += 1
                q.append(hit)
                claimed = True
                break
        if not claimed:
            break
    while -1 in part:
        changed = True
        while changed:
            changed = False
            for i in range(n):
                if part[i] != -1:
                    continue
                cands = sorted({part[j] for j in nbrs[i] if part[j] >= 0}, key=lambda q: (size[q], q))
                if cands:
                    part[i] = cands[0]
                    size[cands[0]] += 1
                    changed = True
        if -1 in part:
            i0 = part.index(-1)
            q = min(range(P), key=lambda q: (size[q], q))
            part[i0] = q
            size[q] += 1
    return np.array(part, dtype=np.int32)


def test_bfs_partition_hand_worked(golden):
    want = np.array([[int(t) for t in r.split()] for r in golden("bfs_partition_4x4_P2_seed7.txt")])
    got = oracle.partition_bfs(problems.poisson2d(4), 2, 7).reshape(4, 4)
    assert np.array_equal(got, want)


def _disconnected_graph():
    # two grids side by side with no coupling: exercises the leftover rule
    A = problems.poisson2d(4)
    S = dense(A)
    import scipy.sparse as sp
    B = sp.csr_matrix(sp.block_diag([sp.csr_matrix(S), sp.csr_matrix(S), sp.csr_matrix(np.array([[2.0]]))]))
    B.sort_indices()
    return problems.CSR(B.shape[0], B.indptr.astype(np.int32), B.indices.astype(np.int32), B.data)


@pytest.mark.parametrize("graph,P,seed", [("g6", 3, 1), ("g10", 7, 3), ("g3d", 8, 3),
                                          ("g10", 1, 0), ("disc", 2, 5), ("g6", 36, 2)])
def test_bfs_partition_matches_independent(graph, P, seed):
    A = {"g6": problems.poisson2d(6), "g10": problems.poisson2d(10),
         "g3d": problems.poisson3d(6), "disc": _disconnected_graph()}[graph]
    got = oracle.partition_bfs(A, P, seed)
    want = bfs_partition_reference(A, P, seed)
    assert np.array_equal(got, want)
    assert got.min() >= 0 and got.max() < P
    assert np.bincount(got, minlength=P).sum() == A.n


def test_bfs_partition_balance_3d():
    A = problems.poisson3d(16)
    P = 32
    part = oracle.partition_bfs(A, P, 3)
    sizes = np.bincount(part, minlength=P)
    assert sizes.min() > 0
    # targets are within +-30% of n/P; growth can leave a part short but
    # leftovers are few on a connected grid
    assert sizes.max() <= 1.3 * A.n / P * 1.15


# ---------------------------------------------------------------- overlap

def _grid_graph(A):
    G = nx.Graph()
    G.add_nodes_from(range(A.n))
    for i in range(A.n):
        for c in A.col[A.row_ptr[i]:A.row_ptr[i + 1]]:
            if c != i:
                G.add_edge(i, int(c))
    return G


@pytest.mark.parametrize("case", ["2d6", "2d5_bfs", "3d5"])
@pytest.mark.parametrize("gamma", [0, 1, 2, 4])
def test_overlap_brute_force(case, gamma):
    if case == "2d6":
        A, P = problems.poisson2d(6), 4
        part = oracle.partition_regular2d(6, 6, 2, 2)
    elif case == "2d5_bfs":
        A, P = problems.poisson2d(5), 3
        part = oracle.partition_bfs(A, P, 11)
    else:
        A, P = problems.poisson3d(5), 4
        part = oracle.partition_bfs(A, P, 2)
    G = _grid_graph(A)
    dist_all = dict(nx.all_pairs_shortest_path_length(G))
    for p in range(P):
        om, owned, iface = oracle.overlap(A, part, P, p, gamma)
        Op = np.nonzero(part == p)[0]
        d = np.array([min(dist_all[i][j] for j in Op) for i in range(A.n)])
        assert np.array_equal(om, np.nonzero(d <= gamma)[0])
        assert np.array_equal(owned.astype(bool), part[om] == p)
        assert np.array_equal(iface, np.nonzero(d == gamma + 1)[0])


def test_overlap_manhattan_closed_form():
    # regular 2D blocks on the 5-point grid: graph distance = L1 distance to
    # the block, so Omega_p = {dx + dy <= gamma} (corners trimmed)
    N, px, py, gamma = 12, 3, 2, 3
    A = problems.poisson2d(N)
    part = oracle.partition_regular2d(N, N, px, py)
    ys, xs = np.divmod(np.arange(N * N), N)
    for p in range(px * py):
        m = part == p
        x0, x1, y0, y1 = xs[m].min(), xs[m].max(), ys[m].min(), ys[m].max()
        dx = np.maximum(0, np.maximum(x0 - xs, xs - x1))
        dy = np.maximum(0, np.maximum(y0 - ys, ys - y1))
        om, _, iface = oracle.overlap(A, part, px * py, p, gamma)
        assert np.array_equal(om, np.nonzero(dx + dy <= gamma)[0])
        assert np.array_equal(iface, np.nonzero(dx + dy == gamma + 1)[0])


def test_overlap_union_and_sizes():
    # config-1 geometry: 128^2, 2x2, gamma 2. A corner block grows on two
    # sides only: 64^2 + 2 * (2 * 64) + 1 point with dx = dy = 1
    N = 128
    A = problems.poisson2d(N)
    part = oracle.partition_regular2d(N, N, 2, 2)
    cover = np.zeros(A.n, int)
    for p in range(4):
        om, owned, _ = oracle.overlap(A, part, 4, p, 2)
        assert om.size == 64 * 64 + 2 * (2 * 64) + 1
        cover[om[owned.astype(bool)]] += 1
    assert np.all(cover == 1)


# ---------------------------------------------------------------- direct solvers

def _band_of(S, w):
    n = S.shape[0]
    band = np.zeros((n, w + 1))
    for i in range(n):
        for j in range(max(0, i - w), i + 1):
            band[i, j - i + w] = S[i, j]
    return band


def _unband(L, w):
    n = L.shape[0]
    M = np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - w), i + 1):
            M[i, j] = L[i, j - i + w]
    return M


@pytest.mark.parametrize("N", [3, 6, 10])
def test_band_cholesky_vs_numpy(N):
    A = problems.diffusion2d(N, problems.grf_coefficient(N, 9))
    S = dense(A)
    L = oracle.band_cholesky(_band_of(S, N), N)
    Ld = _unband(L, N)
    assert np.linalg.norm(Ld @ Ld.T - S) <= 1e-14 * np.linalg.norm(S) * 10
    assert np.allclose(Ld, np.linalg.cholesky(S), rtol=1e-12, atol=1e-13)
    rhs = problems.rhs_uniform(A.n, 2)
    x = oracle.band_solve(L, N, rhs)
    xs = np.linalg.solve(S, rhs)
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)


def test_band_cholesky_not_spd():
    S = np.array([[1.0, 2.0], [2.0, 1.0]])
    with pytest.raises(oracle.OracleError):
        oracle.band_cholesky(_band_of(S, 1), 1)


@pytest.mark.parametrize("prec,eps", [(oracle.FP32, 2.0 ** -24), (oracle.BF16, 2.0 ** -9)])
def test_band_solve_low_precision_error_bound(prec, eps):
    N = 12
    A = problems.poisson2d(N)
    S = dense(A)
    L = oracle.band_cholesky(_band_of(S, N), N)
    rhs = problems.rhs_uniform(A.n, 3)
    x = oracle.band_solve(L, N, rhs, prec)
    xs = np.linalg.solve(S, rhs)
    kappa = np.linalg.cond(S)
    err = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    # backward-stable substitution with perturbed factors: err = O(kappa n eps)
    assert err <= 4 * kappa * (N + 1) * eps
    assert err >= 1e-2 * eps  # really computed in reduced precision
    if prec == oracle.FP32:
        # fp32 arithmetic throughout: reproduce with numpy float32 substitution
        Lf = L.astype(np.float32)
        y = rhs.astype(np.float32)
        n, w = A.n, N
        for i in range(n):
            s = y[i]
            for k in range(max(0, i - w), i):
                s = np.float32(s - np.float32(Lf[i, k - i + w] * y[k]))
            y[i] = np.float32(s / Lf[i, w])
        for i in range(n - 1, -1, -1):
            s = y[i]
            for k in range(i + 1, min(n - 1, i + w) + 1):
                s = np.float32(s - np.float32(Lf[k, i - k + w] * y[k]))
            y[i] = np.float32(s / Lf[i, w])
        assert np.array_equal(x, y.astype(np.float64))


def _gband_of(S, w):
    n = S.shape[0]
    band = np.zeros((n, 2 * w + 1))
    for i in range(n):
        for j in range(max(0, i - w), min(n, i + w + 1)):
            band[i, j - i + w] = S[i, j]
    return band


def _gunband(F, w):
    """(unit lower L, upper U) from the banded LU factors."""
    n = F.shape[0]
    L, U = np.eye(n), np.zeros((n, n))
    for i in range(n):
        for j in range(max(0, i - w), min(n, i + w + 1)):
            if j < i:
                L[i, j] = F[i, j - i + w]
            else:
                U[i, j] = F[i, j - i + w]
    return L, U


@pytest.mark.parametrize("N,bx,by", [(3, 0.5, 0.5), (6, 1.5, -0.7), (10, -3.0, 2.0)])
def test_band_lu_vs_scipy(N, bx, by):
    # the convection-diffusion matrix is column diagonally dominant, so
    # Gaussian elimination with partial pivoting swaps no rows (Golub & Van
    # Loan, Thm. 3.4.3) and scipy's P L U has P = I with the same L and U
    import scipy.linalg as sl

    A = problems.convdiff2d(N, bx, by)
    S = dense(A)
    F = oracle.band_lu(_gband_of(S, N), N)
    L, U = _gunband(F, N)
    Pm, L2, U2 = sl.lu(S)
    assert np.array_equal(Pm, np.eye(A.n))
    assert np.allclose(L, L2, rtol=1e-12, atol=1e-14) and np.allclose(U, U2, rtol=1e-12, atol=1e-13)
    assert np.linalg.norm(L @ U - S) <= 1e-14 * np.linalg.norm(S) * 10
    rhs = problems.rhs_uniform(A.n, 5)
    x = oracle.band_lu_solve(F, N, rhs)
    xs = np.linalg.solve(S, rhs)
    assert np.linalg.norm(x - xs) <= 1e-12 * np.linalg.norm(xs)


def test_band_lu_of_spd_matches_cholesky():
    # for SPD A: L_lu = L_c diag(L_c)^-1 and U = diag(L_c) L_c^T
    N = 7
    A = problems.diffusion2d(N, problems.grf_coefficient(N, 3))
    S = dense(A)
    L, U = _gunband(oracle.band_lu(_gband_of(S, N), N), N)
    Lc = np.linalg.cholesky(S)
    Dc = np.diag(np.diag(Lc))
    assert np.allclose(L, Lc @ np.linalg.inv(Dc), rtol=1e-12, atol=1e-14)
    assert np.allclose(U, Dc @ Lc.T, rtol=1e-12, atol=1e-13)


def test_band_lu_zero_pivot():
    S = np.array([[0.0, 1.0], [1.0, 0.0]])
    with pytest.raises(oracle.OracleError):
        oracle.band_lu(_gband_of(S, 1), 1)
    # a zero pivot that appears only after elimination
    S = np.array([[1.0, 1.0, 0.0], [1.0, 1.0, 1.0], [0.0, 1.0, 1.0]])
    with pytest.raises(oracle.OracleError):
        oracle.band_lu(_gband_of(S, 1), 1)


@pytest.mark.parametrize("prec,eps", [(oracle.FP32, 2.0 ** -24), (oracle.BF16, 2.0 ** -9)])
def test_band_lu_solve_low_precision_error_bound(prec, eps):
    N = 12
    A = problems.convdiff2d(N, 0.8, -0.4)
    S = dense(A)
    F = oracle.band_lu(_gband_of(S, N), N)
    rhs = problems.rhs_uniform(A.n, 6)
    x = oracle.band_lu_solve(F, N, rhs, prec)
    xs = np.linalg.solve(S, rhs)
    kappa = np.linalg.cond(S)
    err = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    assert err <= 4 * kappa * (N + 1) * eps
    assert err >= 1e-2 * eps  # really computed in reduced precision
    if prec == oracle.FP32:
        # float32 substitutions with the factors rounded to float32
        Ff = F.astype(np.float32)
        y = rhs.astype(np.float32)
        n, w = A.n, N
        for i in range(n):
            acc = y[i]
            for k in range(max(0, i - w), i):
                acc = np.float32(acc - np.float32(Ff[i, k - i + w] * y[k]))
            y[i] = acc
        for i in range(n - 1, -1, -1):
            acc = y[i]
            for k in range(i + 1, min(n - 1, i + w) + 1):
                acc = np.float32(acc - np.float32(Ff[i, k - i + w] * y[k]))
            y[i] = np.float32(acc / Ff[i, w])
        assert np.array_equal(x, y.astype(np.float64))


# ---------------------------------------------------------------- GMRES

def _krylov_lsq(S, r, m):
    """Brute force: the d in K_m(S, r) minimising ||r - S d||, by an
    orthonormal basis of the Krylov matrix (numpy QR) and least squares."""
    K = np.empty((r.size, m))
    v = r.copy()
    for j in range(m):
        K[:, j] = v / np.linalg.norm(v)
        v = S @ K[:, j]
    Q, _ = np.linalg.qr(K)
    c, *_ = np.linalg.lstsq(S @ Q, r, rcond=None)
    return Q @ c


@pytest.mark.parametrize("m", [1, 2, 4, 6])
def test_gmres_is_krylov_least_squares(m):
    A = problems.convdiff2d(7, 1.3, -0.6)
    S = dense(A)
    r = problems.rhs_uniform(A.n, 8)
    d = oracle.gmres(A, r, m)
    dk = _krylov_lsq(S, r, m)
    assert np.linalg.norm(d - dk) <= 1e-10 * np.linalg.norm(dk)
    if m == 1:
        # one step: d = (r.Ar / |Ar|^2) r
        Ar = S @ r
        assert np.allclose(d, (r @ Ar) / (Ar @ Ar) * r, rtol=1e-13, atol=0)


def test_gmres_full_space_is_direct_solve():
    A = problems.convdiff2d(6, -0.9, 0.4)
    S = dense(A)
    r = problems.rhs_uniform(A.n, 9)
    xs = np.linalg.solve(S, r)
    for m in (A.n, A.n + 10):  # more steps than unknowns: the same n steps
        d = oracle.gmres(A, r, m)
        assert np.linalg.norm(d - xs) <= 1e-11 * np.linalg.norm(xs)


def test_gmres_residual_monotone_and_below_cg_on_spd():
    A = problems.convdiff2d(12, 0.7, 0.2)
    S = dense(A)
    r = problems.rhs_uniform(A.n, 10)
    res = [np.linalg.norm(r - S @ oracle.gmres(A, r, m)) for m in range(1, 25)]
    assert all(b <= a * (1 + 1e-12) for a, b in zip(res, res[1:]))
    assert res[-1] < 1e-2 * np.linalg.norm(r)
    # SPD: GMRES minimises the residual 2-norm over the same Krylov space as CG
    P2 = problems.poisson2d(12)
    S2 = dense(P2)
    for m in (3, 8, 15):
        rg = np.linalg.norm(r - S2 @ oracle.gmres(P2, r, m))
        rc = np.linalg.norm(r - S2 @ oracle.cg(P2, r, m))
        assert rg <= rc * (1 + 1e-10)


def test_gmres_exact_breakdown_and_zero_rhs():
    # diagonal A, rhs = e_2: A v_1 is parallel to v_1, h_21 = 0 exactly
    n = 5
    rp = np.arange(n + 1, dtype=np.int32)
    ci = np.arange(n, dtype=np.int32)
    D = problems.CSR(n, rp, ci, np.array([2.0, 3.0, 5.0, 7.0, 11.0]))
    r = np.zeros(n)
    r[2] = 4.0
    for prec in (oracle.FP64, oracle.FP32):
        d = oracle.gmres(D, r, 20, prec)
        assert np.array_equal(d, np.array([0.0, 0.0, 0.8, 0.0, 0.0], dtype=np.float32).astype(np.float64)
                              if prec == oracle.FP32 else np.array([0.0, 0.0, 0.8, 0.0, 0.0]))
    assert np.array_equal(oracle.gmres(D, np.zeros(n), 5), np.zeros(n))


def _gmres_float32(A, r, m):
    """GMRES in numpy float32 scalars, one operation at a time in the oracle's
    order (MGS, Givens, back substitution): every float32 operation is
    correctly rounded, so this is plain FP32 arithmetic."""
    f = np.float32
    n = A.n
    val = A.val.astype(f)
    rr = r.astype(f)
    b2 = f(0)
    for i in range(n):
        b2 = f(b2 + f(rr[i] * rr[i]))
    beta = f(np.sqrt(b2))
    m = min(m, n)
    V = [np.array([f(rr[i] / beta) for i in range(n)], dtype=f)]
    H = np.zeros((m + 1, m), dtype=f)
    cs, sn, g = np.zeros(m, f), np.zeros(m, f), np.zeros(m + 1, f)
    g[0] = beta
    k = 0
    for j in range(m):
        vj = V[j]
        w = np.zeros(n, f)
        for i in range(n):
            s = f(0)
            for e in range(A.row_ptr[i], A.row_ptr[i + 1]):
                s = f(s + f(val[e] * vj[A.col[e]]))
            w[i] = s
        for q in range(j + 1):
            h = f(0)
            for i in range(n):
                h = f(h + f(w[i] * V[q][i]))
            H[q, j] = h
            for i in range(n):
                w[i] = f(w[i] - f(h * V[q][i]))
        hn2 = f(0)
        for i in range(n):
            hn2 = f(hn2 + f(w[i] * w[i]))
        hn = f(np.sqrt(hn2))
        H[j + 1, j] = hn
        for q in range(j):
            a, b = H[q, j], H[q + 1, j]
            H[q, j] = f(f(cs[q] * a) + f(sn[q] * b))
            H[q + 1, j] = f(f(cs[q] * b) - f(sn[q] * a))
        a = H[j, j]
        den = f(np.sqrt(f(f(a * a) + f(hn * hn))))
        cs[j], sn[j] = f(a / den), f(hn / den)
        H[j, j], H[j + 1, j] = den, f(0)
        g[j + 1] = -f(sn[j] * g[j])
        g[j] = f(cs[j] * g[j])
        k = j + 1
        if hn == 0:
            break
        V.append(np.array([f(w[i] / hn) for i in range(n)], dtype=f))
    y = np.zeros(k, f)
    for q in range(k - 1, -1, -1):
        s = g[q]
        for t in range(q + 1, k):
            s = f(s - f(H[q, t] * y[t]))
        y[q] = f(s / H[q, q])
    d = np.zeros(n, f)
    for i in range(n):
        s = f(0)
        for q in range(k):
            s = f(s + f(y[q] * V[q][i]))
        d[i] = s
    return d.astype(np.float64)


def test_gmres_fp32_mode_is_float32_arithmetic():
    # the oracle computes in double and rounds each result to float; for
    # + - * / and sqrt of floats that is the correctly rounded float result,
    # so it must equal plain float32 arithmetic bit for bit
    A = problems.convdiff2d(5, 0.9, -0.4)
    r = problems.rhs_uniform(A.n, 13)
    for m in (1, 3, 7):
        assert np.array_equal(oracle.gmres(A, r, m, oracle.FP32), _gmres_float32(A, r, m)), m


def test_gmres_fp32_within_rounding():
    A = problems.convdiff2d(16, 0.5, 0.5)
    r = problems.rhs_uniform(A.n, 11)
    d64 = oracle.gmres(A, r, 20)
    d32 = oracle.gmres(A, r, 20, oracle.FP32)
    err = np.linalg.norm(d32 - d64) / np.linalg.norm(d64)
    assert 1e-9 < err < 1e-4  # really FP32, and only its rounding


def test_dense_lu_vs_numpy():
    rng = np.random.default_rng(1)
    M = rng.standard_normal((40, 40))
    b = rng.standard_normal(40)
    x = oracle.dense_lu_solve(M, b)
    assert np.allclose(x, np.linalg.solve(M, b), rtol=1e-10, atol=1e-12)
    # needs pivoting: zero leading entry
    M2 = np.array([[0.0, 1.0], [1.0, 0.0]])
    assert np.allclose(oracle.dense_lu_solve(M2, np.array([2.0, 3.0])), [3.0, 2.0])


# ---------------------------------------------------------------- iterative local solvers

def test_cg_one_step_closed_form():
    A = problems.poisson2d(5)
    r = problems.rhs_uniform(A.n, 4)
    S = dense(A)
    d = oracle.cg(A, r, 1)
    alpha = (r @ r) / (r @ S @ r)
    assert np.allclose(d, alpha * r, rtol=1e-14, atol=0)


def test_cg_finite_termination():
    A = problems.poisson2d(4)  # n = 16, at most 16 distinct eigenvalues
    r = problems.rhs_uniform(A.n, 5)
    d = oracle.cg(A, r, A.n)
    assert np.linalg.norm(d - np.linalg.solve(dense(A), r)) <= 1e-10 * np.linalg.norm(d)


@pytest.mark.parametrize("m", [3, 10, 20])
def test_cg_vs_scipy(m):
    N = 10
    A = problems.diffusion2d(N, problems.grf_coefficient(N, 3))
    r = problems.rhs_uniform(A.n, 6)
    d = oracle.cg(A, r, m)
    ds, _ = spla.cg(A.to_scipy(), r, x0=np.zeros(A.n), rtol=0.0, atol=0.0, maxiter=m)
    assert np.linalg.norm(d - ds) <= 1e-10 * np.linalg.norm(ds)
    d32 = oracle.cg(A, r, m, oracle.FP32)
    assert np.linalg.norm(d32 - ds) <= 1e-4 * np.linalg.norm(ds)
    assert not np.array_equal(d32, d)


def test_ilu0_pattern_property():
    # ILU(0) reproduces A exactly on A's sparsity pattern: (L U)_ij = a_ij
    N = 6
    A = problems.diffusion2d(N, problems.grf_coefficient(N, 1))
    lu = oracle.ilu0(A)
    n = A.n
    L = np.eye(n)
    U = np.zeros((n, n))
    for i in range(n):
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = A.col[k]
            if j < i:
                L[i, j] = lu[k]
            else:
                U[i, j] = lu[k]
    LU = L @ U
    S = dense(A)
    mask = S != 0
    assert np.allclose(LU[mask], S[mask], rtol=1e-13, atol=1e-13)
    # fill outside the pattern is dropped, and it is non-zero for a 2D grid
    assert np.abs(LU[~mask]).max() > 1e-3


def test_ilu0_tridiagonal_is_exact_lu():
    import scipy.sparse as sp
    n = 12
    T = sp.diags([-1.0, 2.5, -1.0], [-1, 0, 1], shape=(n, n)).tocsr()
    T.sort_indices()
    A = problems.CSR(n, T.indptr.astype(np.int32), T.indices.astype(np.int32), T.data)
    lu = oracle.ilu0(A)
    rhs = problems.rhs_uniform(n, 1)
    # one PCG step with an exact preconditioner solves the system
    d = oracle.pcg_ilu0(A, lu, rhs, 1)
    assert np.allclose(d, np.linalg.solve(T.toarray(), rhs), rtol=1e-12)


@pytest.mark.parametrize("m", [1, 5, 12])
def test_pcg_vs_scipy(m):
    N = 9
    A = problems.poisson2d(N)
    lu = oracle.ilu0(A)
    n = A.n
    import scipy.sparse as sp
    Lsp = sp.lil_matrix((n, n))
    Usp = sp.lil_matrix((n, n))
    for i in range(n):
        Lsp[i, i] = 1.0
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            j = A.col[k]
            (Lsp if j < i else Usp)[i, j] = lu[k]
    Lsp, Usp = Lsp.tocsr(), Usp.tocsr()

    def msolve(v):
        y = spla.spsolve_triangular(Lsp, v, lower=True)
        return spla.spsolve_triangular(Usp, y, lower=False)

    M = spla.LinearOperator((n, n), matvec=msolve)
    rhs = problems.rhs_uniform(n, 8)
    d = oracle.pcg_ilu0(A, lu, rhs, m)
    ds, _ = spla.cg(A.to_scipy(), rhs, x0=np.zeros(n), rtol=0.0, atol=0.0, maxiter=m, M=M)
    assert np.linalg.norm(d - ds) <= 1e-10 * np.linalg.norm(ds)


def test_residual_vs_scipy():
    A = problems.poisson3d(5)
    b = problems.rhs_uniform(A.n, 1)
    x = problems.rhs_uniform(A.n, 2)
    r, rn = oracle.residual(A, b, x)
    rs = b - A.to_scipy() @ x
    assert np.allclose(r, rs, rtol=0, atol=1e-14)
    assert abs(rn - np.linalg.norm(rs)) <= 1e-13 * rn


# ---------------------------------------------------------------- FP32 local solvers, bit for bit

def _f32_spmv(A, vals32, p):
    f = np.float32
    q = np.zeros(A.n, f)
    for i in range(A.n):
        s = f(0)
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            s = f(s + f(vals32[k] * p[A.col[k]]))
        q[i] = s
    return q


def _f32_dot(a, b):
    f = np.float32
    s = f(0)
    for i in range(a.size):
        s = f(s + f(a[i] * b[i]))
    return s


def _cg_float32(A, rhs, m):
    """Textbook CG (q = A p; alpha = rr/(p.q); d += alpha p; r -= alpha q;
    beta = rr'/rr; p = r + beta p) in float32 arithmetic with A rounded to
    float32, sums taken in index order."""
    f = np.float32
    v32 = A.val.astype(f)
    r = rhs.astype(f)
    p = r.copy()
    d = np.zeros(A.n, f)
    rr = _f32_dot(r, r)
    for _ in range(m):
        if rr == f(0):
            break
        q = _f32_spmv(A, v32, p)
        alpha = f(rr / _f32_dot(p, q))
        d = (d + alpha * p).astype(f)
        r = (r - alpha * q).astype(f)
        rr2 = _f32_dot(r, r)
        beta = f(rr2 / rr)
        p = (r + beta * p).astype(f)
        rr = rr2
    return d.astype(np.float64)


def _ilu_apply_float32(A, lu32, r):
    """z = U^{-1} L^{-1} r (L unit lower, U upper from the ILU(0) factors)."""
    f = np.float32
    n = A.n
    z = np.zeros(n, f)
    for i in range(n):
        s = r[i]
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            if A.col[k] >= i:
                break
            s = f(s - f(lu32[k] * z[A.col[k]]))
        z[i] = s
    for i in range(n - 1, -1, -1):
        s, dg = z[i], f(0)
        for k in range(A.row_ptr[i], A.row_ptr[i + 1]):
            c = A.col[k]
            if c > i:
                s = f(s - f(lu32[k] * z[c]))
            elif c == i:
                dg = lu32[k]
        z[i] = f(s / dg)
    return z


def _pcg_ilu0_float32(A, lu, rhs, m):
    """ILU(0)-preconditioned CG (z = M^{-1} r; p = z; alpha = rz/(p.Ap);
    d += alpha p; r -= alpha Ap; z = M^{-1} r; beta = rz'/rz; p = z + beta p)
    in float32 arithmetic with A and the factors rounded to float32."""
    f = np.float32
    v32 = A.val.astype(f)
    lu32 = lu.astype(f)
    r = rhs.astype(f)
    d = np.zeros(A.n, f)
    z = _ilu_apply_float32(A, lu32, r)
    p = z.copy()
    rz = _f32_dot(r, z)
    for _ in range(m):
        if rz == f(0):
            break
        q = _f32_spmv(A, v32, p)
        alpha = f(rz / _f32_dot(p, q))
        d = (d + alpha * p).astype(f)
        r = (r - alpha * q).astype(f)
        z = _ilu_apply_float32(A, lu32, r)
        rz2 = _f32_dot(r, z)
        beta = f(rz2 / rz)
        p = (z + beta * p).astype(f)
        rz = rz2
    return d.astype(np.float64)


@pytest.mark.parametrize("m", [1, 3, 7])
def test_cg_fp32_mode_is_float32_arithmetic(m):
    # the oracle's FP32 CG equals plain float32 arithmetic bit for bit, and
    # differs from its FP64 CG (it really rounds)
    N = 7
    A = problems.diffusion2d(N, problems.grf_coefficient(N, 5))
    r = problems.rhs_uniform(A.n, 21)
    d32 = oracle.cg(A, r, m, oracle.FP32)
    assert np.array_equal(d32, _cg_float32(A, r, m))
    assert not np.array_equal(d32, oracle.cg(A, r, m))


@pytest.mark.parametrize("m", [1, 3, 6])
def test_pcg_ilu0_fp32_mode_is_float32_arithmetic(m):
    # the FP32 branch of the ILU(0)-PCG (factors rounded to float32, both
    # triangular sweeps and every CG operation in float32) equals plain
    # float32 arithmetic bit for bit
    N = 6
    A = problems.diffusion2d(N, problems.grf_coefficient(N, 3))
    r = problems.rhs_uniform(A.n, 17)
    lu = oracle.ilu0(A)
    d32 = oracle.pcg_ilu0(A, lu, r, m, oracle.FP32)
    assert np.array_equal(d32, _pcg_ilu0_float32(A, lu, r, m))
    d64 = oracle.pcg_ilu0(A, lu, r, m)
    err = np.linalg.norm(d32 - d64) / np.linalg.norm(d64)
    assert 1e-10 < err < 1e-5


def test_pcg_ilu0_fp32_3d_pattern():
    # the 7-point pattern of config 3's local solver
    A = problems.poisson3d(4)
    r = problems.rhs_uniform(A.n, 23)
    lu = oracle.ilu0(A)
    for m in (2, 5):
        assert np.array_equal(oracle.pcg_ilu0(A, lu, r, m, oracle.FP32),
                              _pcg_ilu0_float32(A, lu, r, m))
