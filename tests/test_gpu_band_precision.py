"""Banded-Cholesky local solves with factors stored in FP32 and BF16 (the
mixed-precision pattern: factorised in FP64, rounded for storage, applied in
FP32 arithmetic; residual, update and convergence test in FP64) against the
oracle, which emulates the same rounding of the factors with FP32
substitutions (Sec. 3.3.1 local solution, correction form of Sec. 2.1).

The GPU applies each 32-row block through a precomputed inverse diagonal
block, so its rounding differs from the oracle's substitutions: both sit
within the storage rounding of the FP64 iterate, and the bar is element-wise:
max |x_gpu - x_oracle,p| <= 4 max |x_oracle,p - x_oracle,FP64| (+ a floor of
1e-7 max |x|), with the oracle's own gap non-zero (it really rounds) and at
most the storage precision's unit roundoff times a growth factor. Converged
results are compared with the oracle's FP64 direct solve of the whole system.
"""
import numpy as np
import pytest

import oracle
import paper_2003_05361_gb300 as ras
import problems

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]

BAND = ras.RAS_LOCAL_BANDCHOL
PRECS = {ras.RAS_FP32: (oracle.FP32, 2.0 ** -24), ras.RAS_BF16_STORE: (oracle.BF16, 2.0 ** -9)}


def gpu_iterate(ctx, A, b, mode, tol=1e-8, max_updates=0):
    bd = torch.tensor(b, device="cuda")
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    info = ras.ras_solve(ctx, bd, x, tol, mode, max_updates)
    torch.cuda.synchronize()
    return x.cpu().numpy(), info


def emax(a, b):
    return float(np.abs(a - b).max())


def check_lowprec_iterates(A, b, part, P, gamma, ks, oracle_threads=1):
    for prec, (oprec, u) in PRECS.items():
        ctx = ras.ras_setup(A, part, P, gamma, BAND, prec)
        h64 = oracle.RasSetup(A, part, P, gamma, oracle.BANDCHOL, oracle.FP64)
        hlo = oracle.RasSetup(A, part, P, gamma, oracle.BANDCHOL, oprec)
        x64, xlo = np.zeros(A.n), np.zeros(A.n)
        done = 0
        for k in ks:
            h64.iterate(b, x64, max_iter=k - done, nthreads=oracle_threads)
            hlo.iterate(b, xlo, max_iter=k - done, nthreads=oracle_threads)
            done = k
            x, info = gpu_iterate(ctx, A, b, ras.RAS_SYNC, max_updates=k)
            assert info.iterations == k
            scale = float(np.abs(x64).max())
            gap = emax(xlo, x64)
            assert 0.0 < gap <= 1e3 * u * scale, (prec, k, gap / scale)
            assert emax(x, xlo) <= 4.0 * gap + 1e-7 * scale, (prec, k, emax(x, xlo) / gap)
        ras.ras_destroy(ctx)
        h64.close()
        hlo.close()


def test_band_fp32_bf16_iterates_ragged_grid():
    # 45^2 Poisson (45 = 15 * 3 columns, rows split 23 / 22): several 32-row
    # blocks per subdomain and a partial last block
    NX = 45
    A = problems.poisson2d(NX)
    b = problems.rhs_uniform(A.n, 31)
    part = ras.ras_partition_regular2d(NX, NX, 3, 2)
    check_lowprec_iterates(A, b, part, 6, 2, (1, 3))


def test_band_fp32_bf16_iterates_config4_geometry():
    # the config-4 subdomain shape: variable-coefficient diffusion (k = exp of
    # the seeded Gaussian field, sigma 1, ell 1/32), 64 x 64 blocks (4 x 4 on a
    # 256^2 grid), overlap 4: n_p up to 72^2 = 5184 rows, local half-bandwidth
    # 72, 162 chain steps per triangular solve
    N = 256
    A = problems.diffusion2d(N, problems.grf_coefficient(N, 4))
    b = problems.rhs_uniform(A.n, 4)
    part = ras.ras_partition_regular2d(N, N, 4, 4)
    ctx = ras.ras_setup(A, part, 16, 4, BAND, ras.RAS_FP64)
    assert ras.ras_get_info(ctx)["max_bandwidth"] == 72
    # FP64 factors: the same iterates as the oracle's up to summation order
    h = oracle.RasSetup(A, part, 16, 4, oracle.BANDCHOL, oracle.FP64)
    xo = np.zeros(A.n)
    h.iterate(b, xo, max_iter=2, nthreads=8)
    x, info = gpu_iterate(ctx, A, b, ras.RAS_SYNC, max_updates=2)
    assert emax(x, xo) <= 1e-12 * np.abs(xo).max()
    h.close()
    ras.ras_destroy(ctx)
    check_lowprec_iterates(A, b, part, 16, 4, (1, 3), oracle_threads=8)


def test_band_precisions_converge_to_oracle_direct_solution():
    # config-4 recipe at 256^2: every storage precision, sync and async, reaches
    # the FP64 fixed point; at relres 1e-10 (the tolerance at which the 1e-6
    # error bar is met on this ill-conditioned matrix) the error against the
    # oracle's banded Cholesky of the whole system is at most 1e-6
    N = 256
    A = problems.diffusion2d(N, problems.grf_coefficient(N, 4))
    b = problems.rhs_uniform(A.n, 4)
    part = ras.ras_partition_regular2d(N, N, 4, 4)
    xs = oracle.band_direct_solve(A, b)
    for prec in (ras.RAS_FP64, ras.RAS_FP32, ras.RAS_BF16_STORE):
        ctx = ras.ras_setup(A, part, 16, 4, BAND, prec)
        for mode in (ras.RAS_SYNC, ras.RAS_ASYNC):
            x, info = gpu_iterate(ctx, A, b, mode, tol=1e-10)
            assert info.status == 0, info.as_dict()
            _, rn = oracle.residual(A, b, x)
            assert rn < 1e-10 * np.linalg.norm(b)
            assert np.linalg.norm(x - xs) <= 1e-6 * np.linalg.norm(xs), (prec, mode)
        ras.ras_destroy(ctx)
