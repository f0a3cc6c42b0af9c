"""Failure paths of the CUDA library, exercised in the forms that leave the GPU
healthy: a device-side time limit that runs out (the kernel records
RAS_ETIMEOUT and returns; no trap, no hang), a local factorisation that breaks
down on an indefinite matrix (RAS_ENOTSPD from the GPU Cholesky), and
allocation failures injected on the host (RAS_FAULT_ALLOC: the k-th
allocation of a ras_setup call reports out-of-memory without allocating).
After each failure the same process must go on solving correctly."""
import numpy as np
import pytest

import oracle
import paper_2003_05361_gb300 as ras
import problems

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _solve(ctx, A, b, tol, mode, max_updates=0):
    bd = torch.tensor(b, device="cuda")
    x = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    try:
        info = ras.ras_solve(ctx, bd, x, tol, mode, max_updates)
    except ras.RasError as err:
        return None, err
    torch.cuda.synchronize()
    return x.cpu().numpy(), info


@pytest.mark.parametrize("mode", [ras.RAS_SYNC, ras.RAS_ASYNC])
def test_whole_solve_time_limit_ends_with_etimeout(mode, monkeypatch):
    # the benchmark problem with FP64 local CG-20 takes seconds; a 5 ms limit
    # on the whole solve makes every CTA stop at its next check (site 4)
    N = 1024
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 1)
    part = ras.ras_partition_regular2d(N, N, 16, 16)
    ctx = ras.ras_setup(A, part, 256, 4, ras.RAS_LOCAL_CG, ras.RAS_FP64, 20)
    monkeypatch.setenv("RAS_SOLVE_LIMIT_MS", "5")
    _, err = _solve(ctx, A, b, 1e-8, mode)
    assert isinstance(err, ras.RasError) and err.status == ras.RAS_ETIMEOUT
    assert err.info is not None and err.info.error_site == 4
    assert err.info.kernel_ms < 2000.0  # it stopped early, not at convergence
    monkeypatch.delenv("RAS_SOLVE_LIMIT_MS")
    # the context and the device stay usable: a capped synchronous solve gives
    # the oracle's iterate
    x, info = _solve(ctx, A, b, 1e-8, ras.RAS_SYNC, 2)
    assert info.status == ras.RAS_ENOCONV and info.iterations == 2
    xo = oracle.ras_sync(A, b, part, 256, 4, oracle.CG, oracle.FP64, 20, tol=0.0, max_iter=2,
                         nthreads=8, allow_noconv=True)[0]
    assert np.abs(x - xo).max() <= 1e-9 * np.abs(xo).max()
    ras.ras_destroy(ctx)


def test_gpu_cholesky_indefinite_local_block_enotspd():
    # a 2D grid operator with diagonal 1 and off-diagonal -1 is indefinite, and
    # so are its local blocks: the GPU banded Cholesky meets a non-positive
    # pivot and setup returns RAS_ENOTSPD (no context is created)
    N = 12
    A = problems.poisson2d(N)
    rows = np.repeat(np.arange(A.n), np.diff(A.row_ptr))
    val = np.where(A.col == rows, 1.0, A.val)
    B = problems.CSR(A.n, A.row_ptr, A.col, val)
    part = ras.ras_partition_regular2d(N, N, 2, 2)
    for prec in (ras.RAS_FP64, ras.RAS_FP32):
        with pytest.raises(ras.RasError) as ei:
            ras.ras_setup(B, part, 4, 1, ras.RAS_LOCAL_BANDCHOL, prec)
        assert ei.value.status == ras.RAS_ENOTSPD
    # a valid system on the same device afterwards
    b = problems.rhs_uniform(A.n, 2)
    ctx = ras.ras_setup(A, part, 4, 1, ras.RAS_LOCAL_BANDCHOL, ras.RAS_FP64)
    x, info = _solve(ctx, A, b, 1e-8, ras.RAS_SYNC)
    assert info.status == 0
    _, rn = oracle.residual(A, b, x)
    assert rn < 1e-8 * np.linalg.norm(b)
    ras.ras_destroy(ctx)


@pytest.mark.parametrize("kind,prec", [(ras.RAS_LOCAL_BANDCHOL, ras.RAS_FP32),
                                       (ras.RAS_LOCAL_CG, ras.RAS_FP32),
                                       (ras.RAS_LOCAL_ILU0_CG, ras.RAS_FP32)])
def test_injected_allocation_failures_return_enomem(kind, prec, monkeypatch):
    # every allocation of ras_setup fails in turn: each must give RAS_ENOMEM,
    # leave no context and leak no device memory
    N = 48
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 3)
    part = ras.ras_partition_regular2d(N, N, 2, 2)
    ras.ras_destroy(ras.ras_setup(A, part, 4, 2, kind, prec, 8))  # warm the context
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(1, 400):
        monkeypatch.setenv("RAS_FAULT_ALLOC", str(k))
        try:
            ctx = ras.ras_setup(A, part, 4, 2, kind, prec, 8)
        except ras.RasError as err:
            assert err.status == ras.RAS_ENOMEM, (k, err.status)
            failures += 1
            continue
        ras.ras_destroy(ctx)  # k is past the last allocation
        break
    else:
        pytest.fail("setup never completed")
    monkeypatch.delenv("RAS_FAULT_ALLOC")
    assert failures >= 10
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 16 << 20
    ctx = ras.ras_setup(A, part, 4, 2, kind, prec, 8)
    x, info = _solve(ctx, A, b, 1e-8, ras.RAS_SYNC)
    assert info.status == 0
    _, rn = oracle.residual(A, b, x)
    assert rn < 1e-8 * np.linalg.norm(b)
    ras.ras_destroy(ctx)
