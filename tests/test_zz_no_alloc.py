"""GPU test of ras_relres_noalloc, the entry point for callers that cannot
allocate device memory (graph capture, fixed memory pools, allocation-free
loops). It must agree with ras_relres, the context-based entry point, and with
the oracle's FP64 residual, on calls in a row. The shared scratch array keeps
the previous call's contents, so a call with fewer row chunks right after one
with many checks that no stale partial sum is read. The test passes both in a
fresh process and after the rest of the suite; this file is collected last on
purpose."""
import numpy as np
import pytest

import oracle
import paper_2003_05361_gb300 as ras
import problems

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA GPU")]


def _device_csr(A):
    dev = torch.device("cuda")
    return (torch.tensor(A.row_ptr, dtype=torch.int32, device=dev),
            torch.tensor(A.col, dtype=torch.int32, device=dev),
            torch.tensor(A.val, dtype=torch.float64, device=dev))


def _check_calls(N, px, cases):
    A = problems.poisson2d(N)
    part = ras.ras_partition_regular2d(N, N, px, px)
    ctx = ras.ras_setup(A, part, px * px, 1, ras.RAS_LOCAL_CG, ras.RAS_FP64, 2)
    rp, ci, va = _device_csr(A)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for seed, scale in cases:
        bh = problems.rhs_uniform(A.n, seed)
        xh = problems.rhs_uniform(A.n, seed + 10) * scale
        b = torch.tensor(bh, device="cuda")
        x = torch.tensor(xh, device="cuda")
        ras.ras_relres_noalloc(rp, ci, va, b, x, out)
        torch.cuda.synchronize()
        got = float(out.item())
        want = ras.ras_relres(ctx, b, x)
        _, rn = oracle.residual(A, bh, xh)
        want_o = rn / np.linalg.norm(bh)
        assert np.isfinite(got)
        assert abs(got - want) <= 1e-12 * want
        assert abs(got - want_o) <= 1e-12 * want_o
    ras.ras_destroy(ctx)


@pytest.mark.parametrize("N,px", [(128, 2), (700, 10)])
def test_relres_noalloc_matches_ras_relres(N, px):
    # two calls in a row with different vectors (the second a smaller residual)
    _check_calls(N, px, ((1, 1.0), (2, 1e-6)))


def test_relres_noalloc_fewer_chunks_after_more():
    # 700^2 rows fill 479 chunks of the scratch; the 128^2 call right after it
    # uses 16, so any read of a partial it did not write would show
    _check_calls(700, 10, ((3, 1.0),))
    _check_calls(128, 2, ((4, 1e-3), (5, 1.0)))


def test_relres_noalloc_rejects_oversize_and_null():
    lib = ras.load()
    assert lib.ras_relres_noalloc(67108865, 8, 8, 8, 8, 8, 8, None) == ras.RAS_EINVAL
    assert lib.ras_relres_noalloc(0, 8, 8, 8, 8, 8, 8, None) == ras.RAS_EINVAL
    assert lib.ras_relres_noalloc(10, None, 8, 8, 8, 8, 8, None) == ras.RAS_EINVAL
