"""GPU test of ras_relres_noalloc, the entry point for callers that cannot
allocate device memory (graph capture, fixed memory pools, allocation-free
loops). It must agree with ras_relres, the context-based entry point, on two
calls in a row (the shared scratch array keeps the first call's contents, so
the second call checks that nothing stale leaks), both in a fresh process and
after the rest of the suite. This file is collected last on purpose."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("N,px", [(128, 2), (700, 10)])
def test_relres_noalloc_matches_ras_relres(N, px):
    A = problems.poisson2d(N)
    part = ras.ras_partition_regular2d(N, N, px, px)
    ctx = ras.ras_setup(A, part, px * px, 1, ras.RAS_LOCAL_CG, ras.RAS_FP64, 2)
    rp, ci, va = _device_csr(A)
    out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    # two calls in a row with different vectors (the second one a smaller residual)
    for seed, scale in ((1, 1.0), (2, 1e-6)):
        b = torch.tensor(problems.rhs_uniform(A.n, seed), device="cuda")
        x = torch.tensor(problems.rhs_uniform(A.n, seed + 10), device="cuda") * scale
        ras.ras_relres_noalloc(rp, ci, va, b, x, out)
        torch.cuda.synchronize()
        got = float(out.item())
        want = ras.ras_relres(ctx, b, x)
        assert np.isfinite(got)
        assert abs(got - want) <= 1e-12 * want
    ras.ras_destroy(ctx)


def test_relres_noalloc_rejects_oversize_and_null():
    lib = ras.load()
    assert lib.ras_relres_noalloc(67108865, 8, 8, 8, 8, 8, 8, None) == ras.RAS_EINVAL
    assert lib.ras_relres_noalloc(0, 8, 8, 8, 8, 8, 8, None) == ras.RAS_EINVAL
    assert lib.ras_relres_noalloc(10, None, 8, 8, 8, 8, 8, None) == ras.RAS_EINVAL
