"""CPU-side checks of the C-ABI library: it loads, exports every entry point
that include/ras.h declares, and its host-only parts (partitioners, input
validation) agree bit for bit with the oracle. No GPU work is issued."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2003_05361_gb300 as ras
import problems

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "ras.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(ras_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    lib = ras.load()
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name


def test_status_strings():
    for s in range(8):
        assert ras.ras_status_str(s)
    assert ras.ras_status_str(99) == "unknown status"


@pytest.mark.parametrize("nx,ny,px,py", [(128, 128, 2, 2), (1024, 1024, 16, 16), (10, 7, 3, 2),
                                         (33, 65, 1, 5)])
def test_regular2d_bit_exact(nx, ny, px, py):
    assert np.array_equal(ras.ras_partition_regular2d(nx, ny, px, py),
                          oracle.partition_regular2d(nx, ny, px, py))


@pytest.mark.parametrize("case", ["p2d_33", "p3d_20", "diff_40", "p2d_4"])
@pytest.mark.parametrize("P,seed", [(2, 7), (7, 1), (64, 3)])
def test_bfs_partition_bit_exact(case, P, seed):
    A = {"p2d_33": lambda: problems.poisson2d(33), "p3d_20": lambda: problems.poisson3d(20),
         "diff_40": lambda: problems.diffusion2d(40, problems.grf_coefficient(40, 4)),
         "p2d_4": lambda: problems.poisson2d(4)}[case]()
    if P > A.n:
        pytest.skip("more parts than vertices")
    assert np.array_equal(ras.ras_partition_bfs(A, P, seed), oracle.partition_bfs(A, P, seed))


def test_bfs_partition_config3_bit_exact():
    # 3D Poisson 128^3 into 512 parts with seed 3 (the batched-launch workload)
    A = problems.poisson3d(128)
    got = ras.ras_partition_bfs(A, 512, 3)
    want = oracle.partition_bfs(A, 512, 3)
    assert np.array_equal(got, want)
    sizes = np.bincount(got, minlength=512)
    # targets lie within +-30% of n/P; a part whose growth front is enclosed
    # stops early and the leftover sweeps enlarge its neighbours
    assert sizes.sum() == A.n and sizes.min() > 0.6 * A.n / 512
    assert sizes.max() < 2.0 * A.n / 512


def test_partition_invalid_arguments():
    with pytest.raises(ras.RasError) as e:
        ras.ras_partition_regular2d(4, 4, 5, 1)
    assert e.value.status == ras.RAS_EINVAL
    with pytest.raises(ras.RasError):
        ras.ras_partition_bfs(problems.poisson2d(3), 10, 0)


def _bad(A, **kw):
    d = dict(n=A.n, row_ptr=A.row_ptr.copy(), col=A.col.copy(), val=A.val.copy())
    d.update(kw)
    return problems.CSR(d["n"], d["row_ptr"], d["col"], d["val"])


@pytest.mark.parametrize("defect", ["unsorted", "range", "nodiag", "asym", "nan", "rowptr"])
def test_setup_rejects_invalid_matrix_before_gpu_work(defect):
    A = problems.poisson2d(4)
    if defect == "unsorted":
        col = A.col.copy()
        col[[1, 2]] = col[[2, 1]]
        B = _bad(A, col=col)
    elif defect == "range":
        col = A.col.copy()
        col[3] = 99
        B = _bad(A, col=col)
    elif defect == "nodiag":
        # drop row 0's diagonal entry
        keep = np.ones(A.nnz, bool)
        keep[0] = False
        rp = A.row_ptr.copy()
        rp[1:] -= 1
        B = _bad(A, row_ptr=rp, col=A.col[keep], val=A.val[keep])
    elif defect == "asym":
        # 1x... make (0,1) present but (1,0) absent: remove entry (1,0)
        r1 = A.row_ptr[1]
        keep = np.ones(A.nnz, bool)
        keep[r1] = False
        rp = A.row_ptr.copy()
        rp[2:] -= 1
        B = _bad(A, row_ptr=rp, col=A.col[keep], val=A.val[keep])
    elif defect == "nan":
        val = A.val.copy()
        val[5] = np.nan
        B = _bad(A, val=val)
    else:
        rp = A.row_ptr.copy()
        rp[-1] += 1
        B = _bad(A, row_ptr=rp)
    with pytest.raises(ras.RasError) as e:
        ras.ras_setup(B, np.zeros(16, np.int32), 1, 1)
    assert e.value.status == ras.RAS_EINVAL


@pytest.mark.parametrize("what", ["part_range", "empty_part", "overlap", "kind", "kind5", "bf16_cg",
                                  "bf16_gmres", "iters", "gmres_iters0", "gmres_iters33",
                                  "oras_nan", "oras_inf"])
def test_setup_rejects_invalid_options(what):
    A = problems.poisson2d(4)
    part = np.zeros(16, np.int32)
    P, ov, kind, prec, m, alpha = 1, 1, ras.RAS_LOCAL_BANDCHOL, ras.RAS_FP64, 20, 0.0
    if what == "part_range":
        part[3] = 2
        P = 2
    elif what == "empty_part":
        P = 2
    elif what == "overlap":
        ov = -1
    elif what == "kind":
        kind = 9
    elif what == "kind5":
        kind = 5
    elif what == "bf16_cg":
        kind, prec = ras.RAS_LOCAL_CG, ras.RAS_BF16_STORE
    elif what == "bf16_gmres":
        kind, prec = ras.RAS_LOCAL_GMRES, ras.RAS_BF16_STORE
    elif what == "gmres_iters0":
        kind, m = ras.RAS_LOCAL_GMRES, 0
    elif what == "gmres_iters33":
        kind, m = ras.RAS_LOCAL_GMRES, 33  # more Arnoldi steps than the kernel keeps
    elif what == "oras_nan":
        alpha = float("nan")
    elif what == "oras_inf":
        alpha = float("inf")
    else:
        kind, m = ras.RAS_LOCAL_CG, 0
    with pytest.raises(ras.RasError) as e:
        ras.ras_setup(A, part, P, ov, kind, prec, m, oras_alpha=alpha)
    assert e.value.status == ras.RAS_EINVAL


@pytest.mark.parametrize("kind,N", [(ras.RAS_LOCAL_BANDLU, 120), (ras.RAS_LOCAL_BANDCHOL, 170)])
def test_setup_rejects_too_wide_local_band_before_gpu_work(kind, N):
    # one subdomain of an N x N grid has local half-bandwidth N: above the
    # banded LU (112) or Cholesky (160) limit, setup stops with RAS_ENOTSUP
    A = problems.poisson2d(N)
    with pytest.raises(ras.RasError) as e:
        ras.ras_setup(A, np.zeros(A.n, np.int32), 1, 0, kind, ras.RAS_FP64)
    assert e.value.status == ras.RAS_ENOTSUP


def test_binding_structs_match_the_c_header(tmp_path):
    # the ctypes mirrors must have the C layout: compile a probe against
    # include/ras.h (host compiler only) and compare sizes and field offsets
    import ctypes as C
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    structs = [ras.ras_csr, ras.ras_local_solver, ras.ras_solve_info, ras.ras_tune_result]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ras.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(root, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                         text=True).stdout.split("\n") if l)
    for st in structs:
        name = st.__name__
        assert int(got[name]) == C.sizeof(st), name
        for f, _ in st._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(st, f).offset, f"{name}.{f}"
