"""CPU oracle for the RAS solver (ctypes binding over ras_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg. The product package never imports it, and it
never imports the product package.

The C library is compiled on demand with gcc (-O2 -ffp-contract=off
-fopenmp) into oracle/_build/.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ras_oracle.c")
_HDR = os.path.join(_HERE, "ras_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libras_oracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOTSPD, ENOCONV = 0, 1, 3, 4
BANDCHOL, CG, ILU0_CG, BANDLU, GMRES = 0, 1, 2, 3, 4
FP64, FP32, BF16 = 0, 1, 2

_I32P = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_F64P = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_U8P = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle shared library; returns its path."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)) or force or any(
            os.path.getmtime(s) > os.path.getmtime(_LIB_PATH) for s in (_SRC, _HDR)
        )
        if stale:
            os.makedirs(_OUT_DIR, exist_ok=True)
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                   "-fopenmp", "-o", tmp, _SRC, "-lm"]
            subprocess.run(cmd, check=True)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = C.CDLL(build())
    lib.or_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
    lib.or_splitmix64.restype = C.c_uint64
    lib.or_round_bf16.argtypes = [C.c_double]
    lib.or_round_bf16.restype = C.c_double
    lib.or_partition_regular2d.argtypes = [C.c_int] * 4 + [_I32P]
    lib.or_partition_bfs.argtypes = [C.c_int, _I32P, _I32P, C.c_int, C.c_uint64, _I32P]
    lib.or_overlap.argtypes = [C.c_int, _I32P, _I32P, _I32P, C.c_int, C.c_int, C.c_int,
                               _I32P, C.POINTER(C.c_int32), _U8P, _I32P, C.POINTER(C.c_int32)]
    lib.or_band_cholesky.argtypes = [C.c_int, C.c_int, _F64P]
    lib.or_band_solve.argtypes = [C.c_int, C.c_int, _F64P, _F64P]
    lib.or_band_solve.restype = None
    lib.or_band_solve_lowp.argtypes = [C.c_int, C.c_int, _F64P, C.c_int, _F64P]
    lib.or_band_solve_lowp.restype = None
    lib.or_band_lu.argtypes = [C.c_int, C.c_int, _F64P]
    lib.or_band_lu_solve.argtypes = [C.c_int, C.c_int, _F64P, _F64P]
    lib.or_band_lu_solve.restype = None
    lib.or_band_lu_solve_lowp.argtypes = [C.c_int, C.c_int, _F64P, C.c_int, _F64P]
    lib.or_band_lu_solve_lowp.restype = None
    lib.or_gmres.argtypes = [C.c_int, _I32P, _I32P, _F64P, _F64P, C.c_int, C.c_int, _F64P]
    lib.or_gmres.restype = None
    lib.or_dense_lu_solve.argtypes = [C.c_int, _F64P, _F64P]
    lib.or_cg.argtypes = [C.c_int, _I32P, _I32P, _F64P, _F64P, C.c_int, C.c_int, _F64P]
    lib.or_cg.restype = None
    lib.or_ilu0.argtypes = [C.c_int, _I32P, _I32P, _F64P, _F64P]
    lib.or_pcg_ilu0.argtypes = [C.c_int, _I32P, _I32P, _F64P, _F64P, _F64P, C.c_int, C.c_int,
                                _F64P]
    lib.or_pcg_ilu0.restype = None
    lib.or_residual.argtypes = [C.c_int, _I32P, _I32P, _F64P, _F64P, _F64P, C.c_void_p]
    lib.or_residual.restype = C.c_double
    lib.or_ras_sync_ex.argtypes = [C.c_int, _I32P, _I32P, _F64P, _F64P, _I32P, C.c_int, C.c_int,
                                   C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                   C.c_int, _F64P, C.c_void_p, C.POINTER(C.c_int32)]
    lib.or_ras_new.argtypes = [C.c_int, _I32P, _I32P, _F64P, _I32P, C.c_int, C.c_int, C.c_int,
                               C.c_int, C.c_int, C.c_double, C.POINTER(C.c_void_p)]
    lib.or_ras_iterate.argtypes = [C.c_void_p, _F64P, C.c_double, C.c_int, C.c_int, _F64P,
                                   C.c_void_p, C.POINTER(C.c_int32)]
    lib.or_ras_free.argtypes = [C.c_void_p]
    lib.or_ras_free.restype = None
    _lib = lib
    return lib


class OracleError(RuntimeError):
    pass


def _csr(A):
    return (np.ascontiguousarray(A.row_ptr, dtype=np.int32),
            np.ascontiguousarray(A.col, dtype=np.int32),
            np.ascontiguousarray(A.val, dtype=np.float64))


def splitmix64(seed: int, k: int) -> int:
    return int(_load().or_splitmix64(seed, k))


def round_bf16(v: float) -> float:
    return float(_load().or_round_bf16(v))


def partition_regular2d(nx: int, ny: int, px: int, py: int) -> np.ndarray:
    part = np.empty(nx * ny, dtype=np.int32)
    rc = _load().or_partition_regular2d(nx, ny, px, py, part)
    if rc:
        raise OracleError(f"partition_regular2d: {rc}")
    return part


def partition_bfs(A, P: int, seed: int) -> np.ndarray:
    rp, ci, _ = _csr(A)
    part = np.empty(A.n, dtype=np.int32)
    rc = _load().or_partition_bfs(A.n, rp, ci, P, seed, part)
    if rc:
        raise OracleError(f"partition_bfs: {rc}")
    return part


def overlap(A, part: np.ndarray, P: int, p: int, gamma: int):
    """Returns (omega, owned_mask, iface) for subdomain p."""
    rp, ci, _ = _csr(A)
    n = A.n
    omega = np.empty(n, dtype=np.int32)
    owned = np.empty(n, dtype=np.uint8)
    iface = np.empty(n, dtype=np.int32)
    no, ni = C.c_int32(0), C.c_int32(0)
    rc = _load().or_overlap(n, rp, ci, np.ascontiguousarray(part, dtype=np.int32), P, p, gamma,
                            omega, C.byref(no), owned, iface, C.byref(ni))
    if rc:
        raise OracleError(f"overlap: {rc}")
    return omega[: no.value].copy(), owned[: no.value].copy(), iface[: ni.value].copy()


def band_cholesky(band: np.ndarray, w: int) -> np.ndarray:
    """band: (n, w+1) array with band[i, t] = A[i, i-w+t]. Returns L in the same layout."""
    L = np.ascontiguousarray(band, dtype=np.float64).copy()
    rc = _load().or_band_cholesky(L.shape[0], w, L.reshape(-1))
    if rc:
        raise OracleError(f"band_cholesky: {rc}")
    return L


def band_solve(L: np.ndarray, w: int, rhs: np.ndarray, prec: int = FP64) -> np.ndarray:
    x = np.ascontiguousarray(rhs, dtype=np.float64).copy()
    Lc = np.ascontiguousarray(L, dtype=np.float64).reshape(-1)
    if prec == FP64:
        _load().or_band_solve(L.shape[0], w, Lc, x)
    else:
        _load().or_band_solve_lowp(L.shape[0], w, Lc, prec, x)
    return x


def band_lu(band: np.ndarray, w: int) -> np.ndarray:
    """band: (n, 2w+1) array with band[i, t] = A[i, i-w+t]. Returns the LU factors
    in the same layout (unit lower L below the diagonal, U on and above it)."""
    F = np.ascontiguousarray(band, dtype=np.float64).copy()
    rc = _load().or_band_lu(F.shape[0], w, F.reshape(-1))
    if rc:
        raise OracleError(f"band_lu: {rc}")
    return F


def band_lu_solve(F: np.ndarray, w: int, rhs: np.ndarray, prec: int = FP64) -> np.ndarray:
    x = np.ascontiguousarray(rhs, dtype=np.float64).copy()
    Fc = np.ascontiguousarray(F, dtype=np.float64).reshape(-1)
    if prec == FP64:
        _load().or_band_lu_solve(F.shape[0], w, Fc, x)
    else:
        _load().or_band_lu_solve_lowp(F.shape[0], w, Fc, prec, x)
    return x


def gmres(A, rhs: np.ndarray, m: int, prec: int = FP64) -> np.ndarray:
    rp, ci, val = _csr(A)
    d = np.empty(A.n)
    _load().or_gmres(A.n, rp, ci, val, np.ascontiguousarray(rhs, dtype=np.float64), m, prec, d)
    return d


def dense_lu_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    M = np.ascontiguousarray(A, dtype=np.float64).copy()
    x = np.ascontiguousarray(b, dtype=np.float64).copy()
    rc = _load().or_dense_lu_solve(M.shape[0], M.reshape(-1), x)
    if rc:
        raise OracleError(f"dense_lu_solve: {rc}")
    return x


def cg(A, rhs: np.ndarray, m: int, prec: int = FP64) -> np.ndarray:
    rp, ci, val = _csr(A)
    d = np.empty(A.n)
    _load().or_cg(A.n, rp, ci, val, np.ascontiguousarray(rhs, dtype=np.float64), m, prec, d)
    return d


def ilu0(A) -> np.ndarray:
    rp, ci, val = _csr(A)
    lu = np.empty_like(val)
    rc = _load().or_ilu0(A.n, rp, ci, val, lu)
    if rc:
        raise OracleError(f"ilu0: {rc}")
    return lu


def pcg_ilu0(A, lu: np.ndarray, rhs: np.ndarray, m: int, prec: int = FP64) -> np.ndarray:
    rp, ci, val = _csr(A)
    d = np.empty(A.n)
    _load().or_pcg_ilu0(A.n, rp, ci, val, np.ascontiguousarray(lu, dtype=np.float64),
                        np.ascontiguousarray(rhs, dtype=np.float64), m, prec, d)
    return d


def residual(A, b: np.ndarray, x: np.ndarray):
    """Returns (r, ||r||_2) with r = b - A x."""
    rp, ci, val = _csr(A)
    r = np.empty(A.n)
    r2 = _load().or_residual(A.n, rp, ci, val, np.ascontiguousarray(b, dtype=np.float64),
                             np.ascontiguousarray(x, dtype=np.float64), r.ctypes.data)
    return r, float(np.sqrt(r2))


def ras_sync(A, b, part, P: int, gamma: int, kind: int = BANDCHOL, prec: int = FP64,
             m: int = 20, tol: float = 1e-8, max_iter: int = 100000, nthreads: int = 1,
             x0=None, allow_noconv: bool = False, oras_alpha: float = 0.0):
    """Synchronous RAS (optimized local matrices when oras_alpha != 0).
    Returns (x, iterations, relres_history)."""
    rp, ci, val = _csr(A)
    x = np.zeros(A.n) if x0 is None else np.ascontiguousarray(x0, dtype=np.float64).copy()
    hist = np.zeros(max_iter + 1)
    it = C.c_int32(0)
    rc = _load().or_ras_sync_ex(A.n, rp, ci, val, np.ascontiguousarray(b, dtype=np.float64),
                                np.ascontiguousarray(part, dtype=np.int32), P, gamma, kind, prec,
                                m, oras_alpha, tol, max_iter, nthreads, x, hist.ctypes.data,
                                C.byref(it))
    if rc and not (rc == ENOCONV and allow_noconv):
        raise OracleError(f"ras_sync: {rc}")
    k = it.value
    return x, k, hist[: k + 1].copy()


class RasSetup:
    """Synchronous RAS split as Algorithm 1 splits it: the constructor does the
    set-up (overlap maps, local matrices, factorisations; untimed in Sec. 3.1),
    iterate() runs RAS iterations from x with the same arithmetic as
    ras_sync(). setup_s is the wall time of the set-up."""

    def __init__(self, A, part, P: int, gamma: int, kind: int = BANDCHOL, prec: int = FP64,
                 m: int = 20, oras_alpha: float = 0.0):
        import time

        self._arrays = _csr(A)  # the C handle points into these
        self._part = np.ascontiguousarray(part, dtype=np.int32)
        self.n = A.n
        h = C.c_void_p()
        t0 = time.perf_counter()
        rp, ci, val = self._arrays
        rc = _load().or_ras_new(A.n, rp, ci, val, self._part, P, gamma, kind, prec, m,
                                oras_alpha, C.byref(h))
        self.setup_s = time.perf_counter() - t0
        if rc:
            raise OracleError(f"ras setup: {rc}")
        self._h = h

    def iterate(self, b, x, tol: float = 0.0, max_iter: int = 1, nthreads: int = 1,
                allow_noconv: bool = True):
        """Runs at most max_iter iterations from x (updated in place, float64
        C-contiguous). Returns (iterations, relres_history)."""
        assert x.dtype == np.float64 and x.flags["C_CONTIGUOUS"] and x.size == self.n
        hist = np.zeros(max_iter + 1)
        it = C.c_int32(0)
        rc = _load().or_ras_iterate(self._h, np.ascontiguousarray(b, dtype=np.float64), tol,
                                    max_iter, nthreads, x, hist.ctypes.data, C.byref(it))
        if rc and not (rc == ENOCONV and allow_noconv):
            raise OracleError(f"ras iterate: {rc}")
        return it.value, hist[: it.value + 1].copy()

    def close(self):
        if self._h:
            _load().or_ras_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


from .direct import (  # noqa: E402,F401
    band_direct_solve,
    poisson2d_direct,
    poisson3d_direct,
)
