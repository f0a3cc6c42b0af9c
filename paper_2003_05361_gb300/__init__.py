"""Python binding of the GB300 asynchronous RAS solver (libras.so).

Argument marshalling only: every entry point forwards to the C ABI of
include/ras.h with the same name; all computation runs in the library's CUDA
kernels. Device vectors are torch CUDA tensors (float64, contiguous) or raw
device pointers (int). Host matrices are anything with n / row_ptr / col /
val attributes (e.g. problems.CSR) or a scipy CSR matrix.

The library is built in-tree (paper_2003_05361_gb300/_build/libras.so) by
build.py; loading fails loudly if it cannot be built or loaded.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

RAS_OK, RAS_EINVAL, RAS_ENOMEM, RAS_ENOTSPD, RAS_ENOCONV, RAS_ETIMEOUT, RAS_ECUDA, RAS_ENOTSUP = range(8)
RAS_SYNC, RAS_ASYNC, RAS_ASYNC_DECENTRAL = 0, 1, 2
RAS_LOCAL_BANDCHOL, RAS_LOCAL_CG, RAS_LOCAL_ILU0_CG, RAS_LOCAL_BANDLU, RAS_LOCAL_GMRES = 0, 1, 2, 3, 4
RAS_FP64, RAS_FP32, RAS_BF16_STORE = 0, 1, 2

_lock = threading.Lock()
_lib = None


class ras_csr(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("row_ptr", C.POINTER(C.c_int32)),
                ("col_idx", C.POINTER(C.c_int32)), ("val", C.POINTER(C.c_double))]


class ras_local_solver(C.Structure):
    _fields_ = [("kind", C.c_int32), ("prec", C.c_int32), ("inner_iters", C.c_int32),
                ("reserved_", C.c_int32), ("oras_alpha", C.c_double)]


class ras_solve_info(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("updates_min", C.c_int64),
                ("updates_median", C.c_int64), ("updates_max", C.c_int64),
                ("relres", C.c_double), ("solve_ms", C.c_double), ("restarts", C.c_int32),
                ("status", C.c_int32), ("kernel_ms", C.c_double), ("stale_updates", C.c_int64),
                ("error_site", C.c_int32), ("grid", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ras_tune_result(C.Structure):
    _fields_ = [("cta_threads", C.c_int32), ("staged", C.c_int32), ("inner_iters", C.c_int32),
                ("candidates", C.c_int32), ("score", C.c_double), ("schedule", C.c_int32),
                ("grid", C.c_int32), ("per_cta", C.c_int32), ("reserved_", C.c_int32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class RasError(RuntimeError):
    def __init__(self, status: int, where: str, info=None):
        super().__init__(f"{where}: {ras_status_str(status)} (status {status})")
        self.status = status
        self.info = info  # ras_solve_info of a failed solve, when there is one


def lib_path() -> str:
    return _build.LIB


def load():
    """Builds (if stale) and loads libras.so; raises if either fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = C.CDLL(path)
        P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "ras_status_str": ([C.c_int], C.c_char_p),
            "ras_partition_regular2d": ([I32, I32, I32, I32, P], C.c_int),
            "ras_partition_bfs": ([C.POINTER(ras_csr), I32, C.c_uint64, P], C.c_int),
            "ras_setup": ([C.POINTER(ras_csr), P, I32, I32, C.POINTER(ras_local_solver), P,
                           C.POINTER(P)], C.c_int),
            "ras_solve": ([P, P, P, D, I32, I64, C.POINTER(ras_solve_info)], C.c_int),
            "ras_solve_host": ([P, P, P, D, I32, I64, C.POINTER(ras_solve_info)], C.c_int),
            "ras_solve_batch": ([P, I32, P, P, D, I32, I64, P], C.c_int),
            "ras_destroy": ([P], C.c_int),
            "ras_get_maps": ([P, I32, C.POINTER(P), C.POINTER(I32), C.POINTER(P), C.POINTER(P),
                              C.POINTER(I32)], C.c_int),
            "ras_get_info": ([P, C.POINTER(I32), C.POINTER(I32), C.POINTER(I32), C.POINTER(I64)],
                             C.c_int),
            "ras_get_update_counts": ([P, P], C.c_int),
            "ras_relres": ([P, P, P, C.POINTER(D)], C.c_int),
            "ras_relres_noalloc": ([I32, P, P, P, P, P, P, P], C.c_int),
            "ras_solve_begin": ([P, P, P, D], C.c_int),
            "ras_get_phase_times": ([P, P], C.c_int),
            "ras_get_launch": ([P, C.POINTER(I32), C.POINTER(I32), C.POINTER(I32), C.POINTER(I32)],
                               C.c_int),
            "ras_autotune": ([P, P, I32, I32, I32, C.POINTER(ras_tune_result)], C.c_int),
            "ras_batch_step": ([P, I32, I32, I64, I64, P, P], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def ras_status_str(status: int) -> str:
    return load().ras_status_str(int(status)).decode()


def _check(status: int, where: str, allow=()):
    if status != RAS_OK and status not in allow:
        raise RasError(status, where)
    return status


class _HostCSR:
    """Keeps the numpy arrays alive while the C struct points at them."""

    def __init__(self, A):
        if hasattr(A, "indptr"):  # scipy
            n, rp, ci, va = A.shape[0], A.indptr, A.indices, A.data
        else:
            n, rp, ci, va = A.n, A.row_ptr, A.col, A.val
        self.rp = np.ascontiguousarray(rp, dtype=np.int32)
        self.ci = np.ascontiguousarray(ci, dtype=np.int32)
        self.va = np.ascontiguousarray(va, dtype=np.float64)
        self.s = ras_csr(int(n), int(self.rp[-1]), self.rp.ctypes.data_as(C.POINTER(C.c_int32)),
                         self.ci.ctypes.data_as(C.POINTER(C.c_int32)),
                         self.va.ctypes.data_as(C.POINTER(C.c_double)))


def _dptr(t, n=None, what="vector"):
    """Device pointer of a float64 CUDA tensor (or a raw int pointer)."""
    if isinstance(t, int):
        return t
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{what} must be a contiguous float64 CUDA tensor")
    if n is not None and t.numel() != n:
        raise ValueError(f"{what} has {t.numel()} entries, expected {n}")
    return t.data_ptr()


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


def ras_partition_regular2d(nx: int, ny: int, px: int, py: int) -> np.ndarray:
    part = np.empty(nx * ny, dtype=np.int32)
    _check(load().ras_partition_regular2d(nx, ny, px, py, part.ctypes.data), "ras_partition_regular2d")
    return part


def ras_partition_bfs(A, num_parts: int, seed: int) -> np.ndarray:
    h = _HostCSR(A)
    part = np.empty(h.s.n, dtype=np.int32)
    _check(load().ras_partition_bfs(C.byref(h.s), num_parts, seed, part.ctypes.data), "ras_partition_bfs")
    return part


class RasContext:
    """Owns a ras_ctx pointer (freed by ras_destroy or on garbage collection)."""

    def __init__(self, ptr: int, n: int, num_parts: int):
        self.ptr = ptr
        self.n = n
        self.num_parts = num_parts

    def __del__(self):
        try:
            ras_destroy(self)
        except Exception:
            pass


def ras_setup(A, partition, num_parts: int, overlap: int, kind: int = RAS_LOCAL_BANDCHOL,
              prec: int = RAS_FP64, inner_iters: int = 20, stream=None,
              oras_alpha: float = 0.0) -> RasContext:
    h = _HostCSR(A)
    part = np.ascontiguousarray(partition, dtype=np.int32)
    if part.size != h.s.n:
        raise ValueError("partition must have one entry per row")
    ls = ras_local_solver(kind, prec, inner_iters, 0, oras_alpha)
    out = C.c_void_p()
    _check(load().ras_setup(C.byref(h.s), part.ctypes.data, num_parts, overlap, C.byref(ls),
                            _stream_handle(stream), C.byref(out)), "ras_setup")
    return RasContext(out.value, h.s.n, num_parts)


def ras_solve(ctx: RasContext, b, x, tol: float = 1e-8, mode: int = RAS_SYNC,
              max_updates: int = 0) -> ras_solve_info:
    """Solves A x = b on the device; x holds x0 on entry. Raises RasError on
    failure except RAS_ENOCONV, which is reported in info.status."""
    info = ras_solve_info()
    st = load().ras_solve(ctx.ptr, _dptr(b, ctx.n, "b"), _dptr(x, ctx.n, "x"), tol, mode,
                          max_updates, C.byref(info))
    if st not in (RAS_OK, RAS_ENOCONV):
        raise RasError(st, "ras_solve", info)
    return info


def ras_solve_host(ctx: RasContext, b: np.ndarray, x: np.ndarray, tol: float = 1e-8,
                   mode: int = RAS_SYNC, max_updates: int = 0) -> ras_solve_info:
    """Same as ras_solve with host float64 arrays (pinned memory is fastest)."""
    if isinstance(b, np.ndarray):
        assert b.dtype == np.float64 and b.flags.c_contiguous and b.size == ctx.n
        assert x.dtype == np.float64 and x.flags.c_contiguous and x.size == ctx.n
        pb, px = b.ctypes.data, x.ctypes.data
    else:  # pinned torch CPU tensors
        pb, px = b.data_ptr(), x.data_ptr()
    info = ras_solve_info()
    _check(load().ras_solve_host(ctx.ptr, pb, px, tol, mode, max_updates, C.byref(info)),
           "ras_solve_host", allow=(RAS_ENOCONV,))
    return info


def ras_solve_batch(ctxs, bs, xs, tol: float = 1e-8, mode: int = RAS_SYNC, max_updates: int = 0):
    num = len(ctxs)
    cp = (C.c_void_p * num)(*[c.ptr for c in ctxs])
    bp = (C.c_void_p * num)(*[_dptr(b, c.n, "b") for b, c in zip(bs, ctxs)])
    xp = (C.c_void_p * num)(*[_dptr(x, c.n, "x") for x, c in zip(xs, ctxs)])
    infos = (ras_solve_info * num)()
    _check(load().ras_solve_batch(cp, num, bp, xp, tol, mode, max_updates, infos),
           "ras_solve_batch", allow=(RAS_ENOCONV,))
    return list(infos)


def ras_autotune(ctx: RasContext, x_scratch, mode: int = RAS_SYNC, iters: int = 20,
                 tune_inner: bool = True) -> ras_tune_result:
    """Times candidate launch shapes / inner step counts and keeps the best."""
    out = ras_tune_result()
    _check(load().ras_autotune(ctx.ptr, _dptr(x_scratch, ctx.n, "x"), mode, iters,
                               1 if tune_inner else 0, C.byref(out)), "ras_autotune")
    return out


def ras_solve_begin(ctx: RasContext, b, x, tol: float = 1e-8) -> None:
    """Starts a solve (continuous batching); advance it with ras_batch_step."""
    _check(load().ras_solve_begin(ctx.ptr, _dptr(b, ctx.n, "b"), _dptr(x, ctx.n, "x"), tol),
           "ras_solve_begin")


def ras_batch_step(ctxs, mode: int = RAS_ASYNC, step_limit: int = 50, max_updates: int = 0):
    """One batched step over the begun contexts; returns (done flags, infos)."""
    num = len(ctxs)
    cp = (C.c_void_p * num)(*[c.ptr for c in ctxs])
    done = np.zeros(num, dtype=np.int32)
    infos = (ras_solve_info * num)()
    _check(load().ras_batch_step(cp, num, mode, step_limit, max_updates, done.ctypes.data, infos),
           "ras_batch_step", allow=(RAS_ENOCONV,))
    return done.astype(bool), list(infos)


def ras_destroy(ctx: RasContext) -> None:
    if ctx is not None and ctx.ptr:
        p, ctx.ptr = ctx.ptr, None
        _check(load().ras_destroy(p), "ras_destroy")


def ras_get_maps(ctx: RasContext, p: int):
    """Returns numpy copies (omega, owned_mask, iface) of subdomain p."""
    om, ow, ifc = C.c_void_p(), C.c_void_p(), C.c_void_p()
    no, ni = C.c_int32(), C.c_int32()
    _check(load().ras_get_maps(ctx.ptr, p, C.byref(om), C.byref(no), C.byref(ow), C.byref(ifc),
                               C.byref(ni)), "ras_get_maps")

    def arr(ptr, n, ct, dt):
        if n == 0:
            return np.zeros(0, dtype=dt)
        return np.ctypeslib.as_array(C.cast(ptr, C.POINTER(ct)), shape=(n,)).astype(dt).copy()

    return (arr(om, no.value, C.c_int32, np.int32), arr(ow, no.value, C.c_uint8, np.uint8),
            arr(ifc, ni.value, C.c_int32, np.int32))


def ras_get_info(ctx: RasContext) -> dict:
    P, n, w = C.c_int32(), C.c_int32(), C.c_int32()
    b = C.c_int64()
    _check(load().ras_get_info(ctx.ptr, C.byref(P), C.byref(n), C.byref(w), C.byref(b)), "ras_get_info")
    return {"num_parts": P.value, "n": n.value, "max_bandwidth": w.value, "device_bytes": b.value}


def ras_get_update_counts(ctx: RasContext) -> np.ndarray:
    out = np.zeros(ctx.num_parts, dtype=np.int64)
    _check(load().ras_get_update_counts(ctx.ptr, out.ctypes.data), "ras_get_update_counts")
    return out


def ras_get_launch(ctx: RasContext) -> dict:
    v, t, g, m = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(load().ras_get_launch(ctx.ptr, C.byref(v), C.byref(t), C.byref(g), C.byref(m)),
           "ras_get_launch")
    return {"kernel_variant": v.value, "cta_threads": t.value, "grid": g.value,
            "inner_iters": m.value}


def ras_get_phase_times(ctx: RasContext) -> np.ndarray:
    """(num_parts, 3) nanoseconds in gather / local solve / update of the last solve."""
    out = np.zeros(3 * ctx.num_parts, dtype=np.uint64)
    _check(load().ras_get_phase_times(ctx.ptr, out.ctypes.data), "ras_get_phase_times")
    return out.reshape(ctx.num_parts, 3)


def ras_relres(ctx: RasContext, b, x) -> float:
    r = C.c_double()
    _check(load().ras_relres(ctx.ptr, _dptr(b, ctx.n, "b"), _dptr(x, ctx.n, "x"), C.byref(r)), "ras_relres")
    return r.value


def ras_relres_noalloc(row_ptr, col_idx, val, b, x, out, stream=None) -> None:
    """No-allocation relative residual (see include/ras.h): every argument is
    a device tensor (int32 row_ptr / col_idx, float64 val / b / x, and a
    one-element float64 `out` that receives the result, stream-ordered)."""
    n = row_ptr.numel() - 1
    for t, dt, what in ((row_ptr, "int32", "row_ptr"), (col_idx, "int32", "col_idx")):
        if not (t.is_cuda and str(t.dtype).endswith(dt) and t.is_contiguous()):
            raise TypeError(f"{what} must be a contiguous {dt} CUDA tensor")
    _check(load().ras_relres_noalloc(n, row_ptr.data_ptr(), col_idx.data_ptr(),
                                     _dptr(val, None, "val"), _dptr(b, n, "b"), _dptr(x, n, "x"),
                                     _dptr(out, 1, "out"), _stream_handle(stream)),
           "ras_relres_noalloc")
