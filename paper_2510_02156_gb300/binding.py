"""ctypes binding of the C ABI in include/rorbk.h (argument marshalling only).

Every step of the solver runs in the CUDA library ``_build/librorbk.so``; this
module converts numpy arrays and torch CUDA tensors to pointers, calls the
entry point of the same name and turns a non-OK status into an exception.
There is no CPU fallback: if the library is missing, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

RORBK_OK, RORBK_NOT_CONVERGED = 0, 1
STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", -1: "ERR_INVALID_ARG", -2: "ERR_CUDA",
                -3: "ERR_OOM", -4: "ERR_NOT_SPD", -5: "ERR_NUMERIC", -6: "ERR_BOUNDS",
                -7: "ERR_UNSUPPORTED", -8: "ERR_DEVICE_TIMEOUT"}
FORMAT_CSR, FORMAT_DENSE = 0, 1
F64, F32 = 0, 1
PREC_FP64, PREC_MIXED = 0, 1
OK, NOT_CONVERGED = 0, 1
DIST_PAPER, DIST_RESIDUAL_WEIGHTED = 0, 1
RESIDUAL_EXACT, RESIDUAL_INCREMENTAL = 0, 1
FAULT_NONE, FAULT_WAIT_LIMIT = 0, 1


class RorbkError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"rorbk status {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Matrix(C.Structure):
    _fields_ = [("format", C.c_int32), ("dtype", C.c_int32), ("m", C.c_int64),
                ("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("values", C.c_void_p), ("ld", C.c_int64),
                ("on_device", C.c_int32), ("reserved_", C.c_int32)]


class Partition(C.Structure):
    _fields_ = [("num_blocks", C.c_int32), ("reserved_", C.c_int32), ("offsets", C.c_void_p)]


class Trace(C.Structure):
    _fields_ = [("capacity", C.c_int64), ("tau", C.c_void_p), ("rrn", C.c_void_p),
                ("I", C.c_void_p), ("x", C.c_void_p), ("dyn", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("system_id", C.c_uint64), ("n_static", C.c_int32),
                ("precision", C.c_int32), ("start_iter", C.c_int64), ("inner_tol", C.c_double),
                ("inner_maxit", C.c_int64), ("host_loop", C.c_int32), ("poll", C.c_int32),
                ("trace", C.c_void_p), ("stream", C.c_void_p), ("dist_mode", C.c_int32),
                ("residual_mode", C.c_int32), ("refresh", C.c_int32), ("fault_inject", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("iters", C.c_int64), ("rrn", C.c_double), ("converged", C.c_int32),
                ("status", C.c_int32), ("refinements", C.c_int64), ("time_ms", C.c_double)]


class Info(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("nnz", C.c_int64),
                ("num_blocks", C.c_int32), ("dyn_rows", C.c_int32),
                ("max_block_rows", C.c_int32), ("format", C.c_int32), ("lambda_", C.c_double),
                ("device_bytes", C.c_int64)]


class Tuning(C.Structure):
    _fields_ = [("topk_blocks", C.c_int32), ("collect_blocks", C.c_int32),
                ("dyn_mark_blocks", C.c_int32), ("dyn_scatter_blocks", C.c_int32),
                ("residual_blocks", C.c_int32), ("graph_unroll", C.c_int32),
                ("us_default", C.c_double), ("us_tuned", C.c_double)]


# the entry points declared in include/rorbk.h, with their ctypes signatures
_P, _I64, _U64, _D = C.c_void_p, C.c_int64, C.c_uint64, C.c_double
SIGNATURES = {
    "rorbk_default_options": (None, [_P]),
    "rorbk_setup": (C.c_int, [_P, _P, _D, _P, _P]),
    "rorbk_update_values": (C.c_int, [_P, _P, C.c_int32, C.c_int32]),
    "rorbk_solve": (C.c_int, [_P, _P, _P, _P, _D, _I64, _P, _P]),
    "rorbk_solve_host": (C.c_int, [_P, _P, _P, _P, _D, _I64, _P, _P]),
    "rorbk_free": (None, [_P]),
    "rorbk_last_error": (C.c_char_p, [_P]),
    "rorbk_get_info": (C.c_int, [_P, _P]),
    "rorbk_get_proposal": (C.c_int, [_P, _P, _P]),
    "rorbk_get_static_operator": (C.c_int, [_P, _I64, _P]),
    "rorbk_sample": (C.c_int, [_P, _U64, _U64, _I64, _I64, _P]),
    "rorbk_static_update": (C.c_int, [_P, _I64, _P, _P]),
    "rorbk_residual": (C.c_int, [_P, _P, _P, _P, _P]),
    "rorbk_residual32": (C.c_int, [_P, _P, _P, _P, _P]),
    "rorbk_topk": (C.c_int, [_P, _P, _P]),
    "rorbk_dynamic_update": (C.c_int, [_P, _P, _P, _P]),
    "rorbk_dense_gram": (C.c_int, [_P, _P, _P, C.c_int32]),
    "rorbk_weighted_cdf": (C.c_int, [_P, _P, _P]),
    "rorbk_initial_solution": (C.c_int, [_P, _I64, _P, _P]),
    "rorbk_fabgmres": (C.c_int, [_P, _P, _P, _P, _D, _I64, _D, _I64, _P, _P]),
    "rorbk_clone": (C.c_int, [_P, _P]),
    "rorbk_batch_create": (C.c_int, [_P, C.c_int32, C.c_int32, _P]),
    "rorbk_batch_solve": (C.c_int, [_P, _P, _P, _P, _D, _I64, _P, _P, _P]),
    "rorbk_batch_free": (None, [_P]),
    "rorbk_multi_create": (C.c_int, [_P, C.c_int32, _P]),
    "rorbk_solve_multi": (C.c_int, [_P, _P, _P, _P, _D, _I64, _P, _P]),
    "rorbk_solve_multi_host": (C.c_int, [_P, _P, _P, _P, _D, _I64, _P, _P]),
    "rorbk_multi_results": (C.c_int, [_P, _P]),
    "rorbk_residual_multi": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P]),
    "rorbk_autotune": (C.c_int, [_P, _P, C.c_int32, _I64, C.c_char_p, _P]),
    "rorbk_set_tuning": (C.c_int, [_P, _P]),
    "rorbk_setup_adjoint": (C.c_int, [_P, _P, _D, _P, _P]),
    "rorbk_adjoint_solve": (C.c_int, [_P, _P, _P, _D, _I64, _P, _P]),
    "rorbk_value_grad": (C.c_int, [_P, _P, _P, _P]),
    "rorbk_csr_residual_noalloc": (C.c_int, [_I64, _I64, _I64, _P, _P, _P, C.c_int32, _P, _P,
                                             _P, _P, _P]),
}

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def lib(build: bool = True):
    """Load the CUDA library (building it first if its sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library missing: {path} (run __graft_entry__.build())")
            L = C.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(st, h=None):
    if st < 0:
        msg = lib().rorbk_last_error(h)
        raise RorbkError(st, msg.decode() if msg else "")
    return st


def _ptr(x):
    """Device pointer of a torch tensor or host pointer of a numpy array."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return x.ctypes.data_as(C.c_void_p)


def _is_device(x):
    return hasattr(x, "data_ptr") and getattr(x, "is_cuda", False)


def _value_dtype(t):
    """F64 / F32 for a torch tensor of float64 / float32 values."""
    name = str(t.dtype)
    if name == "torch.float64":
        return F64
    if name == "torch.float32":
        return F32
    raise ValueError("values must be float64 or float32")


def default_options(**kw) -> Options:
    o = Options()
    lib().rorbk_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(stream)


class Handle:
    """Owns one rorbk_handle (rorbk_setup ... rorbk_free)."""

    def __init__(self, row_ptr, col_idx, values, m, n, num_blocks, lam, precision=PREC_FP64,
                 offsets=None, stream=None):
        """A from host (numpy) arrays, or, for CSR, from device (torch CUDA)
        tensors: int32 row_ptr and col_idx and float64/float32 values, all on
        the device (rorbk_matrix.on_device = 1)."""
        self._keep = []
        if _is_device(values):
            if row_ptr is None or not (_is_device(row_ptr) and _is_device(col_idx)):
                raise ValueError("device values need device row_ptr and col_idx (CSR)")
            dt = _value_dtype(values)
            self._keep += [row_ptr, col_idx, values]
            A = Matrix(FORMAT_CSR, dt, m, n, int(values.numel()), row_ptr.data_ptr(),
                       col_idx.data_ptr(), values.data_ptr(), 0, 1, 0)
        else:
            vals = np.ascontiguousarray(values)
            if vals.dtype == np.float32:
                dt = F32
            else:
                vals = np.ascontiguousarray(vals, dtype=np.float64)
                dt = F64
            if row_ptr is None:            # dense row-major m x n
                if vals.shape != (m, n):
                    raise ValueError("dense values must have shape (m, n)")
                self._keep.append(vals)
                A = Matrix(FORMAT_DENSE, dt, m, n, m * n, None, None, vals.ctypes.data, n, 0, 0)
            else:
                rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
                ci = np.ascontiguousarray(col_idx, dtype=np.int32)
                self._keep += [rp, ci, vals]
                A = Matrix(FORMAT_CSR, dt, m, n, int(rp[-1]), rp.ctypes.data, ci.ctypes.data,
                           vals.ctypes.data, 0, 0, 0)
        offs = None
        if offsets is not None:
            offs = np.ascontiguousarray(offsets, dtype=np.int64)
            self._keep.append(offs)
        part = Partition(num_blocks, 0, None if offs is None else offs.ctypes.data)
        opt = default_options(precision=precision, stream=_stream_ptr(stream))
        h = C.c_void_p()
        st = lib().rorbk_setup(C.byref(A), C.byref(part), lam, C.byref(opt), C.byref(h))
        _check(st, None)
        self.h = h
        self.info = Info()
        _check(lib().rorbk_get_info(self.h, C.byref(self.info)), self.h)

    nr = 0

    @classmethod
    def _adopt(cls, raw):
        """Wrap an rorbk_handle made by the library (rorbk_setup_adjoint)."""
        self = cls.__new__(cls)
        self._keep = []
        self.h = raw
        self.info = Info()
        _check(lib().rorbk_get_info(self.h, C.byref(self.info)), self.h)
        return self

    def fabgmres(self, b, x, x0=None, tol=1e-8, maxit=50, eta=1e-2, lmax=100, seed=0,
                 system_id=0, n_static=3, start_iter=0, precision=PREC_FP64, stream=None):
        """rorbk_fabgmres (Algorithm 3) on device tensors; returns the Result
        (iters = outer steps, refinements = inner iterations in total)."""
        opt = default_options(seed=seed, system_id=system_id, n_static=n_static,
                              start_iter=start_iter, precision=precision,
                              stream=_stream_ptr(stream))
        res = Result()
        _check(lib().rorbk_fabgmres(self.h, _ptr(b), _ptr(x0), _ptr(x), tol, maxit, eta, lmax,
                                    C.byref(opt), C.byref(res)), self.h)
        return res

    def initial_solution(self, b, x0, block=0):
        """rorbk_initial_solution (Algorithm 2) on device tensors b (m), x0 (n)."""
        _check(lib().rorbk_initial_solution(self.h, block, _ptr(b), _ptr(x0)), self.h)

    def update_values(self, values):
        """rorbk_update_values: new values of A (same pattern), a numpy array
        or a device tensor of the handle's value type; re-forms the set-up on
        the device."""
        if _is_device(values):
            if not values.is_contiguous():
                raise ValueError("values must be contiguous")
            dt, on_dev = _value_dtype(values), 1
        else:
            values = np.ascontiguousarray(values)
            if values.dtype not in (np.float32, np.float64):
                values = np.ascontiguousarray(values, dtype=np.float64)
            dt, on_dev = (F32 if values.dtype == np.float32 else F64), 0
        _check(lib().rorbk_update_values(self.h, _ptr(values), dt, on_dev), self.h)

    def clone(self):
        """rorbk_clone: a Handle sharing this one's set-up, with its own workspace."""
        raw = C.c_void_p()
        _check(lib().rorbk_clone(self.h, C.byref(raw)), self.h)
        return Handle._adopt(raw)

    def multi(self, nr):
        """rorbk_multi_create: a Handle for a block of nr right-hand sides of
        this system (nr = 2, 4, 8, 16 or 32)."""
        raw = C.c_void_p()
        _check(lib().rorbk_multi_create(self.h, nr, C.byref(raw)), self.h)
        h = Handle._adopt(raw)
        h.nr = nr
        return h

    def solve_multi(self, B, X, X0=None, tol=1e-8, maxit=1000, seed=0, system_id=0, n_static=3,
                    start_iter=0, precision=PREC_FP64, traces=None, stream=None, inner_tol=1e-4,
                    inner_maxit=2000000, host_loop=0, poll=64, fault_inject=FAULT_NONE):
        """rorbk_solve_multi on device tensors B (m x nr), X (n x nr), X0 (or
        None), row-major; returns the list of per-column Results."""
        opt = default_options(seed=seed, system_id=system_id, n_static=n_static,
                              start_iter=start_iter, precision=precision,
                              stream=_stream_ptr(stream), inner_tol=inner_tol,
                              inner_maxit=inner_maxit, host_loop=host_loop, poll=poll,
                              fault_inject=fault_inject)
        if traces is not None:
            arr = (Trace * len(traces))(*traces)
            self._keep.append(arr)
            opt.trace = C.cast(arr, C.c_void_p)
        res = (Result * self.nr)()
        st = lib().rorbk_solve_multi(self.h, _ptr(B), _ptr(X0), _ptr(X), tol, maxit, C.byref(opt), res)
        _check(st, self.h)
        return list(res)

    def solve_multi_host(self, B, X, X0=None, tol=1e-8, maxit=1000, seed=0, precision=PREC_FP64,
                         inner_tol=1e-4, stream=None):
        """rorbk_solve_multi_host on numpy arrays (m x nr, n x nr row-major)."""
        opt = default_options(seed=seed, precision=precision, stream=_stream_ptr(stream),
                              inner_tol=inner_tol)
        res = (Result * self.nr)()
        st = lib().rorbk_solve_multi_host(self.h, _ptr(B), _ptr(X0), _ptr(X), tol, maxit,
                                          C.byref(opt), res)
        _check(st, self.h)
        return list(res)

    def residual_multi(self, B, X, R=None, precision=PREC_FP64, wait=True):
        """rorbk_residual_multi on row-major device tensors; returns the nr
        values ||r_j||^2 (or None with wait=False: enqueue only)."""
        rr = np.zeros(self.nr)
        _check(lib().rorbk_residual_multi(self.h, precision, _ptr(B), _ptr(X), _ptr(R),
                                          _ptr(rr) if wait else None), self.h)
        return rr if wait else None

    def autotune(self, b, precision=PREC_FP64, iters=50, cache_file=None):
        """rorbk_autotune: choose the launch shapes for this handle (b: device
        right-hand side(s)); returns the Tuning applied."""
        t = Tuning()
        path = None if cache_file is None else str(cache_file).encode()
        _check(lib().rorbk_autotune(self.h, _ptr(b), precision, iters, path, C.byref(t)), self.h)
        return t

    def set_tuning(self, t=None):
        """rorbk_set_tuning: apply given shapes (None: the defaults)."""
        _check(lib().rorbk_set_tuning(self.h, None if t is None else C.byref(t)), self.h)

    def multi_results(self):
        """rorbk_multi_results: the per-column results of the last solve."""
        res = (Result * self.nr)()
        _check(lib().rorbk_multi_results(self.h, res), self.h)
        return list(res)

    def setup_adjoint(self, num_blocks, lam, precision=PREC_FP64, offsets=None, stream=None):
        """rorbk_setup_adjoint: a Handle for A^T built from this handle's A."""
        offs = None
        if offsets is not None:
            offs = np.ascontiguousarray(offsets, dtype=np.int64)
        part = Partition(num_blocks, 0, None if offs is None else offs.ctypes.data)
        opt = default_options(precision=precision, stream=_stream_ptr(stream))
        raw = C.c_void_p()
        _check(lib().rorbk_setup_adjoint(self.h, C.byref(part), lam, C.byref(opt), C.byref(raw)),
               self.h)
        return Handle._adopt(raw)

    def adjoint_solve(self, y, g, tol=1e-8, maxit=1000, seed=0, system_id=0, n_static=3,
                      precision=PREC_FP64, stream=None, inner_tol=1e-4, inner_maxit=2000000):
        """rorbk_adjoint_solve on a handle from setup_adjoint: A^T g = y."""
        opt = default_options(seed=seed, system_id=system_id, n_static=n_static,
                              precision=precision, stream=_stream_ptr(stream),
                              inner_tol=inner_tol, inner_maxit=inner_maxit)
        res = Result()
        _check(lib().rorbk_adjoint_solve(self.h, _ptr(y), _ptr(g), tol, maxit, C.byref(opt),
                                         C.byref(res)), self.h)
        return res

    def value_grad(self, g, x, dvals):
        """rorbk_value_grad: dvals[p] = -g_i x_j over A's stored entries."""
        _check(lib().rorbk_value_grad(self.h, _ptr(g), _ptr(x), _ptr(dvals)), self.h)

    @classmethod
    def from_system(cls, system, lam=None, precision=PREC_FP64, **kw):
        lam = system.lam if lam is None else lam
        if system.is_dense:
            return cls(None, None, system.dense, system.m, system.n, system.num_blocks, lam,
                       precision, **kw)
        return cls(system.row_ptr, system.col_idx, system.values, system.m, system.n,
                   system.num_blocks, lam, precision, **kw)

    def close(self):
        if getattr(self, "h", None):
            lib().rorbk_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- whole solve --------------------------------------------------------
    def solve(self, b, x, x0=None, tol=1e-8, maxit=1000, seed=0, system_id=0, n_static=3,
              start_iter=0, precision=PREC_FP64, trace=None, stream=None, inner_tol=1e-4,
              inner_maxit=2000000, host_loop=0, poll=64, dist_mode=DIST_PAPER,
              residual_mode=RESIDUAL_EXACT, refresh=0, fault_inject=FAULT_NONE):
        """rorbk_solve on device tensors b (m), x (n), x0 (n or None)."""
        opt = default_options(seed=seed, system_id=system_id, n_static=n_static,
                              start_iter=start_iter, precision=precision,
                              stream=_stream_ptr(stream), inner_tol=inner_tol,
                              inner_maxit=inner_maxit, host_loop=host_loop, poll=poll,
                              dist_mode=dist_mode, residual_mode=residual_mode,
                              refresh=refresh, fault_inject=fault_inject)
        if trace is not None:
            opt.trace = C.cast(C.pointer(trace), C.c_void_p)
        res = Result()
        st = lib().rorbk_solve(self.h, _ptr(b), _ptr(x0), _ptr(x), tol, maxit, C.byref(opt),
                               C.byref(res))
        _check(st, self.h)
        return res

    def solve_host(self, b, x, x0=None, tol=1e-8, maxit=1000, seed=0, system_id=0,
                   n_static=3, start_iter=0, precision=PREC_FP64, stream=None,
                   inner_tol=1e-4, inner_maxit=2000000):
        """rorbk_solve_host on host (numpy float64) arrays."""
        opt = default_options(seed=seed, system_id=system_id, n_static=n_static,
                              start_iter=start_iter, precision=precision,
                              stream=_stream_ptr(stream), inner_tol=inner_tol,
                              inner_maxit=inner_maxit)
        res = Result()
        st = lib().rorbk_solve_host(self.h, _ptr(b), _ptr(x0), _ptr(x), tol, maxit,
                                    C.byref(opt), C.byref(res))
        _check(st, self.h)
        return res

    # -- setup products and single steps -----------------------------------
    def proposal(self):
        k = self.info.num_blocks
        cdf, rs = np.zeros(k), np.zeros(k)
        _check(lib().rorbk_get_proposal(self.h, _ptr(cdf), _ptr(rs)), self.h)
        return cdf, rs

    def static_operator(self, t, s):
        W = np.zeros((s, s))
        _check(lib().rorbk_get_static_operator(self.h, t, _ptr(W)), self.h)
        return W

    def sample(self, seed, system_id, it, l):
        tau = C.c_int64()
        _check(lib().rorbk_sample(self.h, seed, system_id, it, l, C.byref(tau)), self.h)
        return tau.value

    def static_update(self, tau, b, x):
        _check(lib().rorbk_static_update(self.h, tau, _ptr(b), _ptr(x)), self.h)

    def residual(self, b, x, r):
        rr = C.c_double()
        _check(lib().rorbk_residual(self.h, _ptr(b), _ptr(x), _ptr(r), C.byref(rr)), self.h)
        return rr.value

    def residual_async(self, b, x, r):
        """Enqueue r = b - A x on the handle's stream without waiting."""
        _check(lib().rorbk_residual(self.h, _ptr(b), _ptr(x), _ptr(r), None), self.h)

    def residual32(self, b, x, r, wait=True):
        """FP32 residual of the mixed form (float32 device tensors)."""
        rr = C.c_double()
        _check(lib().rorbk_residual32(self.h, _ptr(b), _ptr(x), _ptr(r),
                                      C.byref(rr) if wait else None), self.h)
        return rr.value if wait else None

    def topk(self, r, I):
        _check(lib().rorbk_topk(self.h, _ptr(r), _ptr(I)), self.h)

    def dynamic_update(self, I, r, x):
        _check(lib().rorbk_dynamic_update(self.h, _ptr(I), _ptr(r), _ptr(x)), self.h)

    def weighted_cdf(self, r):
        """rorbk_weighted_cdf: the residual-weighted running sum after the
        device residual r (numpy array of k doubles)."""
        cdf = np.zeros(self.info.num_blocks)
        _check(lib().rorbk_weighted_cdf(self.h, _ptr(r), _ptr(cdf)), self.h)
        return cdf

    def dense_gram(self, I, G, precision=PREC_FP64):
        """rorbk_dense_gram: packed lower A_I A_I^T + mu I into the device tensor G."""
        _check(lib().rorbk_dense_gram(self.h, _ptr(I), _ptr(G), precision), self.h)


class Batch:
    """Owns one rorbk_batch: several handles' solves in one graph launch."""

    def __init__(self, handles, precision=PREC_FP64):
        self.handles = list(handles)
        arr = (C.c_void_p * len(self.handles))(*[h.h for h in self.handles])
        raw = C.c_void_p()
        _check(lib().rorbk_batch_create(arr, len(self.handles), precision, C.byref(raw)), None)
        self.b = raw
        self.precision = precision

    def solve(self, bs, xs, x0s=None, tol=1e-8, maxit=1000, seed=0, system_ids=None, n_static=3,
              inner_tol=1e-4, inner_maxit=2000000, stream=None):
        """rorbk_batch_solve on lists of device tensors; returns (status, results)."""
        k = len(self.handles)
        P = C.c_void_p * k
        b_arr = P(*[b.data_ptr() for b in bs])
        x_arr = P(*[x.data_ptr() for x in xs])
        x0_arr = None if x0s is None else P(*[0 if v is None else v.data_ptr() for v in x0s])
        ids = None if system_ids is None else (C.c_uint64 * k)(*system_ids)
        opt = default_options(seed=seed, n_static=n_static, precision=self.precision,
                              stream=_stream_ptr(stream), inner_tol=inner_tol,
                              inner_maxit=inner_maxit)
        res = (Result * k)()
        st = lib().rorbk_batch_solve(self.b, b_arr, x0_arr, x_arr, tol, maxit, C.byref(opt), ids,
                                     res)
        _check(st, None)
        return st, list(res)

    def close(self):
        if getattr(self, "b", None):
            lib().rorbk_batch_free(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def csr_residual_noalloc(row_ptr, col_idx, values, m, n, b, x, r, rr_out, stream=None):
    """rorbk_csr_residual_noalloc on device tensors (CSR arrays, b, x, r and a
    one-element FP64 tensor rr_out); allocates no device memory."""
    dt = F32 if str(values.dtype) == "torch.float32" else F64
    st = lib().rorbk_csr_residual_noalloc(m, n, int(col_idx.numel()), _ptr(row_ptr), _ptr(col_idx),
                                          _ptr(values), dt, _ptr(b), _ptr(x), _ptr(r), _ptr(rr_out),
                                          _stream_ptr(stream))
    _check(st, None)
