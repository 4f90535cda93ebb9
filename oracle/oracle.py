"""ctypes marshalling for the C oracle (test infrastructure only).

Nothing here computes a step of the method: each wrapper converts numpy
arrays to pointers and calls the function of the same name in
``rorbk_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rorbk_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

ORC_OK, ORC_NOT_CONVERGED = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11 with POSIX threads, -O2, no fast-math)."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class OracleMatrix(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("is_dense", C.c_int32),
                ("pad_", C.c_int32), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("val", C.c_void_p),
                ("dense", C.c_void_p), ("ld", C.c_int64)]


_P = C.c_void_p
_I64 = C.c_int64
_D = C.c_double


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            sig = {
                "orc_philox4x64_10": (None, [_P, _P, _P]),
                "orc_partition": (C.c_int, [_I64, _I64, _P]),
                "orc_orthogonality": (C.c_int, [_P, _I64, _P, _P, _P]),
                "orc_proposal": (None, [_P, _I64, _I64, _P, _P, _P]),
                "orc_sample": (_I64, [_P, _I64, C.c_uint64, C.c_uint64, _I64, _I64]),
                "orc_residual": (_D, [_P, _P, _P, _P]),
                "orc_topk": (C.c_int, [_P, _I64, _I64, _P]),
                "orc_block_gram": (None, [_P, _P, _I64, _D, _P]),
                "orc_cholesky": (C.c_int, [_P, _I64]),
                "orc_chol_solve": (None, [_P, _I64, _P, _P]),
                "orc_spd_inverse": (C.c_int, [_P, _I64, _P]),
                "orc_static_operator": (C.c_int, [_P, _P, _I64, _D, _P]),
                "orc_update_with_inverse": (None, [_P, _P, _I64, _P, _P, _P, _P, _P]),
                "orc_update_with_cholesky": (C.c_int, [_P, _P, _I64, _D, _P, _P, _P]),
                "orc_solve": (C.c_int, [_P, _I64, _D, _P, _P, _P, _D, _I64,
                                        C.c_uint64, C.c_uint64, _I64, _I64, C.c_int, _P,
                                        _P, _P, _P, _P, _P, _P]),
                "orc_thread_count": (C.c_int, [_I64]),
                "orc_block_norms": (None, [_P, _P, _I64, _P]),
                "orc_initial_solution": (C.c_int, [_P, _I64, _I64, _P, _P]),
                "orc_fabgmres": (C.c_int, [_P, _I64, _D, _P, _P, _P, _D, _I64, _D, _I64,
                                           C.c_uint64, C.c_uint64, _I64, _P, _P, _P, _P]),
                "orc_weighted_cdf": (_D, [_P, _P, _I64, _P]),
                "orc_column_gram": (C.c_int, [_P, _P, _I64, _D, _P]),
                "orc_column_operator": (C.c_int, [_P, _P, _I64, _D, _P]),
                "orc_update_woodbury": (C.c_int, [_P, _P, _I64, _P, _P, _P]),
                "orc_update_woodbury_cholesky": (C.c_int, [_P, _P, _I64, _D, _P, _P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _Mat:
    """Keeps the FP64/int arrays alive while the C struct points at them."""

    def __init__(self, system):
        s = system
        self.m, self.n = int(s.m), int(s.n)
        if s.is_dense:
            self.dense = np.ascontiguousarray(s.dense, dtype=np.float64)
            self.st = OracleMatrix(self.m, self.n, 1, 0, None, None, None,
                                   self.dense.ctypes.data, self.n)
        else:
            self.rp = np.ascontiguousarray(s.row_ptr, dtype=np.int64)
            self.ci = np.ascontiguousarray(s.col_idx, dtype=np.int32)
            self.v = np.ascontiguousarray(s.values, dtype=np.float64)
            self.st = OracleMatrix(self.m, self.n, 0, 0, self.rp.ctypes.data,
                                   self.ci.ctypes.data, self.v.ctypes.data, None, 0)

    @property
    def ref(self):
        return C.byref(self.st)


def _mat(system):
    return system if isinstance(system, _Mat) else _Mat(system)


def philox4x64_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def partition(m, k):
    off = np.zeros(k + 1, dtype=np.int64)
    if lib().orc_partition(m, k, _ptr(off)) != 0:
        raise ValueError("bad partition")
    return off


def orthogonality(system, k, full=False):
    M = _mat(system)
    off = partition(M.m, k)
    Cm = np.zeros((k, k)) if full else None
    rs = np.zeros(k)
    if lib().orc_orthogonality(M.ref, k, _ptr(off), _ptr(Cm), _ptr(rs)) != 0:
        raise MemoryError("oracle orthogonality")
    return (Cm, rs) if full else rs


def proposal(C_rowsum, n):
    k = len(C_rowsum)
    rs = np.ascontiguousarray(C_rowsum, dtype=np.float64)
    Pbar, P, cdf = np.zeros(k), np.zeros(k), np.zeros(k)
    lib().orc_proposal(_ptr(rs), k, n, _ptr(Pbar), _ptr(P), _ptr(cdf))
    return Pbar, P, cdf


def sample(cdf, seed, sysid, it, l):
    c = np.ascontiguousarray(cdf, dtype=np.float64)
    return int(lib().orc_sample(_ptr(c), len(c), seed, sysid, it, l))


def residual(system, b, x):
    M = _mat(system)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    r = np.zeros(M.m)
    rr = lib().orc_residual(M.ref, _ptr(b), _ptr(x), _ptr(r))
    return r, rr


def topk(r, K):
    r = np.ascontiguousarray(r, dtype=np.float64)
    I = np.zeros(K, dtype=np.int64)
    if lib().orc_topk(_ptr(r), len(r), K, _ptr(I)) != 0:
        raise ValueError("bad K")
    return I


def block_gram(system, rows, mu):
    M = _mat(system)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    s = len(rows)
    G = np.zeros((s, s))
    lib().orc_block_gram(M.ref, _ptr(rows), s, mu, _ptr(G))
    return G


def cholesky(G):
    L = np.array(G, dtype=np.float64, order="C", copy=True)
    st = lib().orc_cholesky(_ptr(L), L.shape[0])
    if st != 0:
        raise np.linalg.LinAlgError("oracle cholesky: not SPD")
    return L


def chol_solve(L, r):
    L = np.ascontiguousarray(L, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    y = np.zeros_like(r)
    lib().orc_chol_solve(_ptr(L), L.shape[0], _ptr(r), _ptr(y))
    return y


def spd_inverse(L):
    L = np.ascontiguousarray(L, dtype=np.float64)
    W = np.zeros_like(L)
    lib().orc_spd_inverse(_ptr(L), L.shape[0], _ptr(W))
    return W


def static_operator(system, k, t, mu):
    M = _mat(system)
    off = partition(M.m, k)
    s = int(off[t + 1] - off[t])
    W = np.zeros((s, s))
    st = lib().orc_static_operator(M.ref, _ptr(off), t, mu, _ptr(W))
    if st != 0:
        raise np.linalg.LinAlgError(f"oracle static operator status {st}")
    return W


def update_with_inverse(system, rows, W, b, x):
    """Returns the updated copy of x (the input is not modified)."""
    M = _mat(system)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    W = np.ascontiguousarray(W, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.array(x, dtype=np.float64, copy=True)
    scratch = np.zeros(M.n)
    work = np.zeros(2 * len(rows))
    lib().orc_update_with_inverse(M.ref, _ptr(rows), len(rows), _ptr(W), _ptr(b),
                                  _ptr(x), _ptr(scratch), _ptr(work))
    return x


def update_with_cholesky(system, rows, mu, rI, x):
    M = _mat(system)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    rI = np.ascontiguousarray(rI, dtype=np.float64)
    x = np.array(x, dtype=np.float64, copy=True)
    scratch = np.zeros(M.n)
    st = lib().orc_update_with_cholesky(M.ref, _ptr(rows), len(rows), mu, _ptr(rI),
                                        _ptr(x), _ptr(scratch))
    if st != 0:
        raise np.linalg.LinAlgError(f"oracle dynamic update status {st}")
    return x


def column_gram(system, rows, mu):
    """A_B^T A_B + mu I (n x n) over the listed rows (the s >= n form)."""
    M = _mat(system)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    G = np.zeros((M.n, M.n))
    st = lib().orc_column_gram(M.ref, _ptr(rows), len(rows), mu, _ptr(G))
    if st != 0:
        raise MemoryError(f"oracle column Gram status {st}")
    return G


def column_operator(system, k, t, mu):
    """V_t = (A_t^T A_t + mu I)^{-1} (n x n) of static block t."""
    M = _mat(system)
    off = partition(M.m, k)
    V = np.zeros((M.n, M.n))
    st = lib().orc_column_operator(M.ref, _ptr(off), t, mu, _ptr(V))
    if st != 0:
        raise np.linalg.LinAlgError(f"oracle column operator status {st}")
    return V


def update_woodbury(system, rows, V, b, x):
    """x + V A_B^T (b_B - A_B x); returns the updated copy of x."""
    M = _mat(system)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    V = np.ascontiguousarray(V, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.array(x, dtype=np.float64, copy=True)
    st = lib().orc_update_woodbury(M.ref, _ptr(rows), len(rows), _ptr(V), _ptr(b), _ptr(x))
    if st != 0:
        raise MemoryError(f"oracle Woodbury update status {st}")
    return x


def update_woodbury_cholesky(system, rows, mu, rI, x):
    """The dynamic update in the n x n form (K >= n); returns the updated copy."""
    M = _mat(system)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    rI = np.ascontiguousarray(rI, dtype=np.float64)
    x = np.array(x, dtype=np.float64, copy=True)
    st = lib().orc_update_woodbury_cholesky(M.ref, _ptr(rows), len(rows), mu, _ptr(rI), _ptr(x))
    if st != 0:
        raise np.linalg.LinAlgError(f"oracle Woodbury dynamic update status {st}")
    return x


@dataclasses.dataclass
class SolveResult:
    x: np.ndarray
    status: int
    iters: int
    rrn: float
    tau: np.ndarray | None = None
    rrn_trace: np.ndarray | None = None
    I: np.ndarray | None = None
    x_trace: np.ndarray | None = None

    @property
    def converged(self):
        return self.status == ORC_OK


PAPER, RESIDUAL_WEIGHTED = 0, 1


def solve(system, b=None, x0=None, *, k=None, mu=None, tol=None, maxit=100,
          seed=0, sysid=0, n_static=3, start_iter=0, trace_tau=False,
          trace_rrn=False, trace_I=False, trace_x=False, dist_mode=PAPER, force_tau=None):
    """Algorithm 1 on one right-hand side.  ``system`` is a workloads.System
    (or its prepared matrix); b defaults to system.b.  dist_mode=RESIDUAL_WEIGHTED
    draws the static blocks with weights Pbar_t * ||r_{B_t}||^2 from the
    previous iteration's residual (not in the paper).  force_tau (iterations x
    n_static, -1 = draw) replays given blocks in place of the draws."""
    M = _mat(system)
    k = system.num_blocks if k is None else k
    mu = system.lam if mu is None else mu
    tol = system.tol if tol is None else tol
    b = np.ascontiguousarray(system.b if b is None else b, dtype=np.float64)
    x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    x = np.zeros(M.n)
    K = M.m // k
    tr_tau = np.full(maxit * n_static, -1, dtype=np.int64) if trace_tau else None
    tr_rrn = np.full(maxit, np.nan) if trace_rrn else None
    tr_I = np.full(maxit * K, -1, dtype=np.int64) if trace_I else None
    tr_x = np.zeros(maxit * M.n) if trace_x else None
    ft = None
    if force_tau is not None:
        ft = np.full(maxit * n_static, -1, dtype=np.int64)
        given = np.ascontiguousarray(force_tau, dtype=np.int64).ravel()[: ft.size]
        ft[: given.size] = given
    iters = C.c_int64(0)
    rrn = C.c_double(0.0)
    st = lib().orc_solve(M.ref, k, mu, _ptr(b), _ptr(x0), _ptr(x), tol, maxit,
                         C.c_uint64(seed), C.c_uint64(sysid), n_static, start_iter,
                         int(dist_mode), _ptr(ft), C.byref(iters), C.byref(rrn), _ptr(tr_tau),
                         _ptr(tr_rrn), _ptr(tr_I), _ptr(tr_x))
    if st < 0:
        raise RuntimeError(f"oracle solve failed with status {st}")
    it = iters.value
    return SolveResult(
        x=x, status=st, iters=it, rrn=rrn.value,
        tau=None if tr_tau is None else tr_tau[: it * n_static].reshape(it, n_static),
        rrn_trace=None if tr_rrn is None else tr_rrn[:it],
        I=None if tr_I is None else tr_I[: it * K].reshape(it, K),
        x_trace=None if tr_x is None else tr_x[: it * M.n].reshape(it, M.n),
    )


def fabgmres(system, b=None, x0=None, *, tol=None, maxit=50, eta=1e-2, lmax=100, seed=0,
             sysid=0, n_static=3):
    """Algorithm 3: flexible AB-GMRES with ROR-BK inner solves.  Returns
    (x, outer, inner, rrn, estimates, status)."""
    M = _mat(system)
    b = np.ascontiguousarray(system.b if b is None else b, dtype=np.float64)
    x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
    tol = system.tol if tol is None else tol
    x = np.zeros(M.n)
    est = np.full(maxit, np.nan)
    outer, inner, rrn = C.c_int64(0), C.c_int64(0), C.c_double(0.0)
    st = lib().orc_fabgmres(M.ref, system.num_blocks, system.lam, _ptr(b), _ptr(x0), _ptr(x), tol,
                            maxit, eta, lmax, C.c_uint64(seed), C.c_uint64(sysid), n_static,
                            C.byref(outer), C.byref(inner), C.byref(rrn), _ptr(est))
    if st < 0:
        raise RuntimeError(f"oracle FAB-GMRES status {st}")
    return x, outer.value, inner.value, rrn.value, est[: outer.value], st


def initial_solution(system, first, count, b=None):
    """Algorithm 2: x0 = (<b, A y> / ||A y||^2) y, y = sum of rows first ..
    first + count - 1."""
    M = _mat(system)
    b = np.ascontiguousarray(system.b if b is None else b, dtype=np.float64)
    x0 = np.zeros(M.n)
    st = lib().orc_initial_solution(M.ref, first, count, _ptr(b), _ptr(x0))
    if st != 0:
        raise ValueError(f"oracle initial solution status {st}")
    return x0


def block_norms(r, off):
    """rho_t = sum of r_i^2 over block t's rows (fused, rows ascending)."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    off = np.ascontiguousarray(off, dtype=np.int64)
    rho = np.zeros(off.size - 1)
    lib().orc_block_norms(_ptr(r), _ptr(off), off.size - 1, _ptr(rho))
    return rho


def weighted_cdf(Pbar, rho):
    """Running sum cdf_t = sum_{i <= t} Pbar_i * rho_i in block order."""
    Pbar = np.ascontiguousarray(Pbar, dtype=np.float64)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    cdf = np.zeros(Pbar.size)
    lib().orc_weighted_cdf(_ptr(Pbar), _ptr(rho), Pbar.size, _ptr(cdf))
    return cdf


def thread_count(rows):
    """Host threads the oracle's residual and top-K use for ``rows`` rows."""
    return int(lib().orc_thread_count(int(rows)))


def prepare(system):
    """Pre-marshal a system's matrix so repeated calls skip the conversion."""
    return _Mat(system)
