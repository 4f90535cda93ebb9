"""Seeded synthetic inputs for the ROR-BK solver and its oracle.

This module builds test and benchmark systems only.  It holds none of the
solver's arithmetic (no partition, no orthogonality, no block update), so both
the CUDA path and the CPU oracle can consume the same arrays without sharing
any step of the method.  It imports nothing else from this package.

Every system is consistent by construction: a seeded ``x_true`` is drawn and
``b = A @ x_true`` is formed in FP64 (the noise-free setting of the paper's
Section 3 experiments, where b is generated from a random N(0,1) solution).

Workloads (sizes are the defaults; every generator takes smaller sizes too):

* ``laplace2d``  -- 5-point Dirichlet Laplacian on a g x g grid, rows scaled by
  D = diag(10**U(-3, 0)); g = 45 gives n = 2025, nnz = 9945, cond ~ 1e7.
* ``powerlaw``   -- random square CSR: per row an off-diagonal count
  d = min(dmax, round(dmin * U**(-1/(alpha-1)))) (continuous Pareto tail,
  alpha = 2.5), columns uniform without replacement, values N(0,1), diagonal
  1 + sum|off-diagonal| ("diagonal shift"), rows scaled by 10**U(-4, 0), then
  rounded to FP32; the system is *defined* by the FP32 matrix, so an FP64
  residual over the FP32-stored values is exact.
* ``dense_usv``  -- A = U diag(s) V^T with U, V orthonormal (QR of seeded
  Gaussians) and s geometric from 1 to smin.

Arrays are numpy; CSR uses int64 row pointers and int32 column indices with
columns sorted ascending inside each row.
"""
from __future__ import annotations

import dataclasses
import os
from typing import Optional

import numpy as np


@dataclasses.dataclass
class System:
    """A consistent linear system A x = b with its generating solution."""

    name: str
    m: int
    n: int
    # CSR (sparse) ...
    row_ptr: Optional[np.ndarray] = None   # int64 [m+1]
    col_idx: Optional[np.ndarray] = None   # int32 [nnz]
    values: Optional[np.ndarray] = None    # float64 or float32 [nnz]
    # ... or dense row-major
    dense: Optional[np.ndarray] = None     # [m, n]
    x_true: Optional[np.ndarray] = None    # float64 [n] or [n, nrhs]
    b: Optional[np.ndarray] = None         # float64 [m] or [m, nrhs]
    num_blocks: int = 1
    lam: float = 1e-6
    tol: float = 1e-8

    @property
    def is_dense(self) -> bool:
        return self.dense is not None

    @property
    def nnz(self) -> int:
        return int(self.m * self.n) if self.is_dense else int(self.row_ptr[-1])

    def values_f64(self) -> np.ndarray:
        """CSR values widened to FP64 (exact when they were stored as FP32)."""
        return np.ascontiguousarray(self.values, dtype=np.float64)

    def dense_f64(self) -> np.ndarray:
        """Dense matrix as FP64 (exact widening of an FP32-stored matrix)."""
        return np.ascontiguousarray(self.dense, dtype=np.float64)

    def to_dense(self) -> np.ndarray:
        """Dense FP64 copy (small systems only)."""
        if self.is_dense:
            return self.dense_f64()
        out = np.zeros((self.m, self.n))
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        out[rows, self.col_idx] = self.values_f64()
        return out


def _csr_matvec(row_ptr, col_idx, values, x):
    """b = A x for input construction (float64, any row order)."""
    v = np.asarray(values, dtype=np.float64)
    prod = v * x[col_idx] if x.ndim == 1 else v[:, None] * x[col_idx]
    rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    if x.ndim == 1:
        return np.bincount(rows, weights=prod, minlength=len(row_ptr) - 1)
    out = np.zeros((len(row_ptr) - 1, x.shape[1]))
    for j in range(x.shape[1]):
        out[:, j] = np.bincount(rows, weights=prod[:, j], minlength=len(row_ptr) - 1)
    return out


def laplace2d(g: int = 45, seed: int = 0, num_blocks: int = 32,
              lam: float = 1e-6, tol: float = 1e-8, nrhs: int = 0) -> System:
    """Row-scaled 5-point Laplacian (g*g unknowns).

    Ordering: unknown (i, j) of the grid is row i*g + j.  Row scaling
    D = 10**U(-3, 0) is drawn first, then x_true ~ N(0, 1), both from
    ``numpy.random.default_rng(seed)``.
    """
    n = g * g
    rows, cols, vals = [], [], []
    for i in range(g):
        for j in range(g):
            r = i * g + j
            for (di, dj, v) in ((-1, 0, -1.0), (0, -1, -1.0), (0, 0, 4.0),
                                (0, 1, -1.0), (1, 0, -1.0)):
                ii, jj = i + di, j + dj
                if 0 <= ii < g and 0 <= jj < g:
                    rows.append(r)
                    cols.append(ii * g + jj)
                    vals.append(v)
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int32)
    vals = np.asarray(vals, dtype=np.float64)
    rng = np.random.default_rng(seed)
    d = 10.0 ** rng.uniform(-3.0, 0.0, n)
    vals = vals * d[rows]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    x_true = rng.standard_normal((n, nrhs) if nrhs else n)
    b = _csr_matvec(row_ptr, cols, vals, x_true)
    return System(f"laplace2d_g{g}", n, n, row_ptr=row_ptr, col_idx=cols,
                  values=vals, x_true=x_true, b=b, num_blocks=num_blocks,
                  lam=lam, tol=tol)


def powerlaw(n: int = 1 << 20, seed: int = 1, num_blocks: int = 4096,
             alpha: float = 2.5, dmin: int = 3, dmax: int = 200,
             scale_decades: float = 4.0, lam: float = 1e-6,
             tol: float = 1e-8, nrhs: int = 0,
             cache: Optional[str] = None) -> System:
    """Random square CSR system with power-law row lengths, stored in FP32.

    Draw order from ``numpy.random.default_rng(seed)``: off-diagonal counts,
    column indices, values, row scales, x_true.
    """
    key = f"powerlaw_n{n}_s{seed}_a{alpha}_{dmin}_{dmax}_{scale_decades}_r{nrhs}"
    if cache:
        path = os.path.join(cache, key + ".npz")
        if os.path.exists(path):
            z = np.load(path)
            return System(key, n, n, row_ptr=z["row_ptr"], col_idx=z["col_idx"],
                          values=z["values"], x_true=z["x_true"], b=z["b"],
                          num_blocks=num_blocks, lam=lam, tol=tol)
    rng = np.random.default_rng(seed)
    u = 1.0 - rng.random(n)                       # (0, 1]
    d = np.minimum(dmax, np.rint(dmin * u ** (-1.0 / (alpha - 1.0)))).astype(np.int64)
    d = np.minimum(d, n - 1)
    tot = int(d.sum())
    rows = np.repeat(np.arange(n, dtype=np.int64), d)
    # columns uniform over the n-1 off-diagonal positions, without replacement
    # inside a row: draw, then redraw the (rare) duplicates until none remain.
    c = rng.integers(0, n - 1, tot, dtype=np.int64)
    while True:
        c = np.where(c >= rows, c + 1, c)         # skip the diagonal
        key2 = rows * n + c
        order = np.argsort(key2, kind="stable")
        dup = np.zeros(tot, dtype=bool)
        sk = key2[order]
        dup[order[1:]] = sk[1:] == sk[:-1]
        if not dup.any():
            break
        redraw = rng.integers(0, n - 1, int(dup.sum()), dtype=np.int64)
        c = np.where(c > rows, c - 1, c)          # undo the diagonal skip
        c[dup] = redraw
    v = rng.standard_normal(tot)
    diag = 1.0 + np.bincount(rows, weights=np.abs(v), minlength=n)
    all_rows = np.concatenate([rows, np.arange(n, dtype=np.int64)])
    all_cols = np.concatenate([c, np.arange(n, dtype=np.int64)])
    all_vals = np.concatenate([v, diag])
    scale = 10.0 ** rng.uniform(-scale_decades, 0.0, n)
    all_vals = all_vals * scale[all_rows]
    order = np.lexsort((all_cols, all_rows))
    col_idx = all_cols[order].astype(np.int32)
    values = all_vals[order].astype(np.float32)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(d + 1)
    x_true = rng.standard_normal((n, nrhs) if nrhs else n)
    b = _csr_matvec(row_ptr, col_idx, values, x_true)
    if cache:
        os.makedirs(cache, exist_ok=True)
        np.savez(os.path.join(cache, key + ".npz"), row_ptr=row_ptr,
                 col_idx=col_idx, values=values, x_true=x_true, b=b)
    return System(key, n, n, row_ptr=row_ptr, col_idx=col_idx, values=values,
                  x_true=x_true, b=b, num_blocks=num_blocks, lam=lam, tol=tol)


def batched_sizes(count: int = 256, nmin: int = 5000, nmax: int = 200000,
                  seed: int = 42) -> np.ndarray:
    """Row counts of the batched workload: n ~ U[nmin, nmax] (integers,
    inclusive), one per system, from ``numpy.random.default_rng(seed)``."""
    return np.random.default_rng(seed).integers(nmin, nmax + 1, count)


def batched_system(i: int, n: int, lam: float = 1e-8, tol: float = 1e-8,
                   cache: Optional[str] = None) -> System:
    """System i of the batched workload: the power-law recipe with at most 50
    off-diagonals per row, generator seed 100 + i, blocks of 256 rows."""
    return powerlaw(n=int(n), num_blocks=max(1, int(n) // 256), seed=100 + i, dmax=50,
                    lam=lam, tol=tol, cache=cache)


def rhs_block(system: System, nrhs: int, seed: int) -> np.ndarray:
    """B = A X_true (m x nrhs, row-major, FP64 products of the stored values)
    for X_true ~ N(0,1) (n x nrhs) from ``numpy.random.default_rng(seed)``;
    column 0 is the system's own b."""
    rng = np.random.default_rng(seed)
    Xt = rng.standard_normal((system.n, nrhs))
    Bm = _csr_matvec(system.row_ptr, system.col_idx, system.values, Xt)
    Bm[:, 0] = system.b
    return np.ascontiguousarray(Bm)


def dense_usv(m: int, n: int, seed: int = 2, smin: float = 1e-8,
              block_rows: int = 256, lam: float = 1e-6, tol: float = 1e-8,
              nrhs: int = 0, dtype=np.float64) -> System:
    """Dense A = U diag(s) V^T, U (m x r) and V (n x r) orthonormal, r=min(m,n).

    s_i = smin**(i/(r-1)), i = 0..r-1.  The partition uses floor(m/block_rows)
    contiguous blocks.  x_true is drawn after U and V.
    """
    rng = np.random.default_rng(seed)
    r = min(m, n)
    U, _ = np.linalg.qr(rng.standard_normal((m, r)))
    V, _ = np.linalg.qr(rng.standard_normal((n, r)))
    s = smin ** (np.arange(r) / max(r - 1, 1))
    A = (U * s) @ V.T
    A = np.ascontiguousarray(A.astype(dtype))
    x_true = rng.standard_normal((n, nrhs) if nrhs else n)
    b = A.astype(np.float64) @ x_true
    k = max(1, m // block_rows)
    return System(f"dense_usv_{m}x{n}", m, n, dense=A, x_true=x_true, b=b,
                  num_blocks=k, lam=lam, tol=tol)


def dense_usv_cuda(m: int, n: int, seed: int = 2, smin: float = 1e-8,
                   block_rows: int = 256, lam: float = 1e-6, tol: float = 1e-8) -> System:
    """The dense_usv recipe at sizes where host QR is slow: U (m x r) and
    V (n x r) are the Q factors of seeded N(0,1) matrices drawn and factored on
    the current CUDA device with torch (input generation only), A = U diag(s)
    V^T in FP64, x_true ~ N(0,1), b = A x_true.  Returned as host arrays.  The
    stream differs from dense_usv's (another generator), not the recipe."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    r = min(m, n)
    U, _ = torch.linalg.qr(torch.randn(m, r, generator=g, device="cuda", dtype=torch.float64))
    V, _ = torch.linalg.qr(torch.randn(n, r, generator=g, device="cuda", dtype=torch.float64))
    sv = smin ** (torch.arange(r, device="cuda", dtype=torch.float64) / max(r - 1, 1))
    A = (U * sv) @ V.T
    del U
    x_true = torch.randn(n, generator=g, device="cuda", dtype=torch.float64)
    b = A @ x_true
    A_h = A.cpu().numpy()
    del A
    torch.cuda.empty_cache()
    k = max(1, m // block_rows)
    return System(f"dense_usv_{m}x{n}", m, n, dense=np.ascontiguousarray(A_h),
                  x_true=x_true.cpu().numpy(), b=b.cpu().numpy(), num_blocks=k, lam=lam, tol=tol)


def gaussian_dense(m: int, n: int, seed: int = 3, num_blocks: int = 4,
                   lam: float = 1e-6, tol: float = 1e-8) -> System:
    """Dense N(0,1) matrix with a consistent right-hand side (small tests)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n))
    x_true = rng.standard_normal(n)
    return System(f"gauss_{m}x{n}", m, n, dense=A, x_true=x_true, b=A @ x_true,
                  num_blocks=num_blocks, lam=lam, tol=tol)


def random_sparse(m: int, n: int, density: float, seed: int = 4,
                  num_blocks: int = 4, lam: float = 1e-6, tol: float = 1e-8,
                  empty_rows: int = 0) -> System:
    """Small random CSR matrix (tests): Bernoulli(density) pattern, N(0,1)
    values, optionally ``empty_rows`` all-zero rows, consistent b."""
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    vals = rng.standard_normal((m, n)) * mask
    if empty_rows:
        vals[rng.choice(m, empty_rows, replace=False)] = 0.0
        mask = vals != 0.0
    rows, cols = np.nonzero(mask)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(row_ptr, rows + 1, 1)
    row_ptr = np.cumsum(row_ptr)
    x_true = rng.standard_normal(n)
    values = vals[rows, cols].astype(np.float64)
    b = _csr_matvec(row_ptr, cols.astype(np.int32), values, x_true)
    return System(f"rand_{m}x{n}", m, n, row_ptr=row_ptr,
                  col_idx=cols.astype(np.int32), values=values, x_true=x_true,
                  b=b, num_blocks=num_blocks, lam=lam, tol=tol)
