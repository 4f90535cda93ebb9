"""Differentiable ROR-BK solve: x = A^{-1} b as a torch.autograd.Function.

The paper solves A x = b and does not differentiate the solution.  For a
square non-singular A and a loss L(x):

    dL/db = g   with   A^T g = dL/dx     (the adjoint system)
    dL/da_ij = -g_i x_j                  (for every stored entry of a sparse A)

The forward pass is one ROR-BK solve of A x = b; the backward pass is one
ROR-BK solve of A^T g = dL/dx (rorbk_adjoint_solve) on a handle the library
builds from the forward handle's copy of A (rorbk_setup_adjoint: A^T with
A's row scaling taken out of its columns, which ROR-BK needs to converge on
row-scaled systems), followed by the library's value-gradient kernel
(rorbk_value_grad).  Every arithmetic step runs
in the CUDA library; this module only marshals tensors.

Both solves stop at their own tolerance, so the gradient carries the solve
error: roughly cond(A) times the tolerance in the relative sense.

The handle lives on the SolveSpec.  The first forward sets it up from device
copies of the pattern and the values; every later forward with the same
spec hands the new values to rorbk_update_values, which re-forms the set-up
on the device (no host copy of A, no new handle).  The adjoint handle is
built on the device too (rorbk_setup_adjoint).  SolveSpec.close() frees the
handle.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from . import binding as B


@dataclass
class SolveSpec:
    """Pattern and solver settings of a differentiable solve (not differentiated)."""
    row_ptr: np.ndarray
    col_idx: np.ndarray
    m: int
    n: int
    num_blocks: int
    lam: float
    tol: float = 1e-10
    maxit: int = 1_000_000
    seed: int = 0
    precision: int = B.PREC_FP64
    adjoint_blocks: Optional[int] = None      # blocks of A^T's rows (default num_blocks)
    adjoint_tol: Optional[float] = None       # default tol
    inner_tol: float = 1e-4
    last_forward: Optional[B.Result] = field(default=None, repr=False)
    last_adjoint: Optional[B.Result] = field(default=None, repr=False)
    # the cached handle, its device pattern, and which forward's values it holds
    _handle: Optional[B.Handle] = field(default=None, repr=False)
    _pattern: Optional[tuple] = field(default=None, repr=False)
    _holds: int = field(default=0, repr=False)
    _forwards: int = field(default=0, repr=False)
    setups: int = 0                            # handles set up (1 after any number of forwards)

    def handle_for(self, vals, version):
        """The cached handle holding `vals` (device, this spec's value type)."""
        torch = _torch()
        if self._handle is None:
            if self._pattern is None:
                self._pattern = (torch.as_tensor(self.row_ptr, dtype=torch.int32, device="cuda"),
                                 torch.as_tensor(self.col_idx, dtype=torch.int32, device="cuda"))
            rp, ci = self._pattern
            self._handle = B.Handle(rp, ci, vals, self.m, self.n, self.num_blocks, self.lam,
                                    precision=self.precision)
            self.setups += 1
        elif self._holds != version:
            self._handle.update_values(vals)
        self._holds = version
        return self._handle

    def close(self):
        """Frees the cached handle."""
        if self._handle is not None:
            self._handle.close()
            self._handle = None


def _torch():
    import torch
    return torch


class RorbkSolve:
    """x = RorbkSolve.apply(values, b, spec): ROR-BK solve with an adjoint
    backward.  values: the nnz stored values of A in spec's CSR order (float64
    or float32, any device); b: (m,) float64.  Returns x (n,) float64 on the
    current CUDA device."""

    _fn = None

    @classmethod
    def function(cls):
        if cls._fn is None:
            torch = _torch()

            class _Solve(torch.autograd.Function):
                @staticmethod
                def forward(ctx, values, b, spec):
                    if spec.m != spec.n:
                        raise ValueError("the differentiable solve needs a square A")
                    vdt = torch.float32 if values.dtype == torch.float32 else torch.float64
                    vals = values.detach().to(device="cuda", dtype=vdt).contiguous()
                    spec._forwards += 1
                    version = spec._forwards
                    h = spec.handle_for(vals, version)
                    bd = b.detach().to(device="cuda", dtype=torch.float64).contiguous()
                    x = torch.empty(spec.n, dtype=torch.float64, device="cuda")
                    spec.last_forward = h.solve(bd, x, tol=spec.tol, maxit=spec.maxit,
                                                seed=spec.seed, precision=spec.precision,
                                                inner_tol=spec.inner_tol)
                    ctx.spec = spec
                    ctx.version = version
                    ctx.vmeta = (values.dtype, values.device)
                    ctx.bmeta = (b.dtype, b.device)
                    ctx.save_for_backward(x, vals)
                    return x

                @staticmethod
                def backward(ctx, gx):
                    x, vals = ctx.saved_tensors
                    spec = ctx.spec
                    # the handle again holds this forward's values (a later
                    # forward of the same spec may have replaced them)
                    h = spec.handle_for(vals, ctx.version)
                    kt = spec.adjoint_blocks or spec.num_blocks
                    adj = h.setup_adjoint(kt, spec.lam, precision=spec.precision)
                    try:
                        rhs = gx.detach().to(device="cuda", dtype=torch.float64).contiguous()
                        g = torch.empty(spec.m, dtype=torch.float64, device="cuda")
                        spec.last_adjoint = adj.adjoint_solve(
                            rhs, g, tol=spec.adjoint_tol or spec.tol, maxit=spec.maxit,
                            seed=spec.seed, precision=spec.precision, inner_tol=spec.inner_tol)
                    finally:
                        adj.close()
                    dvals = db = None
                    if ctx.needs_input_grad[0]:
                        dv = torch.empty(int(spec.row_ptr[-1]), dtype=torch.float64, device="cuda")
                        h.value_grad(g, x, dv)
                        dvals = dv.to(dtype=ctx.vmeta[0], device=ctx.vmeta[1])
                    if ctx.needs_input_grad[1]:
                        db = g.to(dtype=ctx.bmeta[0], device=ctx.bmeta[1])
                    return dvals, db, None

            cls._fn = _Solve
        return cls._fn

    @classmethod
    def apply(cls, values, b, spec: SolveSpec):
        return cls.function().apply(values, b, spec)


def solve(row_ptr, col_idx, values, b, *, num_blocks, lam, tol=1e-10, maxit=1_000_000,
          seed=0, precision=B.PREC_FP64, adjoint_tol=None, adjoint_blocks=None):
    """Differentiable x = A^{-1} b for a square CSR A given by (row_ptr,
    col_idx, values); gradients flow to values and b.  Returns (x, spec);
    spec.last_forward / spec.last_adjoint hold the solver results."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    m = rp.size - 1
    spec = SolveSpec(rp, ci, m, m, num_blocks, lam, tol=tol, maxit=maxit, seed=seed,
                     precision=precision, adjoint_tol=adjoint_tol, adjoint_blocks=adjoint_blocks)
    return RorbkSolve.apply(values, b, spec), spec
