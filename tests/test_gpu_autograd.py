"""Differentiable solve: gradients from the adjoint ROR-BK solve.

For x = A^{-1} b and L = 0.5 ||x - x_t||^2 the exact gradients are
dL/db = A^{-T}(x - x_t) and dL/da_ij = -(dL/db)_i x_j.  The references are
FP64 sparse LU solves (scipy) and central finite differences of the exactly
solved loss; the solver under test stops at a relative residual of 1e-12.

The 2025-unknown systems come from the power-law generator of the large
benchmark system: the row-scaled 45x45 Laplacian converges too slowly for a
1e-5 gradient check (its FP64 oracle still has a relative residual of 1.8e-5
after 120,000 iterations), so it checks properties that hold at any accuracy.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import oracle
from paper_2510_02156_gb300 import autograd as AG
from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GRAD_RTOL = 1e-5


def _csr(s):
    return sp.csr_matrix((s.values.astype(np.float64), s.col_idx, s.row_ptr), shape=(s.m, s.n))


def _system2025():
    return W.powerlaw(n=2025, num_blocks=8, seed=3, lam=1e-8)


def _grads(s, x_t, tol=1e-12, vdtype=torch.float64, **kw):
    vals = torch.tensor(s.values.astype(np.float64), dtype=vdtype, requires_grad=True)
    b = torch.tensor(s.b, dtype=torch.float64, requires_grad=True)
    x, spec = AG.solve(s.row_ptr, s.col_idx, vals, b, num_blocks=s.num_blocks, lam=s.lam,
                       tol=tol, **kw)
    L = 0.5 * ((x - torch.as_tensor(x_t, device=x.device)) ** 2).sum()
    L.backward()
    return x.detach().cpu().numpy(), vals.grad, b.grad, spec


def _reference(s, x_t):
    A = _csr(s)
    x = spla.spsolve(A.tocsc(), s.b)
    g = spla.spsolve(A.T.tocsc(), x - x_t)
    rows = np.repeat(np.arange(s.m), np.diff(s.row_ptr))
    return A, x, g, -g[rows] * x[s.col_idx]


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def test_gradients_match_fp64_reference(cuda_ok):
    s = _system2025()
    x_t = np.random.default_rng(21).standard_normal(s.n)
    x, dvals, db, spec = _grads(s, x_t)
    assert spec.last_forward.converged and spec.last_adjoint.converged
    A, x_ref, g_ref, dv_ref = _reference(s, x_t)
    assert _rel(x, x_ref) <= GRAD_RTOL
    assert _rel(db.numpy(), g_ref) <= GRAD_RTOL, _rel(db.numpy(), g_ref)
    assert _rel(dvals.numpy(), dv_ref) <= GRAD_RTOL, _rel(dvals.numpy(), dv_ref)


def test_gradients_match_central_differences(cuda_ok):
    """Directional derivatives along 10 random directions in b and 10 in the
    stored values, against central differences of the exactly solved loss."""
    s = _system2025()
    rng = np.random.default_rng(22)
    x_t = rng.standard_normal(s.n)
    _, dvals, db, _ = _grads(s, x_t)
    rows = np.repeat(np.arange(s.m), np.diff(s.row_ptr))
    base = s.values.astype(np.float64)

    def loss(vals, b):
        A = sp.csr_matrix((vals, s.col_idx, s.row_ptr), shape=(s.m, s.n))
        x = spla.spsolve(A.tocsc(), b)
        return 0.5 * float(np.sum((x - x_t) ** 2))

    for _ in range(10):
        d = rng.standard_normal(s.m)
        eps = 1e-3 * np.linalg.norm(s.b) / np.linalg.norm(d)   # L is quadratic in b
        fd = (loss(base, s.b + eps * d) - loss(base, s.b - eps * d)) / (2 * eps)
        an = float(db.numpy() @ d)
        assert abs(an - fd) <= GRAD_RTOL * abs(fd), (an, fd)
    for _ in range(10):
        d = rng.standard_normal(base.size) * np.abs(base)     # relative perturbation
        eps = 1e-6
        fd = (loss(base + eps * d, s.b) - loss(base - eps * d, s.b)) / (2 * eps)
        an = float(dvals.numpy() @ d)
        assert abs(an - fd) <= GRAD_RTOL * abs(fd), (an, fd)
    assert rows.size == base.size


def test_fp32_values_keep_their_dtype(cuda_ok):
    """An FP32 values tensor gets an FP32 gradient (the FP64 gradient
    rounded); the system is the same FP32-stored matrix."""
    s = _system2025()
    x_t = np.random.default_rng(23).standard_normal(s.n)
    _, dv32, db, _ = _grads(s, x_t, vdtype=torch.float32)
    _, _, _, dv_ref = _reference(s, x_t)
    assert dv32.dtype == torch.float32 and db.dtype == torch.float64
    assert _rel(dv32.double().numpy(), dv_ref) <= GRAD_RTOL


def test_adjoint_solve_follows_oracle_on_equilibrated_transpose(cuda_ok):
    """The adjoint solve is ROR-BK on At~ = A^T C^{-1} (C = diag of A's row
    norms) followed by g = C^{-1} h: the first 100 iterations agree with the
    FP64 oracle run on At~ (built here independently of the library)."""
    s = _system2025()
    A = _csr(s)
    c = np.sqrt(np.asarray(A.multiply(A).sum(axis=1)).ravel())
    At = (sp.diags(1.0 / c) @ A).T.tocsr()
    At.sort_indices()
    y = np.random.default_rng(24).standard_normal(s.n)
    T = W.System("adjoint", s.n, s.m, row_ptr=At.indptr.astype(np.int64),
                 col_idx=At.indices.astype(np.int32), values=At.data, b=y,
                 num_blocks=s.num_blocks, lam=s.lam, tol=0.0)
    with B.Handle.from_system(s) as h:
        adj = h.setup_adjoint(s.num_blocks, s.lam)
        try:
            for its in (1, 7, 100):
                g = torch.empty(s.m, dtype=torch.float64, device="cuda")
                res = adj.adjoint_solve(torch.as_tensor(y, device="cuda"), g, tol=0.0, maxit=its,
                                        seed=5)
                ro = oracle.solve(T, maxit=its, tol=0.0, seed=5)
                assert res.iters == ro.iters == its
                assert _rel(g.cpu().numpy(), ro.x / c) <= 1e-9
        finally:
            adj.close()


def test_laplacian_backward_properties(cuda_ok):
    """On the row-scaled Laplacian (slow to converge) the backward pass runs a
    bounded number of iterations.  What holds at any accuracy: the adjoint
    iterate h = C g (C = diag of A's row norms) starts at 0 and its error
    never grows (each regularised block update is non-expansive, Theorem 1),
    the residual of A^T g = dL/dx has dropped below its start, and the value
    gradient is exactly -g_i x_j."""
    s = W.laplace2d()
    x_t = np.random.default_rng(25).standard_normal(s.n)
    vals = torch.tensor(s.values, dtype=torch.float64, requires_grad=True)
    b = torch.tensor(s.b, dtype=torch.float64, requires_grad=True)
    x, spec = AG.solve(s.row_ptr, s.col_idx, vals, b, num_blocks=s.num_blocks, lam=s.lam,
                       tol=0.0, maxit=3000)
    xs = x.detach().cpu().numpy()
    gx = xs - x_t
    L = 0.5 * ((x - torch.as_tensor(x_t, device=x.device)) ** 2).sum()
    L.backward()
    A = _csr(s)
    g = b.grad.numpy()
    assert spec.last_adjoint.iters == 3000 and not spec.last_adjoint.converged
    assert np.linalg.norm(A.T @ g - gx) / np.linalg.norm(gx) < 1.0
    c = np.sqrt(np.asarray(A.multiply(A).sum(axis=1)).ravel())
    g_star = spla.spsolve(A.T.tocsc(), gx)
    assert np.linalg.norm(c * (g - g_star)) <= np.linalg.norm(c * g_star)
    rows = np.repeat(np.arange(s.m), np.diff(s.row_ptr))
    np.testing.assert_array_equal(vals.grad.numpy(), -(g[rows] * xs[s.col_idx]))


def test_full_size_forward_backward(cuda_ok):
    """The differentiable solve on the 262,144-unknown power-law system
    (1024 blocks of 256 rows): forward and adjoint reach their tolerance,
    measured on the host; the value gradient equals -g_i x_j exactly."""
    s = W.powerlaw(n=1 << 18, num_blocks=1024, seed=1, lam=1e-8)
    x_t = np.random.default_rng(26).standard_normal(s.n)
    x, dvals, db, spec = _grads(s, x_t, tol=1e-8)
    A = _csr(s)
    assert spec.last_forward.converged and spec.last_adjoint.converged
    assert np.linalg.norm(A @ x - s.b) / np.linalg.norm(s.b) <= 1.001e-8
    g = db.numpy()
    gx = x - x_t
    assert np.linalg.norm(A.T @ g - gx) / np.linalg.norm(gx) <= 1.001e-8
    rows = np.repeat(np.arange(s.m), np.diff(s.row_ptr))
    idx = np.random.default_rng(27).choice(rows.size, 4096, replace=False)
    np.testing.assert_array_equal(dvals.numpy()[idx], -(g[rows[idx]] * x[s.col_idx[idx]]))


def test_adjoint_solve_needs_an_adjoint_handle(cuda_ok):
    s = _system2025()
    with B.Handle.from_system(s) as h:
        g = torch.empty(s.m, dtype=torch.float64, device="cuda")
        with pytest.raises(B.RorbkError):
            h.adjoint_solve(torch.zeros(s.n, dtype=torch.float64, device="cuda"), g)
