"""The s >= n form on the GPU (Lemma 1, Section 3.1): a static block with at
least as many rows as A has columns stores V_t = (A_t^T A_t + mu I)^{-1} and
updates x += V_t A_t^T (b_t - A_t x); when K >= n the dynamic block uses
(A_I^T A_I + mu I)^{-1} A_I^T r_I.  The GPU keeps the oracle's chains (column
sums over rows ascending, V's rows over columns ascending, the same Cholesky
and solves), so the drawn blocks, the top-K sets and the iterates equal the
oracle's bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


CASES = {
    # s = K = 80 >= n = 40: every static block and the dynamic block in the n x n form
    "sparse_tall": lambda: W.random_sparse(400, 40, 0.3, seed=17, num_blocks=5, lam=1e-3),
    # s = K = 200 >= n = 160
    "dense_tall": lambda: W.gaussian_dense(1600, 160, seed=7, num_blocks=8, lam=1e-8),
    # blocks of 40 and 41 rows on n = 41: both static forms side by side; K = 40 < n
    "sparse_mixed_forms": lambda: W.random_sparse(445, 41, 0.3, seed=5, num_blocks=11, lam=1e-4),
}


def _trace(h, s, iters, seed):
    K, n = h.info.dyn_rows, s.n
    tr = B.Trace()
    tau = torch.full((iters * 3,), -1, dtype=torch.int64, device="cuda")
    I = torch.full((iters * K,), -1, dtype=torch.int32, device="cuda")
    X = torch.zeros((iters, n), dtype=torch.float64, device="cuda")
    tr.capacity, tr.tau, tr.I, tr.x = iters, tau.data_ptr(), I.data_ptr(), X.data_ptr()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = h.solve(_dev(s.b), x, tol=0.0, maxit=iters, seed=seed, trace=tr)
    torch.cuda.synchronize()
    return res, tau.cpu().numpy().reshape(iters, 3), I.cpu().numpy().reshape(iters, K), X.cpu().numpy()


@pytest.mark.parametrize("name", sorted(CASES))
def test_iterations_equal_oracle(cuda_ok, name):
    s = CASES[name]()
    iters = 60
    with B.Handle.from_system(s) as h:
        res, tau, I, X = _trace(h, s, iters, seed=7)
    o = oracle.solve(s, maxit=iters, tol=0.0, seed=7, trace_tau=True, trace_I=True, trace_x=True)
    assert res.iters == o.iters == iters
    np.testing.assert_array_equal(tau, o.tau)
    np.testing.assert_array_equal(I, o.I)
    np.testing.assert_array_equal(X, o.x_trace)


@pytest.mark.parametrize("name", ["sparse_tall", "dense_tall", "sparse_mixed_forms"])
def test_stored_operators_and_single_static_updates_equal_oracle(cuda_ok, name):
    s = CASES[name]()
    k = s.num_blocks
    off = oracle.partition(s.m, k)
    rng = np.random.default_rng(3)
    with B.Handle.from_system(s) as h:
        for t in range(k):
            rows = np.arange(off[t], off[t + 1])
            x0 = rng.standard_normal(s.n)
            x = _dev(x0)
            b = _dev(s.b)
            h.static_update(t, b, x)
            if len(rows) >= s.n:
                Vg = h.static_operator(t, s.n)
                Vo = oracle.column_operator(s, k, t, s.lam)
                np.testing.assert_array_equal(Vg, Vo)
                xo = oracle.update_woodbury(s, rows, Vo, s.b, x0)
            else:
                Wo = oracle.static_operator(s, k, t, s.lam)
                xo = oracle.update_with_inverse(s, rows, Wo, s.b, x0)
            np.testing.assert_array_equal(x.cpu().numpy(), xo)


@pytest.mark.parametrize("name", ["sparse_tall", "dense_tall"])
def test_single_dynamic_update_equals_oracle(cuda_ok, name):
    s = CASES[name]()
    with B.Handle.from_system(s) as h:
        K = h.info.dyn_rows
        assert K >= s.n
        rng = np.random.default_rng(8)
        I = np.sort(rng.choice(s.m, K, replace=False)).astype(np.int32)
        x0 = rng.standard_normal(s.n)
        r = s.b - (s.to_dense() if not s.is_dense else s.dense) @ x0
        x = _dev(x0)
        h.dynamic_update(_dev(I), _dev(r), x)
    xo = oracle.update_woodbury_cholesky(s, I.astype(np.int64), s.lam, r[I], x0)
    np.testing.assert_array_equal(x.cpu().numpy(), xo)


@pytest.mark.parametrize("name", ["sparse_tall", "dense_tall"])
def test_mixed_precision_on_tall_systems_reaches_tolerance(cuda_ok, name):
    s = CASES[name]()
    A = s.to_dense() if not s.is_dense else s.dense
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(_dev(s.b), x, tol=1e-10, maxit=5000, seed=3, precision=B.PREC_MIXED)
    assert res.converged
    assert np.linalg.norm(A @ x.cpu().numpy() - s.b) / np.linalg.norm(s.b) <= 1.001e-10


def test_lambda_zero_with_full_column_rank_blocks(cuda_ok):
    """With mu = 0 every A_t A_t^T of a tall block is singular, so the s x s
    form cannot be set up; the n x n form needs only full column rank.  One
    static block then solves the consistent system."""
    s = W.gaussian_dense(1600, 160, seed=7, num_blocks=8, lam=0.0)
    with B.Handle.from_system(s, lam=0.0) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(_dev(s.b), x, tol=1e-12, maxit=10, seed=3)
    assert res.converged and res.iters == 1
    assert np.linalg.norm(x.cpu().numpy() - s.x_true) <= 1e-10 * np.linalg.norm(s.x_true)


def test_incremental_residual_refuses_the_nxn_dynamic_form(cuda_ok):
    s = CASES["sparse_tall"]()
    with B.Handle.from_system(s) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        with pytest.raises(B.RorbkError):
            h.solve(_dev(s.b), x, tol=1e-8, maxit=10, residual_mode=B.RESIDUAL_INCREMENTAL)
