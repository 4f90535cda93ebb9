"""Dense A (row-major) on the GPU against the FP64 oracle's dense path.

A dense A is held as CSR with every entry stored, so the static updates, the
residual and the top-K run the sparse kernels; the dynamic block, where every
row of I shares every column, has a dense Gram, factor and scatter of its own.
Every product chain keeps the definition's order, so the iterates are the
oracle's bit for bit (the tests assert the 1e-9 bound and, beyond it,
equality)."""
import numpy as np
import pytest

import oracle
from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


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


DENSE = {
    "gauss_tall": lambda: W.gaussian_dense(700, 120, seed=3, num_blocks=5, lam=1e-6),
    "usv_tall": lambda: W.dense_usv(2600, 256, seed=2, block_rows=256, lam=2.56e-4),
}


@pytest.mark.parametrize("name", sorted(DENSE))
def test_dense_iterations_equal_oracle(cuda_ok, name):
    s = DENSE[name]()
    iters = 60
    with B.Handle.from_system(s) as h:
        assert h.info.format == B.FORMAT_DENSE
        res, tau, I, X = _trace(h, s, iters, seed=4)
    o = oracle.solve(s, maxit=iters, tol=0.0, seed=4, trace_tau=True, trace_I=True, trace_x=True)
    assert res.iters == o.iters == iters
    np.testing.assert_array_equal(tau, o.tau)
    np.testing.assert_array_equal(I, o.I)
    worst = max(_rel(X[j], o.x_trace[j]) for j in range(iters))
    assert worst <= 1e-9, worst
    np.testing.assert_array_equal(X, o.x_trace)


def test_dense_single_dynamic_update_equals_oracle(cuda_ok):
    s = W.dense_usv(2600, 256, seed=2, block_rows=256, lam=2.56e-4)
    rng = np.random.default_rng(5)
    x0 = rng.standard_normal(s.n)
    with B.Handle.from_system(s) as h:
        K = h.info.dyn_rows
        r = s.b - s.dense @ x0
        I = np.sort(rng.choice(s.m, K, replace=False)).astype(np.int32)
        x = _dev(x0)
        h.dynamic_update(_dev(I), _dev(r), x)
        # K = n = 256 here: the n x n form of Lemma 1 applies (K >= n)
        if K >= s.n:
            xo = oracle.update_woodbury_cholesky(s, I, s.lam, r[I], x0)
        else:
            xo = oracle.update_with_cholesky(s, I, s.lam, r[I], x0)
    np.testing.assert_array_equal(x.cpu().numpy(), xo)


def test_dense_wide_system_reaches_min_norm_solution(cuda_ok):
    """m < n from x0 = 0: the iterates stay in range(A^T) and converge to the
    minimum-norm solution (Lemma 2)."""
    s = W.gaussian_dense(200, 600, seed=6, num_blocks=4, lam=1e-8)
    with B.Handle.from_system(s) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(_dev(s.b), x, tol=1e-11, maxit=20000, seed=1)
    assert res.converged
    x_mn = np.linalg.lstsq(s.dense, s.b, rcond=None)[0]
    assert _rel(x.cpu().numpy(), x_mn) <= 1e-8


def test_dense_solve_to_tolerance_matches_oracle(cuda_ok):
    s = W.gaussian_dense(1600, 160, seed=7, num_blocks=8, lam=1e-8)
    o = oracle.solve(s, maxit=5000, tol=1e-10, seed=3)
    assert o.converged
    with B.Handle.from_system(s) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(_dev(s.b), x, tol=1e-10, maxit=5000, seed=3)
    assert res.converged and res.iters == o.iters
    np.testing.assert_array_equal(x.cpu().numpy(), o.x)


def test_dense_mixed_precision_reaches_tolerance(cuda_ok):
    """Blocks of 100 rows on 400 columns: the mixed form reaches the
    tolerance, measured in FP64 on the host."""
    s = W.gaussian_dense(1600, 400, seed=7, num_blocks=16, lam=1e-8)
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(_dev(s.b), x, tol=1e-10, maxit=50000, seed=3, precision=B.PREC_MIXED)
    xh = x.cpu().numpy()
    assert res.converged
    assert np.linalg.norm(s.dense @ xh - s.b) / np.linalg.norm(s.b) <= 1.001e-10


def test_mixed_precision_with_blocks_longer_than_n(cuda_ok):
    """Blocks of 200 rows on 160 columns: each block Gram A_t A_t^T is
    singular, so its inverse would carry 1/mu on the null space, which FP32
    cannot hold.  The s >= n form (Lemma 1, Section 3.1) stores the n x n
    inverse instead, and the dynamic block (K = 200 >= n) uses the same form:
    the mixed solve reaches the tolerance, measured in FP64 on the host."""
    s = W.gaussian_dense(1600, 160, seed=7, num_blocks=8, lam=1e-8)
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(_dev(s.b), x, tol=1e-10, maxit=2000, seed=3, precision=B.PREC_MIXED)
    xh = x.cpu().numpy()
    assert res.converged
    assert np.linalg.norm(s.dense @ xh - s.b) / np.linalg.norm(s.b) <= 1.001e-10


def test_dense_full_size_iterations_equal_oracle(cuda_ok):
    """The dense least-squares size of the benchmark, m = 200,000 x n = 2,048
    with 781 blocks of 256 rows (a Gaussian matrix: the layout and sizes
    matter here, not the spectrum): two whole iterations equal the oracle."""
    s = W.gaussian_dense(200_000, 2048, seed=8, num_blocks=781, lam=2.56e-4)
    iters = 2
    with B.Handle.from_system(s) as h:
        res, tau, I, X = _trace(h, s, iters, seed=9)
    o = oracle.solve(s, maxit=iters, tol=0.0, seed=9, trace_tau=True, trace_I=True, trace_x=True)
    np.testing.assert_array_equal(tau, o.tau)
    np.testing.assert_array_equal(I, o.I)
    np.testing.assert_array_equal(X, o.x_trace)
