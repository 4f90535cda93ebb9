"""A block of right-hand sides (rorbk_multi_create / rorbk_solve_multi).

Every column of a block is solved as rorbk_solve solves it alone: the same
Philox stream, top-K sets, dynamic updates and stopping test.  The block only
changes the data movement (one pass over A for all columns' residuals, one
grid row per column in the other kernels), and every (row, column) residual
is the one-column kernel's chain in the same order.  So:
- each column's drawn blocks, top-K sets and iterates equal the FP64
  oracle's one-column run of that right-hand side (100 iterations, bit for
  bit; the parity bound 1e-9 is asserted as well), on the power-law, the
  row-scaled Laplacian and a ragged system with empty rows;
- each column's solve equals the one-column solve of the library bit for bit
  in FP64 and in the mixed form (same iterations, RRN and x), unless a stopping
  test falls within rounding of the tolerance (the sums of squares of a block
  run in another order), which these cases do not meet;
- columns stop independently (a zero right-hand side, an earlier converging
  column), the host-driven loop equals the graph, batches may mix blocks and
  one-column handles, and unsupported forms are refused.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dt)


def _rhs(s, nr, seed):
    """B = A X_true (FP64 products of the stored values), column 0 = s.b."""
    A = sp.csr_matrix((s.values.astype(np.float64), s.col_idx, s.row_ptr), shape=(s.m, s.n))
    rng = np.random.default_rng(seed)
    Xt = rng.standard_normal((s.n, nr))
    Bm = np.asarray(A @ Xt)
    Bm[:, 0] = s.b
    return np.ascontiguousarray(Bm)


def _traces(nr, iters, K, n):
    keep, trs = [], []
    for _ in range(nr):
        tau = torch.full((iters * 3,), -1, dtype=torch.int64, device="cuda")
        I = torch.full((iters * K,), -1, dtype=torch.int32, device="cuda")
        X = torch.zeros((iters, n), dtype=torch.float64, device="cuda")
        tr = B.Trace()
        tr.capacity, tr.tau, tr.I, tr.x = iters, tau.data_ptr(), I.data_ptr(), X.data_ptr()
        keep.append((tau, I, X))
        trs.append(tr)
    return keep, trs


CASES = {
    "powerlaw16k": lambda: W.powerlaw(n=1 << 14, num_blocks=64, lam=1e-8),
    "laplace45": lambda: W.laplace2d(),
    "ragged": lambda: W.random_sparse(997, 600, 0.01, seed=7, num_blocks=13, lam=1e-6, empty_rows=9),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_every_column_follows_the_oracle_for_100_iterations(cuda_ok, name):
    s = CASES[name]()
    nr, iters = 4, 100
    Bm = _rhs(s, nr, seed=21)
    with B.Handle.from_system(s) as h0, h0.multi(nr) as h:
        K = h.info.dyn_rows
        keep, trs = _traces(nr, iters, K, s.n)
        X = torch.zeros((s.n, nr), dtype=torch.float64, device="cuda")
        res = h.solve_multi(_dev(Bm), X, tol=0.0, maxit=iters, seed=5, traces=trs)
        torch.cuda.synchronize()
    for j in range(nr):
        o = oracle.solve(s, b=Bm[:, j], maxit=iters, tol=0.0, seed=5, trace_tau=True, trace_I=True,
                         trace_x=True)
        tau, I, Xt = (t.cpu().numpy() for t in keep[j])
        assert res[j].iters == o.iters == iters
        np.testing.assert_array_equal(tau.reshape(iters, 3), o.tau)
        np.testing.assert_array_equal(I.reshape(iters, K), o.I)
        worst = max(np.linalg.norm(Xt[t] - o.x_trace[t]) / np.linalg.norm(o.x_trace[t]) for t in range(iters))
        assert worst <= 1e-9, (name, j, worst)
        np.testing.assert_array_equal(Xt, o.x_trace)
        np.testing.assert_array_equal(X[:, j].cpu().numpy(), o.x)


@pytest.mark.parametrize("nr", [2, 16, 32])
@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_MIXED])
def test_every_column_equals_its_one_column_solve(cuda_ok, nr, precision):
    s = W.powerlaw(n=1 << 13, num_blocks=32, seed=9, lam=1e-8, tol=1e-8)
    Bm = _rhs(s, nr, seed=nr)
    with B.Handle.from_system(s, precision=precision) as h0, h0.multi(nr) as h:
        X = torch.zeros((s.n, nr), dtype=torch.float64, device="cuda")
        res = h.solve_multi(_dev(Bm), X, tol=1e-8, maxit=200000, seed=3, precision=precision)
        for j in range(nr):
            x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
            r1 = h0.solve(_dev(Bm[:, j]), x, tol=1e-8, maxit=200000, seed=3, precision=precision)
            assert res[j].converged and r1.converged, (j, res[j].rrn)
            # the RRN is the same residual's norm, its squares summed in another order
            assert (res[j].iters, res[j].refinements) == (r1.iters, r1.refinements), j
            assert abs(res[j].rrn - r1.rrn) <= 1e-13 * r1.rrn, j
            assert torch.equal(X[:, j], x), j
    # the FP64 residual of every column, checked on the host
    A = sp.csr_matrix((s.values.astype(np.float64), s.col_idx, s.row_ptr), shape=(s.m, s.n))
    Xh = X.cpu().numpy()
    for j in range(nr):
        assert np.linalg.norm(Bm[:, j] - A @ Xh[:, j]) / np.linalg.norm(Bm[:, j]) <= 1.001e-8


def test_solve_to_tolerance_matches_the_oracle_per_column(cuda_ok):
    s = W.powerlaw(n=1 << 13, num_blocks=32, seed=9, lam=1e-8, tol=1e-8)
    nr = 4
    Bm = _rhs(s, nr, seed=44)
    with B.Handle.from_system(s) as h0, h0.multi(nr) as h:
        X = torch.zeros((s.n, nr), dtype=torch.float64, device="cuda")
        res = h.solve_multi(_dev(Bm), X, tol=1e-8, maxit=100000, seed=2)
    for j in range(nr):
        o = oracle.solve(s, b=Bm[:, j], maxit=100000, seed=2)
        assert o.converged and res[j].converged
        assert res[j].iters == o.iters, (j, res[j].iters, o.iters)
        assert abs(res[j].rrn - o.rrn) <= 1e-12 * o.rrn
        np.testing.assert_array_equal(X[:, j].cpu().numpy(), o.x)


def test_columns_stop_independently(cuda_ok):
    """A zero right-hand side stops at once (x = 0, no iterations); a column
    started at its solution stops after one iteration; the others run on."""
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=3, lam=1e-8, tol=1e-8)
    nr = 4
    Bm = _rhs(s, nr, seed=8)
    Bm[:, 1] = 0.0
    X0 = np.zeros((s.n, nr))
    X0[:, 2] = s.x_true
    Bm[:, 2] = s.b
    with B.Handle.from_system(s) as h0, h0.multi(nr) as h:
        X = torch.zeros((s.n, nr), dtype=torch.float64, device="cuda")
        res = h.solve_multi(_dev(Bm), X, X0=_dev(X0), tol=1e-8, maxit=100000, seed=1)
        assert all(r.converged for r in res)
        assert res[1].iters == 0 and torch.count_nonzero(X[:, 1]) == 0
        assert res[2].iters <= 1
        assert res[0].iters > 10 and res[3].iters > 10
        assert [r.iters for r in h.multi_results()] == [r.iters for r in res]


def test_host_loop_equals_graph(cuda_ok):
    s = W.powerlaw(n=1 << 13, num_blocks=32, seed=9, lam=1e-8)
    nr = 8
    Bm = _rhs(s, nr, seed=3)
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h0, h0.multi(nr) as h:
        for prec in (B.PREC_FP64, B.PREC_MIXED):
            X1 = torch.zeros((s.n, nr), dtype=torch.float64, device="cuda")
            X2 = torch.zeros((s.n, nr), dtype=torch.float64, device="cuda")
            r1 = h.solve_multi(_dev(Bm), X1, tol=1e-8, maxit=3000, seed=4, precision=prec)
            r2 = h.solve_multi(_dev(Bm), X2, tol=1e-8, maxit=3000, seed=4, precision=prec,
                               host_loop=1, poll=16)
            assert [r.iters for r in r1] == [r.iters for r in r2]
            assert torch.equal(X1, X2)


def test_host_buffers(cuda_ok):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=3, lam=1e-8)
    nr = 4
    Bm = _rhs(s, nr, seed=2)
    with B.Handle.from_system(s) as h0, h0.multi(nr) as h:
        Xh = np.zeros((s.n, nr))
        rh = h.solve_multi_host(Bm, Xh, tol=1e-8, maxit=300, seed=6)
        X = torch.zeros((s.n, nr), dtype=torch.float64, device="cuda")
        rd = h.solve_multi(_dev(Bm), X, tol=1e-8, maxit=300, seed=6)
    assert [r.iters for r in rh] == [r.iters for r in rd]
    np.testing.assert_array_equal(Xh, X.cpu().numpy())


def test_batch_of_blocks_and_single_handles(cuda_ok):
    """Two blocks of different systems and a one-column handle in one graph
    launch: each equals its own solve."""
    s1 = W.powerlaw(n=1 << 12, num_blocks=16, seed=3, lam=1e-8)
    s2 = W.powerlaw(n=3000, num_blocks=12, seed=4, lam=1e-8)
    B1, B2 = _rhs(s1, 8, 1), _rhs(s2, 4, 2)
    with B.Handle.from_system(s1) as h1, B.Handle.from_system(s2) as h2, \
            h1.multi(8) as m1, h2.multi(4) as m2, B.Handle.from_system(s2) as single:
        bs = [_dev(B1), _dev(B2), _dev(s2.b)]
        xs = [torch.zeros((s1.n, 8), dtype=torch.float64, device="cuda"),
              torch.zeros((s2.n, 4), dtype=torch.float64, device="cuda"),
              torch.zeros(s2.n, dtype=torch.float64, device="cuda")]
        with B.Batch([m1, m2, single]) as bt:
            st, res = bt.solve(bs, xs, tol=1e-8, maxit=50000, seed=9)
        assert st == B.OK
        cols1 = m1.multi_results()
        assert res[0].iters == max(r.iters for r in cols1) and res[0].converged
        X1 = torch.zeros((s1.n, 8), dtype=torch.float64, device="cuda")
        r1 = m1.solve_multi(bs[0], X1, tol=1e-8, maxit=50000, seed=9)
        assert [r.iters for r in r1] == [r.iters for r in cols1]
        assert torch.equal(X1, xs[0])
        X2 = torch.zeros((s2.n, 4), dtype=torch.float64, device="cuda")
        m2.solve_multi(bs[1], X2, tol=1e-8, maxit=50000, seed=9)
        assert torch.equal(X2, xs[1])
        x3 = torch.zeros(s2.n, dtype=torch.float64, device="cuda")
        single.solve(bs[2], x3, tol=1e-8, maxit=50000, seed=9)
        assert torch.equal(x3, xs[2])


def test_full_size_columns_follow_the_oracle(cuda_ok):
    """n = 2^20 power-law system, a block of 16 right-hand sides: two of its
    columns over 3 whole iterations against the oracle (the sampled outputs
    the oracle computes in seconds at this size)."""
    s = W.powerlaw(n=1 << 20, num_blocks=4096, seed=1, lam=1e-8)
    nr, iters = 16, 3
    Bm = _rhs(s, nr, seed=7)
    with B.Handle.from_system(s) as h0, h0.multi(nr) as h:
        X = torch.zeros((s.n, nr), dtype=torch.float64, device="cuda")
        res = h.solve_multi(_dev(Bm), X, tol=0.0, maxit=iters, seed=1)
        Xh = X.cpu().numpy()
    for j in (0, 11):
        o = oracle.solve(s, b=Bm[:, j], maxit=iters, tol=0.0, seed=1)
        assert res[j].iters == iters
        assert abs(res[j].rrn - o.rrn) <= 1e-12 * o.rrn
        assert np.linalg.norm(Xh[:, j] - o.x) / np.linalg.norm(o.x) <= 1e-9
        np.testing.assert_array_equal(Xh[:, j], o.x)


def test_refusals(cuda_ok):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=3, lam=1e-8)
    with B.Handle.from_system(s) as h0:
        for bad in (3, 1, 64):
            with pytest.raises(B.RorbkError) as e:
                h0.multi(bad)
            assert e.value.status == -1
        with h0.multi(4) as h:
            x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
            with pytest.raises(B.RorbkError) as e:
                h.solve(_dev(s.b), x, maxit=2)
            assert e.value.status == -1
            with pytest.raises(B.RorbkError) as e:
                h.multi(2)
            assert e.value.status == -1
            X = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda")
            Bm = _dev(np.repeat(s.b[:, None], 4, axis=1))
            with pytest.raises(B.RorbkError) as e:
                h.solve_multi(Bm, X, maxit=2, precision=B.PREC_MIXED)      # not set up for it
            assert e.value.status == -7
    d = W.gaussian_dense(300, 80, seed=4, num_blocks=3)
    with B.Handle.from_system(d) as hd:
        with pytest.raises(B.RorbkError) as e:
            hd.multi(4)
        assert e.value.status == -7


@pytest.mark.parametrize("nr", [4, 16])
@pytest.mark.parametrize("name", ["powerlaw16k", "ragged"])
def test_block_residual_equals_one_column_residuals(cuda_ok, nr, name):
    """R = B - A X in one pass for all columns: every column bit for bit the
    one-column residual (FP64 chains, and FP32 chains of the mixed form), and
    ||r_j||^2 to rounding (summed in another order)."""
    s = CASES[name]()
    Bm = _rhs(s, nr, seed=5)
    rng = np.random.default_rng(6)
    Xm = rng.standard_normal((s.n, nr))
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h0, h0.multi(nr) as h:
        R = torch.full((s.m, nr), np.nan, dtype=torch.float64, device="cuda")
        rr = h.residual_multi(_dev(Bm), _dev(Xm), R)
        R32 = torch.full((s.m, nr), np.nan, dtype=torch.float32, device="cuda")
        rr32 = h.residual_multi(_dev(Bm, torch.float32), _dev(Xm, torch.float32), R32,
                                precision=B.PREC_MIXED)
        for j in range(nr):
            r = torch.empty(s.m, dtype=torch.float64, device="cuda")
            rr1 = h0.residual(_dev(Bm[:, j]), _dev(Xm[:, j]), r)
            assert torch.equal(R[:, j], r), j
            assert rr[j] == pytest.approx(rr1, rel=1e-13)
            r32 = torch.empty(s.m, dtype=torch.float32, device="cuda")
            rr1 = h0.residual32(_dev(Bm[:, j], torch.float32), _dev(Xm[:, j], torch.float32), r32)
            assert torch.equal(R32[:, j], r32), j
            assert rr32[j] == pytest.approx(rr1, rel=1e-5)
