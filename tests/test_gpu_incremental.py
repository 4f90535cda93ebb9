"""Incremental residual (RORBK_RESIDUAL_INCREMENTAL): r -= A dx from the
iteration's change log instead of r = b - A x over all of A.  The iterates
carry the rounding drift of the updates and of the atomic adds, so they are
compared with tolerances; what must hold exactly:
  - with refresh = 1 every residual is exact, and the solve is the EXACT
    mode's solve bit for bit (the gating of the two residual kernels);
  - with a log too small for an iteration's changes (n_static = 64) every
    residual falls back to the exact one, again bit for bit;
  - a solve stops only on an exact residual: the relative residual measured
    on the host in FP64 is at the tolerance."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

INC = B.RESIDUAL_INCREMENTAL


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _rrn(s, x):
    A = sp.csr_matrix((s.values.astype(np.float64), s.col_idx, s.row_ptr), shape=(s.m, s.n))
    return float(np.linalg.norm(A @ x - s.b) / np.linalg.norm(s.b))


def _solve(h, s, **kw):
    x = torch.empty(s.n, dtype=torch.float64, device="cuda")
    res = h.solve(_dev(s.b), x, **kw)
    return x, res


@pytest.mark.parametrize("n,blocks", [(1 << 14, 64), (1 << 16, 256)])
def test_converges_on_an_exact_residual(cuda_ok, n, blocks):
    s = W.powerlaw(n=n, num_blocks=blocks, seed=5, lam=1e-8)
    with B.Handle.from_system(s) as h:
        xe, re = _solve(h, s, tol=1e-8, maxit=200000, seed=3)
        xi, ri = _solve(h, s, tol=1e-8, maxit=200000, seed=3, residual_mode=INC)
    assert re.converged and ri.converged
    assert ri.rrn <= 1e-8
    assert _rrn(s, xi.cpu().numpy()) <= 1.001e-8
    # the same method up to rounding: the iteration counts stay close
    assert abs(ri.iters - re.iters) <= 0.05 * re.iters + 5, (ri.iters, re.iters)


def test_first_100_iterates_follow_the_oracle(cuda_ok):
    """Rounding drift in r changes no top-K set on these inputs: the iterate
    after 1, 10 and 100 iterations is the oracle's within 1e-9."""
    s = W.powerlaw(n=1 << 14, num_blocks=64, seed=5, lam=1e-8)
    with B.Handle.from_system(s) as h:
        for its in (1, 10, 100):
            x, r = _solve(h, s, tol=0.0, maxit=its, seed=9, residual_mode=INC, refresh=1000)
            o = oracle.solve(s, maxit=its, tol=0.0, seed=9)
            assert r.iters == o.iters == its
            xo = o.x
            rel = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
            assert rel <= 1e-9, (its, rel)


def test_refresh_one_is_the_exact_solve(cuda_ok):
    s = W.powerlaw(n=1 << 13, num_blocks=32, seed=9, lam=1e-8)
    with B.Handle.from_system(s) as h:
        xe, re = _solve(h, s, tol=1e-10, maxit=50000, seed=4)
        xi, ri = _solve(h, s, tol=1e-10, maxit=50000, seed=4, residual_mode=INC, refresh=1)
    assert ri.iters == re.iters and ri.rrn == re.rrn
    assert torch.equal(xi, xe)


def test_overflowing_log_falls_back_to_the_exact_residual(cuda_ok):
    """64 static updates per iteration log more changes than the log holds:
    every residual is then formed exactly."""
    s = W.powerlaw(n=1 << 14, num_blocks=64, seed=5, lam=1e-8)
    with B.Handle.from_system(s) as h:
        xe, re = _solve(h, s, tol=0.0, maxit=60, seed=2, n_static=64)
        xi, ri = _solve(h, s, tol=0.0, maxit=60, seed=2, n_static=64, residual_mode=INC)
    assert ri.iters == re.iters == 60
    assert torch.equal(xi, xe)


def test_mixed_precision_incremental(cuda_ok):
    s = W.powerlaw(n=1 << 16, num_blocks=256, seed=5, lam=1e-8)
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h:
        xe, re = _solve(h, s, tol=1e-8, maxit=200000, seed=3, precision=B.PREC_MIXED)
        xi, ri = _solve(h, s, tol=1e-8, maxit=200000, seed=3, precision=B.PREC_MIXED,
                        residual_mode=INC)
    assert re.converged and ri.converged
    assert _rrn(s, xi.cpu().numpy()) <= 1.001e-8
    assert abs(ri.iters - re.iters) <= 0.05 * re.iters + 50, (ri.iters, re.iters)


def test_host_loop_incremental(cuda_ok):
    s = W.powerlaw(n=1 << 14, num_blocks=64, seed=5, lam=1e-8)
    with B.Handle.from_system(s) as h:
        xi, ri = _solve(h, s, tol=1e-8, maxit=200000, seed=3, residual_mode=INC, host_loop=1,
                        poll=32)
    assert ri.converged and _rrn(s, xi.cpu().numpy()) <= 1.001e-8


def test_a_later_exact_solve_is_unchanged(cuda_ok):
    """An incremental solve leaves nothing behind that changes the next
    EXACT solve of the same handle."""
    s = W.powerlaw(n=1 << 13, num_blocks=32, seed=9, lam=1e-8)
    with B.Handle.from_system(s) as h:
        x1, r1 = _solve(h, s, tol=1e-10, maxit=50000, seed=4)
        _solve(h, s, tol=1e-10, maxit=50000, seed=4, residual_mode=INC)
        x2, r2 = _solve(h, s, tol=1e-10, maxit=50000, seed=4)
    assert r1.iters == r2.iters and torch.equal(x1, x2)


def test_rejected_combinations(cuda_ok):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=3, lam=1e-8)
    with B.Handle.from_system(s) as h:
        x = torch.empty(s.n, dtype=torch.float64, device="cuda")
        with pytest.raises(B.RorbkError):
            h.solve(_dev(s.b), x, tol=1e-8, maxit=10, residual_mode=INC,
                    dist_mode=B.DIST_RESIDUAL_WEIGHTED)
        with pytest.raises(B.RorbkError):
            h.solve(_dev(s.b), x, tol=1e-8, maxit=10, residual_mode=7)
        with pytest.raises(B.RorbkError):
            h.solve(_dev(s.b), x, tol=1e-8, maxit=10, residual_mode=INC, refresh=-1)
    d = W.gaussian_dense(300, 60, seed=3, num_blocks=5, lam=1e-6)
    with B.Handle.from_system(d) as h:
        x = torch.empty(d.n, dtype=torch.float64, device="cuda")
        with pytest.raises(B.RorbkError):
            h.solve(_dev(d.b), x, tol=1e-8, maxit=10, residual_mode=INC)
