"""Residual-weighted draws (not in the paper, whose proposal P is static):
iteration j draws block t with weight Pbar_t * ||r_{B_t}||^2 from the
residual of iteration j-1.  The oracle defines the running sum of the weights
as the plain sequential sum; the GPU forms the block norms in the oracle's
order and the running sum in chunks of 64 blocks, which differs from the
sequential sum by rounding only (checked against a stated bound).  A draw can
therefore differ only when it lands within that rounding of a block boundary;
the iteration tests count such draws, replay the oracle with the GPU's blocks
when one occurs, and require the top-K sets and iterates to agree."""
import numpy as np
import pytest

import oracle
from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

WEIGHTED = B.DIST_RESIDUAL_WEIGHTED


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _trace(h, s, iters, seed, host_loop=0):
    K, n = h.info.dyn_rows, s.n
    tr = B.Trace()
    tau = torch.full((iters * 3,), -1, dtype=torch.int64, device="cuda")
    I = torch.full((iters * K,), -1, dtype=torch.int32, device="cuda")
    X = torch.zeros((iters, n), dtype=torch.float64, device="cuda")
    tr.capacity, tr.tau, tr.I, tr.x = iters, tau.data_ptr(), I.data_ptr(), X.data_ptr()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = h.solve(_dev(s.b), x, tol=0.0, maxit=iters, seed=seed, trace=tr, dist_mode=WEIGHTED,
                  host_loop=host_loop, poll=16)
    torch.cuda.synchronize()
    return res, tau.cpu().numpy().reshape(iters, 3), I.cpu().numpy().reshape(iters, K), X.cpu().numpy()


CASES = {
    "powerlaw16k": lambda: W.powerlaw(n=1 << 14, num_blocks=64, lam=1e-8),
    "laplace45": lambda: W.laplace2d(),
    "dense_tall": lambda: W.gaussian_dense(700, 120, seed=3, num_blocks=5, lam=1e-6),
}


@pytest.mark.parametrize("name,k", [("powerlaw16k", 64), ("powerlaw64k_4096", 4096), ("laplace45", 32)])
def test_weighted_cdf_within_rounding_of_the_sequential_sum(cuda_ok, name, k):
    """The GPU's chunked running sum against the oracle's sequential one on the
    same residual: every entry within 2 k 2^-53 cdf[k-1] (the summation error
    bound of both orders), and the block weights themselves exact."""
    s = (W.powerlaw(n=1 << 16, num_blocks=4096, lam=1e-8) if name == "powerlaw64k_4096"
         else CASES[name]())
    assert s.num_blocks == k
    rng = np.random.default_rng(17)
    r = rng.standard_normal(s.m) * 10.0 ** rng.uniform(-3, 0, s.m)
    with B.Handle.from_system(s) as h:
        gpu = h.weighted_cdf(_dev(r))
    Pbar, _, _ = oracle.proposal(oracle.orthogonality(s, k), s.n)
    ref = oracle.weighted_cdf(Pbar, oracle.block_norms(r, oracle.partition(s.m, k)))
    bound = 2 * k * 2.0 ** -53 * ref[-1]
    assert np.max(np.abs(gpu - ref)) <= bound, (np.max(np.abs(gpu - ref)), bound)
    assert gpu[0] == ref[0]                      # one weight: no sum yet


@pytest.mark.parametrize("name", sorted(CASES))
def test_weighted_iterations_equal_oracle(cuda_ok, name):
    s = CASES[name]()
    iters = 100
    with B.Handle.from_system(s) as h:
        res, tau, I, X = _trace(h, s, iters, seed=7)
    o = oracle.solve(s, maxit=iters, tol=0.0, seed=7, trace_tau=True, trace_I=True, trace_x=True,
                     dist_mode=oracle.RESIDUAL_WEIGHTED)
    assert res.iters == o.iters == iters
    near_boundary = int((tau != o.tau).sum())
    if near_boundary:
        # a draw within rounding of a boundary went the other way: replay the
        # oracle with the GPU's blocks; everything else must still agree
        print(f"{name}: {near_boundary} draw(s) within rounding of a boundary, replayed")
        assert near_boundary <= max(1, tau.size // 100)
        o = oracle.solve(s, maxit=iters, tol=0.0, seed=7, trace_tau=True, trace_I=True,
                         trace_x=True, dist_mode=oracle.RESIDUAL_WEIGHTED, force_tau=tau)
    np.testing.assert_array_equal(tau, o.tau)
    np.testing.assert_array_equal(I, o.I)
    worst = max(np.linalg.norm(X[j] - o.x_trace[j]) / np.linalg.norm(o.x_trace[j])
                for j in range(iters))
    assert worst <= 1e-9, worst
    np.testing.assert_array_equal(X, o.x_trace)


def test_weighted_draws_differ_from_paper_draws(cuda_ok):
    """The weighting is in effect: on a row-scaled system the drawn blocks
    differ from the static proposal's under the same Philox stream."""
    s = W.powerlaw(n=1 << 14, num_blocks=64, lam=1e-8)
    with B.Handle.from_system(s) as h:
        _, tau_w, _, _ = _trace(h, s, 50, seed=7)
    o = oracle.solve(s, maxit=50, tol=0.0, seed=7, trace_tau=True)
    assert (tau_w != o.tau).mean() > 0.5


def test_weighted_solve_to_tolerance_matches_oracle(cuda_ok):
    s = W.powerlaw(n=1 << 13, num_blocks=32, seed=9, lam=1e-8, tol=1e-8)
    o = oracle.solve(s, maxit=20000, seed=2, dist_mode=oracle.RESIDUAL_WEIGHTED)
    assert o.converged
    with B.Handle.from_system(s) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(_dev(s.b), x, tol=s.tol, maxit=20000, seed=2, dist_mode=WEIGHTED)
    assert res.converged
    # equal unless a draw landed within rounding of a block boundary (then the
    # runs part ways but both must reach the tolerance in a similar count)
    if res.iters == o.iters:
        np.testing.assert_array_equal(x.cpu().numpy(), o.x)
    else:
        assert abs(res.iters - o.iters) <= 0.1 * o.iters


def test_weighted_host_loop_equals_graph(cuda_ok):
    s = W.powerlaw(n=1 << 14, num_blocks=64, lam=1e-8)
    with B.Handle.from_system(s) as h:
        r1, t1, _, X1 = _trace(h, s, 40, seed=3)
        r2, t2, _, X2 = _trace(h, s, 40, seed=3, host_loop=1)
    np.testing.assert_array_equal(t1, t2)
    np.testing.assert_array_equal(X1, X2)


def test_weighted_needs_fp64(cuda_ok):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=3, lam=1e-8)
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        with pytest.raises(B.RorbkError) as e:
            h.solve(_dev(s.b), x, tol=1e-8, maxit=10, precision=B.PREC_MIXED, dist_mode=WEIGHTED)
        assert e.value.status == -7
