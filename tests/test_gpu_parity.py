"""Parity of the CUDA FP64 path with the FP64 oracle, through the C ABI.

Each step of Algorithm 1 is compared element by element on the same seeded
inputs: the setup products (cdf of P, static operators W_t), the sampler,
one static update, the residual, the top-K set, one dynamic update, and the
whole iteration (x after each of the first 100 iterations, the tau and I
sequences, the final relative residual).  The FP64 path evaluates every
quantity in the oracle's order without contraction, so the expected
difference is zero; the tests assert the parity bound (relative 1e-9 per
iterate) and report the observed maximum.
"""
import numpy as np
import pytest

import oracle
from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

REL = 1e-9


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    d = np.linalg.norm(a - b)
    s = np.linalg.norm(b)
    return d / s if s > 0 else d


SYSTEMS = {
    "laplace45": lambda: W.laplace2d(),
    "powerlaw16k": lambda: W.powerlaw(n=1 << 14, num_blocks=64, lam=1e-8),
    "ragged": lambda: W.random_sparse(997, 600, 0.01, seed=7, num_blocks=13, lam=1e-6, empty_rows=9),
    "wide": lambda: W.random_sparse(300, 1000, 0.02, seed=8, num_blocks=5, lam=1e-6),
}


@pytest.fixture(scope="module", params=sorted(SYSTEMS))
def case(request, cuda_ok):
    s = SYSTEMS[request.param]()
    h = B.Handle.from_system(s)
    yield request.param, s, h
    h.close()


def test_setup_proposal_matches_oracle(case):
    name, s, h = case
    cdf, rs = h.proposal()
    rs_o = oracle.orthogonality(s, s.num_blocks)
    _, _, cdf_o = oracle.proposal(rs_o, s.n)
    np.testing.assert_allclose(rs, rs_o, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(cdf, cdf_o, rtol=1e-14)


def test_static_operators_match_oracle(case):
    name, s, h = case
    off = oracle.partition(s.m, s.num_blocks)
    ts = sorted(set([0, s.num_blocks - 1, s.num_blocks // 2]))
    for t in ts:
        sz = int(off[t + 1] - off[t])
        Wg = h.static_operator(t, sz)
        Wo = oracle.static_operator(s, s.num_blocks, t, s.lam)
        assert np.max(np.abs(Wg - Wo)) <= 1e-12 * max(1.0, np.max(np.abs(Wo))), (name, t)


def test_sampler_matches_oracle(case):
    name, s, h = case
    cdf, _ = h.proposal()
    for it in list(range(20)) + [2**40 + 3]:
        for l in range(3):
            assert h.sample(11, 5, it, l) == oracle.sample(cdf, 11, 5, it, l)


def test_static_update_matches_oracle(case):
    name, s, h = case
    rng = np.random.default_rng(3)
    x = rng.standard_normal(s.n)
    off = oracle.partition(s.m, s.num_blocks)
    for t in sorted(set([0, s.num_blocks - 1, 1 % s.num_blocks])):
        xd = dev(x)
        h.static_update(t, dev(s.b), xd)
        rows = np.arange(off[t], off[t + 1])
        xo = oracle.update_with_inverse(s, rows, oracle.static_operator(s, s.num_blocks, t, s.lam),
                                        s.b, x)
        assert rel(xd.cpu().numpy(), xo) <= 1e-13, (name, t)


def test_residual_matches_oracle(case):
    name, s, h = case
    x = np.random.default_rng(4).standard_normal(s.n)
    r = torch.empty(s.m, dtype=torch.float64, device="cuda")
    rr = h.residual(dev(s.b), dev(x), r)
    ro, rro = oracle.residual(s, s.b, x)
    np.testing.assert_array_equal(r.cpu().numpy(), ro)      # same order, no contraction
    assert rr == pytest.approx(rro, rel=1e-12)


def test_topk_matches_oracle_with_ties(case):
    name, s, h = case
    K = h.info.dyn_rows
    rng = np.random.default_rng(5)
    for trial in range(3):
        r = rng.standard_normal(s.m)
        if trial == 1:
            r = np.round(r * 4) / 4                 # many exact ties, both signs
        if trial == 2:
            r[:] = 0.0
            r[rng.choice(s.m, K // 2, replace=False)] = 1.0   # ties at zero for the rest
        I = torch.empty(K, dtype=torch.int32, device="cuda")
        h.topk(dev(r), I)
        np.testing.assert_array_equal(I.cpu().numpy(), oracle.topk(r, K))


def test_dynamic_update_matches_oracle(case):
    name, s, h = case
    K = h.info.dyn_rows
    rng = np.random.default_rng(6)
    x = rng.standard_normal(s.n)
    ro, _ = oracle.residual(s, s.b, x)
    I = oracle.topk(ro, K)
    xd = dev(x)
    h.dynamic_update(dev(I, torch.int32), dev(ro), xd)
    xo = oracle.update_with_cholesky(s, I, s.lam, ro[I], x)
    assert rel(xd.cpu().numpy(), xo) <= 1e-13


def _gpu_trace(h, s, iters, seed=0, x0=None, tol=0.0):
    K, n = h.info.dyn_rows, s.n
    tr = B.Trace()
    tau = torch.full((iters * 3,), -1, dtype=torch.int64, device="cuda")
    rrn = torch.full((iters,), float("nan"), dtype=torch.float64, device="cuda")
    I = torch.full((iters * K,), -1, dtype=torch.int32, device="cuda")
    X = torch.zeros((iters, n), dtype=torch.float64, device="cuda")
    tr.capacity, tr.tau, tr.rrn, tr.I, tr.x = iters, tau.data_ptr(), rrn.data_ptr(), I.data_ptr(), X.data_ptr()
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    res = h.solve(dev(s.b), x, x0=None if x0 is None else dev(x0), tol=tol, maxit=iters,
                  seed=seed, trace=tr)
    torch.cuda.synchronize()
    it = res.iters
    return (res, x.cpu().numpy(), tau.cpu().numpy()[: it * 3].reshape(it, 3),
            rrn.cpu().numpy()[:it], I.cpu().numpy()[: it * K].reshape(it, K), X.cpu().numpy()[:it])


def test_first_100_iterations_match_oracle(case):
    """The iterates stay within relative 1e-9 of the oracle's over the first
    100 iterations under the same Philox block sequence."""
    name, s, h = case
    iters = 100
    res, x, tau, rrn, I, X = _gpu_trace(h, s, iters, seed=7)
    o = oracle.solve(s, maxit=iters, tol=0.0, seed=7, trace_tau=True, trace_rrn=True,
                     trace_I=True, trace_x=True)
    assert res.iters == o.iters == iters
    np.testing.assert_array_equal(tau, o.tau)
    np.testing.assert_array_equal(I, o.I)
    worst = max(rel(X[j], o.x_trace[j]) for j in range(iters))
    assert worst <= REL, worst
    np.testing.assert_allclose(rrn, o.rrn_trace, rtol=1e-12)
    print(f"{name}: max relative iterate difference over {iters} iterations = {worst:.3e}")


def test_solve_to_tolerance_matches_oracle(cuda_ok):
    """Same iteration count and final RRN at convergence."""
    s = W.powerlaw(n=1 << 13, num_blocks=32, seed=9, lam=1e-8, tol=1e-8)
    o = oracle.solve(s, maxit=5000, seed=2)
    assert o.converged
    with B.Handle.from_system(s) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(dev(s.b), x, tol=s.tol, maxit=5000, seed=2)
    assert res.converged and res.iters == o.iters
    assert res.rrn == pytest.approx(o.rrn, rel=1e-9)
    assert rel(x.cpu().numpy(), o.x) <= REL
    assert rel(x.cpu().numpy(), s.x_true) < 1e-5


def test_host_buffers_equal_device_buffers(cuda_ok):
    s = W.laplace2d(g=20, num_blocks=10)
    with B.Handle.from_system(s) as h:
        xd = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        r1 = h.solve(dev(s.b), xd, tol=1e-6, maxit=300, seed=1)
        xh = np.zeros(s.n)
        r2 = h.solve_host(np.ascontiguousarray(s.b), xh, tol=1e-6, maxit=300, seed=1)
    assert r1.iters == r2.iters
    np.testing.assert_array_equal(xd.cpu().numpy(), xh)


def test_edge_cases(cuda_ok):
    s = W.laplace2d(g=9, num_blocks=4)
    with B.Handle.from_system(s) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(torch.zeros(s.m, dtype=torch.float64, device="cuda"), x, maxit=10)
        assert res.converged and res.iters == 0 and not x.any()
        res = h.solve(dev(s.b), x, x0=dev(s.x_true), tol=1e-10, maxit=10)
        assert res.converged and res.iters == 1
        res = h.solve(dev(s.b), x, tol=1e-12, maxit=0)
        assert res.iters == 0 and not res.converged
        o = oracle.solve(s, maxit=7, tol=0.0, n_static=0)
        res = h.solve(dev(s.b), x, tol=0.0, maxit=7, n_static=0)
        assert rel(x.cpu().numpy(), o.x) <= 1e-13
        # resume: 2 x 5 iterations == 10 iterations
        x10 = torch.zeros_like(x)
        h.solve(dev(s.b), x10, tol=0.0, maxit=10, seed=3)
        h.solve(dev(s.b), x, tol=0.0, maxit=5, seed=3)
        h.solve(dev(s.b), x, x0=x.clone(), tol=0.0, maxit=5, seed=3, start_iter=5)
        assert torch.equal(x, x10)


@pytest.mark.parametrize("k", [1, 81])
def test_extreme_partitions(cuda_ok, k):
    """k = 1 (one block, K = m) and k = m (one-row blocks, K = 1)."""
    s = W.laplace2d(g=9, num_blocks=k)
    o = oracle.solve(s, maxit=30, tol=0.0, seed=5)
    with B.Handle.from_system(s) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(dev(s.b), x, tol=0.0, maxit=30, seed=5)
    assert res.iters == 30
    assert rel(x.cpu().numpy(), o.x) <= REL


def test_errors_are_reported(cuda_ok):
    with pytest.raises(B.RorbkError) as e:
        B.Handle(np.array([0, 2, 3]), np.array([1, 0, 0]), np.array([1.0, 2.0, 3.0]), 2, 2, 1, 0.0)
    assert e.value.status == -1
    A = np.ones((8, 3))
    s = W.System("dup", 8, 3, row_ptr=np.arange(0, 25, 3), col_idx=np.tile(np.arange(3), 8).astype(np.int32),
                  values=A.ravel(), b=A @ np.ones(3), num_blocks=2, lam=0.0)
    with pytest.raises(B.RorbkError) as e:
        B.Handle.from_system(s)
    assert e.value.status == -4


def test_full_size_powerlaw_iterations_and_residual(cuda_ok):
    """The 2^20-row power-law system with 4096 blocks: the setup cdf, a full
    residual, and the first 3 iterations against the oracle."""
    s = W.powerlaw(n=1 << 20, num_blocks=4096, lam=1e-8)
    with B.Handle.from_system(s) as h:
        cdf, _ = h.proposal()
        _, _, cdf_o = oracle.proposal(oracle.orthogonality(s, 4096), s.n)
        np.testing.assert_allclose(cdf, cdf_o, rtol=1e-14)
        xr = np.random.default_rng(0).standard_normal(s.n)
        r = torch.empty(s.m, dtype=torch.float64, device="cuda")
        h.residual(dev(s.b), dev(xr), r)
        np.testing.assert_array_equal(r.cpu().numpy(), oracle.residual(s, s.b, xr)[0])
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        h.solve(dev(s.b), x, tol=0.0, maxit=3, seed=1)
    o = oracle.solve(s, maxit=3, tol=0.0, seed=1)
    assert rel(x.cpu().numpy(), o.x) <= REL


def test_host_loop_equals_graph_loop(cuda_ok):
    """The host-driven loop (profiling mode) and the device-side graph loop
    run the same iterations and give the same x."""
    s = W.powerlaw(n=1 << 13, num_blocks=32, seed=4, lam=1e-8, tol=1e-6)
    with B.Handle.from_system(s) as h:
        x1 = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        x2 = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        r1 = h.solve(dev(s.b), x1, tol=s.tol, maxit=3000, seed=6)
        r2 = h.solve(dev(s.b), x2, tol=s.tol, maxit=3000, seed=6, host_loop=1, poll=7)
    assert r1.iters == r2.iters and r1.converged and r2.converged
    assert torch.equal(x1, x2)


def test_dense_coupling_takes_both_factor_schedules(cuda_ok):
    """A matrix whose dynamic rows couple densely (every row shares columns
    with every other) exercises the column-by-column factorisation; the
    power-law system exercises the tree-level one.  Both agree with the
    oracle."""
    s = W.random_sparse(400, 120, 0.3, seed=13, num_blocks=8, lam=1e-6)
    o = oracle.solve(s, maxit=20, tol=0.0, seed=2)
    with B.Handle.from_system(s) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        h.solve(dev(s.b), x, tol=0.0, maxit=20, seed=2)
    assert rel(x.cpu().numpy(), o.x) <= REL


def test_residual_fp32_subnormal_and_signed_zero_values(cuda_ok):
    """FP32-stored values are widened exactly (normal, subnormal, +-0): the
    FP64 residual still equals the oracle's bit for bit."""
    s = W.random_sparse(500, 300, 0.05, seed=21, num_blocks=5)
    v = s.values.copy()
    rng = np.random.default_rng(0)
    pick = rng.choice(len(v), len(v) // 3, replace=False)
    v[pick[: len(pick) // 2]] *= 1e-41                  # FP32 subnormals
    v[pick[len(pick) // 2:][:5]] = -0.0
    s.values = v.astype(np.float32)
    x = rng.standard_normal(s.n) * 1e30
    with B.Handle.from_system(s) as h:
        r = torch.empty(s.m, dtype=torch.float64, device="cuda")
        h.residual(dev(s.b), dev(x), r)
    np.testing.assert_array_equal(r.cpu().numpy(), oracle.residual(s, s.b, x)[0])


def test_mixed_precision_reaches_fp64_tolerance(cuda_ok):
    """FP64 refinement around FP32 ROR-BK reaches ||b - A x|| / ||b|| <= tol in
    FP64 on the power-law system; its error against the FP64 oracle's
    solution is reported (there is no exact pin for the mixed form)."""
    s = W.powerlaw(n=1 << 13, num_blocks=32, seed=9, lam=1e-8, tol=1e-8)
    o = oracle.solve(s, maxit=5000, seed=2)
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(dev(s.b), x, tol=s.tol, maxit=20000, seed=2, precision=B.PREC_MIXED,
                      inner_tol=1e-4)
        xh = np.zeros(s.n)
        res2 = h.solve(dev(s.b), torch.zeros_like(x), tol=s.tol, maxit=20000, seed=2,
                       precision=B.PREC_MIXED, inner_tol=1e-4, host_loop=1, poll=16)
        x64 = torch.zeros_like(x)
        r64 = h.solve(dev(s.b), x64, tol=s.tol, maxit=5000, seed=2)
    xm = x.cpu().numpy()
    r_check = np.linalg.norm(s.b - s.to_dense() @ xm) / np.linalg.norm(s.b)
    assert res.converged and res.refinements >= 2 and r_check <= 1.001e-8, (res.iters, res.rrn, r_check)
    assert res2.iters == res.iters and res2.refinements == res.refinements
    assert r64.converged and r64.iters == o.iters
    err = rel(xm, o.x)
    print(f"mixed: {res.iters} inner iterations, {res.refinements} refinements, "
          f"rrn {res.rrn:.2e}, rel. difference to the FP64 oracle {err:.2e}")
    assert err < 1e-5
