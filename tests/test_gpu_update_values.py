"""New values for a handle's A (rorbk_update_values) and set-up from device
arrays.  A refresh re-forms every value-dependent part of Algorithm 1's set-up
(proposal, static operators W_t, the SELL copy, row norms, the incremental
residual's column-major copy) with the set-up's own kernels, so a refreshed
handle equals a fresh set-up bit for bit: the proposal, the operators and whole
solves are compared exactly.  The differentiable solve keeps one handle per
SolveSpec and refreshes it on every forward."""
import numpy as np
import pytest

from paper_2510_02156_gb300 import autograd as AG
from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a, dtype=None):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=dtype)


def _other_values(s, seed):
    """The same pattern with new values (a row-wise rescaling and a random
    relative change of every entry), rounded like the system's own values."""
    rng = np.random.default_rng(seed)
    v = s.values.astype(np.float64) * (1.0 + 0.25 * rng.standard_normal(s.values.size))
    return v.astype(s.values.dtype)


def _solve(h, s, b, precision, residual_mode=B.RESIDUAL_EXACT, maxit=50_000):
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    r = h.solve(b, x, tol=1e-8, maxit=maxit, seed=4, precision=precision,
                residual_mode=residual_mode)
    return r, x


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_refreshed_handle_equals_a_fresh_set_up(cuda_ok, dtype):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=5, lam=1e-8)
    s = W.System(s.name, s.m, s.n, row_ptr=s.row_ptr, col_idx=s.col_idx,
                 values=s.values.astype(dtype), b=s.b, num_blocks=s.num_blocks, lam=s.lam, tol=s.tol)
    v2 = _other_values(s, 7)
    s2 = W.System(s.name + "-v2", s.m, s.n, row_ptr=s.row_ptr, col_idx=s.col_idx, values=v2,
                  b=s.b, num_blocks=s.num_blocks, lam=s.lam, tol=s.tol)
    b = _dev(s.b)
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h, \
            B.Handle.from_system(s2, precision=B.PREC_MIXED) as fresh:
        # the incremental residual's column-major copy exists before the refresh
        _solve(h, s, b, B.PREC_FP64, B.RESIDUAL_INCREMENTAL, maxit=5)
        h.update_values(_dev(v2))
        c1, r1 = h.proposal()
        c2, r2 = fresh.proposal()
        np.testing.assert_array_equal(c1, c2)
        np.testing.assert_array_equal(r1, r2)
        for t in (0, 7, 15):
            rows = h.info.max_block_rows
            np.testing.assert_array_equal(h.static_operator(t, rows), fresh.static_operator(t, rows))
        for prec in (B.PREC_FP64, B.PREC_MIXED):
            ra, xa = _solve(h, s2, b, prec)
            rb, xb = _solve(fresh, s2, b, prec)
            assert (ra.iters, ra.converged, ra.rrn) == (rb.iters, rb.converged, rb.rrn), prec
            assert torch.equal(xa, xb), prec
        # the incremental residual applies r -= A dx with atomic adds, whose
        # order varies from run to run: 40 iterations with no exact refresh
        # after the first agree to rounding, while a column-major copy left
        # with the old values would be off by the 25% change of every entry
        ra, xa = _solve(h, s2, b, B.PREC_FP64, B.RESIDUAL_INCREMENTAL, maxit=40)
        rb, xb = _solve(fresh, s2, b, B.PREC_FP64, B.RESIDUAL_INCREMENTAL, maxit=40)
        assert ra.iters == rb.iters == 40
        assert float(torch.linalg.norm(xa - xb) / torch.linalg.norm(xb)) <= 1e-10
        # and back to the first values from host memory
        h.update_values(s.values)
        with B.Handle.from_system(s, precision=B.PREC_MIXED) as first:
            ra, xa = _solve(h, s, b, B.PREC_FP64)
            rb, xb = _solve(first, s, b, B.PREC_FP64)
            assert ra.iters == rb.iters and torch.equal(xa, xb)


def test_refresh_reaches_clones_and_blocks(cuda_ok):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=6, lam=1e-8)
    v2 = _other_values(s, 8)
    s2 = W.System(s.name + "-v2", s.m, s.n, row_ptr=s.row_ptr, col_idx=s.col_idx, values=v2,
                  b=s.b, num_blocks=s.num_blocks, lam=s.lam, tol=s.tol)
    Bm = _dev(W.rhs_block(s2, 4, seed=9))
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h, \
            B.Handle.from_system(s2, precision=B.PREC_MIXED) as fresh:
        blk = h.multi(4)
        X = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda")
        blk.solve_multi(Bm, X, tol=1e-8, maxit=3, seed=2)       # its graph exists before the refresh
        cl = h.clone()
        b = _dev(s2.b)
        _solve(cl, s, b, B.PREC_FP64, B.RESIDUAL_INCREMENTAL, maxit=5)   # the clone's own CSC copy
        h.update_values(v2)
        # the clone's copy is formed again at its next incremental solve
        ra, xa = _solve(cl, s2, b, B.PREC_FP64, B.RESIDUAL_INCREMENTAL, maxit=40)
        rb, xb = _solve(fresh, s2, b, B.PREC_FP64, B.RESIDUAL_INCREMENTAL, maxit=40)
        assert ra.iters == rb.iters == 40
        assert float(torch.linalg.norm(xa - xb) / torch.linalg.norm(xb)) <= 1e-10
        ra, xa = _solve(cl, s2, b, B.PREC_FP64)
        rb, xb = _solve(fresh, s2, b, B.PREC_FP64)
        assert ra.iters == rb.iters and torch.equal(xa, xb)
        cl.close()
        fb = fresh.multi(4)
        for prec in (B.PREC_FP64, B.PREC_MIXED):
            X1 = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda")
            X2 = torch.zeros((s.n, 4), dtype=torch.float64, device="cuda")
            ra = blk.solve_multi(Bm, X1, tol=1e-8, maxit=50_000, seed=2, precision=prec)
            rb = fb.solve_multi(Bm, X2, tol=1e-8, maxit=50_000, seed=2, precision=prec)
            assert [r.iters for r in ra] == [r.iters for r in rb]
            assert torch.equal(X1, X2)
        blk.close()
        fb.close()


def test_refresh_refuses_bad_values_and_leaves_the_handle(cuda_ok):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=6, lam=1e-8)
    b = _dev(s.b)
    with B.Handle.from_system(s) as h:
        r0, x0 = _solve(h, s, b, B.PREC_FP64)
        bad = s.values.copy()
        bad[123] = np.nan
        with pytest.raises(B.RorbkError) as e:
            h.update_values(_dev(bad))
        assert e.value.status == -5                  # RORBK_ERR_NUMERIC
        other = np.float64 if s.values.dtype == np.float32 else np.float32
        with pytest.raises(B.RorbkError) as e:
            h.update_values(_dev(s.values.astype(other)))   # not the handle's value type
        assert e.value.status == -1
        r1, x1 = _solve(h, s, b, B.PREC_FP64)
        assert r1.iters == r0.iters and torch.equal(x1, x0)
        adj = h.setup_adjoint(s.num_blocks, s.lam)
        try:
            with pytest.raises(B.RorbkError) as e:
                adj.update_values(_dev(s.values.astype(np.float64)))
            assert e.value.status == -7              # RORBK_ERR_UNSUPPORTED
        finally:
            adj.close()


def test_set_up_from_device_arrays_equals_host_set_up(cuda_ok):
    s = W.powerlaw(n=1 << 13, num_blocks=32, seed=5, lam=1e-8)
    b = _dev(s.b)
    rp = _dev(s.row_ptr.astype(np.int32))
    ci = _dev(s.col_idx.astype(np.int32))
    with B.Handle.from_system(s) as h, \
            B.Handle(rp, ci, _dev(s.values), s.m, s.n, s.num_blocks, s.lam) as d:
        np.testing.assert_array_equal(h.proposal()[0], d.proposal()[0])
        ra, xa = _solve(h, s, b, B.PREC_FP64)
        rb, xb = _solve(d, s, b, B.PREC_FP64)
        assert ra.iters == rb.iters and torch.equal(xa, xb)


def test_differentiable_solve_keeps_one_handle(cuda_ok):
    """Forwards of one SolveSpec refresh its handle instead of setting up a
    new one, and give the gradients of fresh specs bit for bit, also when a
    second forward runs before the first one's backward."""
    s = W.powerlaw(n=2025, num_blocks=8, seed=3, lam=1e-8)
    x_t = torch.as_tensor(np.random.default_rng(30).standard_normal(s.n), device="cuda")
    vals = [s.values.astype(np.float64), _other_values(s, 31).astype(np.float64),
            _other_values(s, 32).astype(np.float64)]

    def grads(spec, v):
        vt = torch.tensor(v, dtype=torch.float64, device="cuda", requires_grad=True)
        bt = torch.tensor(s.b, dtype=torch.float64, device="cuda", requires_grad=True)
        x = AG.RorbkSolve.apply(vt, bt, spec)
        return x, vt, bt

    def spec_new():
        return AG.SolveSpec(np.asarray(s.row_ptr, np.int32), np.asarray(s.col_idx, np.int32), s.m, s.n,
                            s.num_blocks, s.lam, tol=1e-12)

    ref = []
    for v in vals:
        sp1 = spec_new()
        x, vt, bt = grads(sp1, v)
        (0.5 * ((x - x_t) ** 2).sum()).backward()
        ref.append((x.detach().clone(), vt.grad.clone(), bt.grad.clone()))
        sp1.close()
    spec = spec_new()
    for v, (xr, gvr, gbr) in zip(vals, ref):
        x, vt, bt = grads(spec, v)
        (0.5 * ((x - x_t) ** 2).sum()).backward()
        assert torch.equal(x.detach(), xr) and torch.equal(vt.grad, gvr) and torch.equal(bt.grad, gbr)
    # two forwards, then the backward of the first
    xa, va, ba = grads(spec, vals[0])
    xb, vb, bb = grads(spec, vals[1])
    (0.5 * ((xa - x_t) ** 2).sum()).backward()
    assert torch.equal(va.grad, ref[0][1]) and torch.equal(ba.grad, ref[0][2])
    (0.5 * ((xb - x_t) ** 2).sum()).backward()
    assert torch.equal(vb.grad, ref[1][1]) and torch.equal(bb.grad, ref[1][2])
    assert spec.setups == 1
    spec.close()
