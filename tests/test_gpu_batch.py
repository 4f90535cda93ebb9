"""Many solves in one graph launch: clones (one per right-hand side) and
systems of different sizes.  Every solve of a batch must be the solve
rorbk_solve runs on its own -- same iterate bits, iterations and residual --
since the batch only places the same loops side by side in one graph."""
import numpy as np
import pytest

from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _single(h, b, tol, maxit, seed, sysid, precision=B.PREC_FP64, x0=None):
    x = torch.empty(h.info.n, dtype=torch.float64, device="cuda")
    res = h.solve(b, x, x0=x0, tol=tol, maxit=maxit, seed=seed, system_id=sysid,
                  precision=precision)
    return x, res


def test_clones_solve_each_rhs_like_a_single_solve(cuda_ok):
    """Four right-hand sides of one system: the source handle and three
    clones share the set-up and the sampled block stream (same system id)."""
    s = W.powerlaw(n=1 << 13, num_blocks=32, seed=9, lam=1e-8)
    rng = np.random.default_rng(31)
    A_rhs = [s.b] + [None] * 3
    with B.Handle.from_system(s) as h:
        import scipy.sparse as sp
        A = sp.csr_matrix((s.values.astype(np.float64), s.col_idx, s.row_ptr), shape=(s.m, s.n))
        for j in range(1, 4):
            A_rhs[j] = A @ rng.standard_normal(s.n)
        clones = [h.clone() for _ in range(3)]
        hs = [h] + clones
        bs = [_dev(v) for v in A_rhs]
        xs = [torch.empty(s.n, dtype=torch.float64, device="cuda") for _ in hs]
        with B.Batch(hs) as bt:
            st, res = bt.solve(bs, xs, tol=1e-8, maxit=100000, seed=3, system_ids=[7] * 4)
        assert st == B.OK
        for j in range(4):
            xr, rr = _single(h, bs[j], 1e-8, 100000, 3, 7)
            assert res[j].converged and rr.converged
            assert res[j].iters == rr.iters and res[j].rrn == rr.rrn
            assert torch.equal(xs[j], xr)
        for c in clones:
            c.close()


def test_systems_of_different_sizes_in_one_launch(cuda_ok):
    """Three systems of different sizes and one that stops at maxit: each
    solve equals its own single solve; the batch reports not-converged."""
    systems = [W.powerlaw(n=1 << 12, num_blocks=16, seed=3, lam=1e-8),
               W.powerlaw(n=3000, num_blocks=12, seed=4, lam=1e-8),
               W.laplace2d(g=20, num_blocks=8)]
    hs = [B.Handle.from_system(s) for s in systems]
    try:
        bs = [_dev(s.b) for s in systems]
        xs = [torch.empty(s.n, dtype=torch.float64, device="cuda") for s in systems]
        with B.Batch(hs) as bt:
            st, res = bt.solve(bs, xs, tol=1e-10, maxit=400, seed=11, system_ids=[0, 1, 2])
        assert st == B.NOT_CONVERGED
        for i, (h, s) in enumerate(zip(hs, systems)):
            xr, rr = _single(h, bs[i], 1e-10, 400, 11, i)
            assert res[i].iters == rr.iters and res[i].rrn == rr.rrn
            assert res[i].converged == rr.converged
            assert torch.equal(xs[i], xr)
        assert not res[2].converged and res[2].iters == 400
    finally:
        for h in hs:
            h.close()


def test_mixed_precision_batch_matches_single_mixed_solves(cuda_ok):
    s = W.powerlaw(n=1 << 13, num_blocks=32, seed=9, lam=1e-8)
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h:
        c = h.clone()
        b = _dev(s.b)
        b2 = _dev(2.0 * s.b)
        xs = [torch.empty(s.n, dtype=torch.float64, device="cuda") for _ in range(2)]
        with B.Batch([h, c], precision=B.PREC_MIXED) as bt:
            st, res = bt.solve([b, b2], xs, tol=1e-8, maxit=100000, seed=2)
        for j, bj in enumerate((b, b2)):
            xr, rr = _single(h, bj, 1e-8, 100000, 2, 0, precision=B.PREC_MIXED)
            assert res[j].iters == rr.iters and res[j].refinements == rr.refinements
            assert torch.equal(xs[j], xr)
        c.close()


def test_clone_outlives_its_source(cuda_ok):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=3, lam=1e-8)
    h = B.Handle.from_system(s)
    b = _dev(s.b)
    x_ref, r_ref = _single(h, b, 1e-10, 10000, 1, 0)
    c = h.clone()
    h.close()
    x, r = _single(c, b, 1e-10, 10000, 1, 0)
    assert r.iters == r_ref.iters and torch.equal(x, x_ref)
    c.close()


def test_batch_rejects_bad_arguments(cuda_ok):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=3, lam=1e-8)
    with B.Handle.from_system(s) as h:
        with pytest.raises(B.RorbkError):
            B.Batch([h, h])                              # the same handle twice
        with pytest.raises(B.RorbkError):
            B.Batch([h], precision=B.PREC_MIXED)         # not set up for mixed
        with B.Batch([h]) as bt:
            x = torch.empty(s.n, dtype=torch.float64, device="cuda")
            opt_bad = dict(tol=1e-8, maxit=10)
            bt.precision = B.PREC_MIXED                  # options disagree with the batch
            with pytest.raises(B.RorbkError):
                bt.solve([_dev(s.b)], [x], **opt_bad)
