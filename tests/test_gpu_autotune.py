"""Launch-shape tuning (rorbk_autotune / rorbk_set_tuning).  The tuned grids
are those that leave results unchanged, so a solve with the chosen shapes
equals the solve with the defaults bit for bit (one column: every shape; a
block: the block residual's grid only reorders its sums of squares, which
moves no stopping test here).  The graph's unroll (iterations per execution of
the WHILE body) runs the same iterations, including a loop that ends inside a
body.  A cache file replays a choice without timing."""
import numpy as np
import pytest

from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("nr", [0, 16])
@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_MIXED])
def test_tuned_shapes_leave_the_solve_unchanged(cuda_ok, tmp_path, nr, precision):
    s = W.powerlaw(n=1 << 14, num_blocks=64, seed=2, lam=1e-8, tol=1e-8)
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h0:
        h = h0.multi(nr) if nr else h0
        b = _dev(W.rhs_block(s, nr, seed=3)) if nr else _dev(s.b)
        shape = (s.n, nr) if nr else (s.n,)

        def solve():
            x = torch.zeros(shape, dtype=torch.float64, device="cuda")
            if nr:
                res = h.solve_multi(b, x, tol=1e-8, maxit=100000, seed=1, precision=precision)
            else:
                res = [h.solve(b, x, tol=1e-8, maxit=100000, seed=1, precision=precision)]
            return x, [r.iters for r in res]

        x0, it0 = solve()
        cache = tmp_path / "tune.txt"
        t = h.autotune(b, precision=precision, iters=30, cache_file=cache)
        assert t.us_default > 0 and t.us_tuned > 0 and t.us_tuned <= t.us_default * 1.0001
        assert min(t.topk_blocks, t.collect_blocks, t.dyn_mark_blocks, t.dyn_scatter_blocks) >= 1
        assert t.graph_unroll in (1, 2, 4, 8)
        x1, it1 = solve()
        assert it1 == it0
        assert torch.equal(x1, x0)
        # replayed from the cache without timing
        h.set_tuning(None)
        t2 = h.autotune(b, precision=precision, iters=30, cache_file=cache)
        assert (t2.topk_blocks, t2.dyn_mark_blocks, t2.dyn_scatter_blocks, t2.residual_blocks,
                t2.graph_unroll) == \
            (t.topk_blocks, t.dyn_mark_blocks, t.dyn_scatter_blocks, t.residual_blocks, t.graph_unroll)
        assert t2.us_tuned == pytest.approx(t.us_tuned, rel=1e-3)
        assert len(cache.read_text().splitlines()) == 1
        if nr:
            h.close()


@pytest.mark.parametrize("nr", [0, 16])
@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_MIXED])
def test_graph_unroll_runs_the_same_iterations(cuda_ok, nr, precision):
    s = W.powerlaw(n=1 << 14, num_blocks=64, seed=2, lam=1e-8, tol=1e-8)
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h0:
        h = h0.multi(nr) if nr else h0
        b = _dev(W.rhs_block(s, nr, seed=3)) if nr else _dev(s.b)
        shape = (s.n, nr) if nr else (s.n,)

        def solve(maxit):
            x = torch.zeros(shape, dtype=torch.float64, device="cuda")
            if nr:
                res = h.solve_multi(b, x, tol=1e-8, maxit=maxit, seed=1, precision=precision)
            else:
                res = [h.solve(b, x, tol=1e-8, maxit=maxit, seed=1, precision=precision)]
            return x, [(r.iters, r.status, r.converged, r.rrn) for r in res]

        # 37 iterations stop inside a body of 2, 3 or 8; the solve to the
        # tolerance stops wherever its stopping test fires
        ref = {mx: solve(mx) for mx in (37, 100000)}
        for u in (2, 3, 8):
            t = B.Tuning()
            t.graph_unroll = u
            h.set_tuning(t)
            for mx, (x0, info0) in ref.items():
                x, info = solve(mx)
                # a block's sums of squares come from a slice queue, in an
                # order that varies from run to run: its RRN to rounding
                assert [q[:3] for q in info] == [q[:3] for q in info0], (u, mx)
                for q, q0 in zip(info, info0):
                    assert q[3] == (pytest.approx(q0[3], rel=1e-13) if nr else q0[3]), (u, mx)
                assert torch.equal(x, x0), (u, mx)
        h.set_tuning(None)
        if nr:
            h.close()


def test_graph_unroll_keeps_the_trace(cuda_ok):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=2, lam=1e-8)
    with B.Handle.from_system(s) as h:
        K, iters = h.info.dyn_rows, 37

        def run():
            tr = B.Trace()
            tau = torch.full((iters * 3,), -1, dtype=torch.int64, device="cuda")
            rrn = torch.full((iters,), float("nan"), dtype=torch.float64, device="cuda")
            I = torch.full((iters * K,), -1, dtype=torch.int32, device="cuda")
            X = torch.zeros((iters, s.n), dtype=torch.float64, device="cuda")
            tr.capacity, tr.tau, tr.rrn, tr.I, tr.x = iters, tau.data_ptr(), rrn.data_ptr(), I.data_ptr(), \
                X.data_ptr()
            x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
            res = h.solve(_dev(s.b), x, tol=0.0, maxit=iters, seed=5, trace=tr)
            return res.iters, x, tau, rrn, I, X

        a = run()
        t = B.Tuning()
        t.graph_unroll = 8
        h.set_tuning(t)
        c = run()
        assert a[0] == c[0] == iters
        for u, v in zip(a[1:], c[1:]):
            assert torch.equal(u, v)


def test_set_tuning_checks_its_argument(cuda_ok):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=2, lam=1e-8)
    with B.Handle.from_system(s) as h:
        t = B.Tuning()
        t.topk_blocks = -1
        with pytest.raises(B.RorbkError) as e:
            h.set_tuning(t)
        assert e.value.status == -1
        for u in (-1, 17):
            t = B.Tuning()
            t.graph_unroll = u
            with pytest.raises(B.RorbkError):
                h.set_tuning(t)
        with pytest.raises(B.RorbkError):
            h.autotune(None, iters=5)
