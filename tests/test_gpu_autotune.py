"""Launch-shape tuning (rorbk_autotune / rorbk_set_tuning).  The tuned grids
are those that leave results unchanged, so a solve with the chosen shapes
equals the solve with the defaults bit for bit (one column: every shape; a
block: the block residual's grid only reorders its sums of squares, which
moves no stopping test here).  A cache file replays a choice without timing."""
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
        x1, it1 = solve()
        assert it1 == it0
        assert torch.equal(x1, x0)
        # replayed from the cache without timing
        h.set_tuning(None)
        t2 = h.autotune(b, precision=precision, iters=30, cache_file=cache)
        assert (t2.topk_blocks, t2.dyn_mark_blocks, t2.dyn_scatter_blocks, t2.residual_blocks) == \
            (t.topk_blocks, t.dyn_mark_blocks, t.dyn_scatter_blocks, t.residual_blocks)
        assert t2.us_tuned == pytest.approx(t.us_tuned, rel=1e-3)
        assert len(cache.read_text().splitlines()) == 1
        if nr:
            h.close()


def test_set_tuning_checks_its_argument(cuda_ok):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=2, lam=1e-8)
    with B.Handle.from_system(s) as h:
        t = B.Tuning()
        t.topk_blocks = -1
        with pytest.raises(B.RorbkError) as e:
            h.set_tuning(t)
        assert e.value.status == -1
        with pytest.raises(B.RorbkError):
            h.autotune(None, iters=5)
