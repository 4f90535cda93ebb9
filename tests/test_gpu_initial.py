"""Algorithm 2's initial solution on the GPU against the oracle and the
Remark after it: x0 = alpha y with y the row sum of one static block,
||b - A x0|| <= ||b||, and b - A x0 orthogonal to A y."""
import numpy as np
import pytest

import oracle
from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


@pytest.mark.parametrize("make,block", [
    (lambda: W.powerlaw(n=1 << 14, num_blocks=64, lam=1e-8), 5),
    (lambda: W.laplace2d(), 0),
    (lambda: W.gaussian_dense(700, 120, seed=3, num_blocks=5, lam=1e-6), 2),
])
def test_initial_solution_matches_oracle_and_remark(cuda_ok, make, block):
    s = make()
    with B.Handle.from_system(s) as h:
        off = np.concatenate([[0], np.cumsum([s.m // s.num_blocks + (t < s.m % s.num_blocks)
                                              for t in range(s.num_blocks)])])
        x0 = torch.empty(s.n, dtype=torch.float64, device="cuda")
        h.initial_solution(_dev(s.b), x0, block=block)
        xg = x0.cpu().numpy()
    xo = oracle.initial_solution(s, int(off[block]), int(off[block + 1] - off[block]))
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-12
    A = s.to_dense()
    y = A[off[block]:off[block + 1]].sum(axis=0)
    r0 = s.b - A @ xg
    assert np.linalg.norm(r0) <= np.linalg.norm(s.b)
    assert abs(r0 @ (A @ y)) <= 1e-9 * np.linalg.norm(r0) * np.linalg.norm(A @ y)


def test_initial_solution_starts_a_solve(cuda_ok):
    """Passed as x0, it is the start of the solve (the first iteration runs
    from it) and the solve reaches the tolerance."""
    s = W.powerlaw(n=1 << 13, num_blocks=32, seed=9, lam=1e-8, tol=1e-8)
    with B.Handle.from_system(s) as h:
        b = _dev(s.b)
        x0 = torch.empty(s.n, dtype=torch.float64, device="cuda")
        h.initial_solution(b, x0, block=3)
        x = torch.empty(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(b, x, x0=x0, tol=s.tol, maxit=20000, seed=2)
        o = oracle.solve(s, x0=x0.cpu().numpy(), maxit=20000, seed=2)
    assert res.converged and o.converged and res.iters == o.iters


def test_initial_solution_rejects_bad_block(cuda_ok):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=3, lam=1e-8)
    with B.Handle.from_system(s) as h:
        x0 = torch.empty(s.n, dtype=torch.float64, device="cuda")
        with pytest.raises(B.RorbkError):
            h.initial_solution(_dev(s.b), x0, block=16)
