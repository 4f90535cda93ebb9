"""Algorithm 3 on the GPU: flexible AB-GMRES whose preconditioner is a
bounded ROR-BK solve.  Compared with the FP64 oracle's run of the same
algorithm (its inner solves are bit-exact; the Arnoldi inner products are
summed in another order, so results agree to rounding), and with what the
paper states: x lies in range(A^T), so a wide system gives the minimum-norm
solution."""
import numpy as np
import pytest

import oracle
from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def test_fabgmres_matches_oracle_on_laplacian(cuda_ok):
    s = W.laplace2d(g=12, num_blocks=4)
    xo, outer, inner, rrn_o, est, st = oracle.fabgmres(s, tol=1e-10, maxit=60, eta=1e-1, lmax=50)
    with B.Handle.from_system(s) as h:
        x = torch.empty(s.n, dtype=torch.float64, device="cuda")
        res = h.fabgmres(_dev(s.b), x, tol=1e-10, maxit=60, eta=1e-1, lmax=50)
    xg = x.cpu().numpy()
    assert res.converged and res.rrn <= 1e-10
    assert abs(res.iters - outer) <= 1
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-8
    true = np.linalg.norm(s.b - s.to_dense() @ xg) / np.linalg.norm(s.b)
    assert true == pytest.approx(res.rrn, rel=1e-9)


def test_fabgmres_wide_dense_gives_min_norm_solution(cuda_ok):
    s = W.gaussian_dense(80, 200, seed=6, num_blocks=4, lam=1e-10)
    with B.Handle.from_system(s) as h:
        x = torch.empty(s.n, dtype=torch.float64, device="cuda")
        res = h.fabgmres(_dev(s.b), x, tol=1e-11, maxit=40, eta=1e-2, lmax=200)
    assert res.converged
    x_mn = np.linalg.lstsq(s.dense, s.b, rcond=None)[0]
    assert np.linalg.norm(x.cpu().numpy() - x_mn) / np.linalg.norm(x_mn) <= 1e-8


@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_MIXED])
def test_fabgmres_powerlaw_reaches_tolerance(cuda_ok, precision):
    """On a row-scaled power-law system the outer GMRES reaches 1e-8 with
    FP64 or mixed-precision inner solves; the residual is checked on the host."""
    import scipy.sparse as sp
    s = W.powerlaw(n=1 << 14, num_blocks=64, lam=1e-8, tol=1e-8)
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h:
        x = torch.empty(s.n, dtype=torch.float64, device="cuda")
        res = h.fabgmres(_dev(s.b), x, tol=1e-8, maxit=60, eta=1e-2, lmax=300, precision=precision)
    A = sp.csr_matrix((s.values.astype(np.float64), s.col_idx, s.row_ptr), shape=(s.m, s.n))
    xh = x.cpu().numpy()
    assert res.converged
    assert np.linalg.norm(A @ xh - s.b) / np.linalg.norm(s.b) <= 1.001e-8


def test_fabgmres_rejects_bad_arguments(cuda_ok):
    s = W.laplace2d(g=8, num_blocks=4)
    with B.Handle.from_system(s) as h:
        x = torch.empty(s.n, dtype=torch.float64, device="cuda")
        with pytest.raises(B.RorbkError):
            h.fabgmres(_dev(s.b), x, maxit=0)
