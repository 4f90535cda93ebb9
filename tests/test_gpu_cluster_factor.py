"""The cluster factor of large coupled sets (more rows of the dynamic block
share columns than one block's shared memory can factor).

On the 65,536-unknown power-law system with 256 blocks most dynamic blocks
couple more than 176 of their 256 rows; those are factored by a cluster of
thread blocks.  The cluster applies the same operations in the same order as
the one-block factorisation, so the iterates must still equal the FP64
oracle's (the test asserts the 1e-9 relative bound and, beyond it, equality).
"""
import numpy as np
import pytest

import oracle
from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def test_cluster_factor_iterates_equal_oracle(cuda_ok):
    s = W.powerlaw(n=1 << 16, num_blocks=256, seed=5, lam=1e-8)
    iters = 100
    with B.Handle.from_system(s) as h:
        K, n = h.info.dyn_rows, s.n
        tr = B.Trace()
        tau = torch.full((iters * 3,), -1, dtype=torch.int64, device="cuda")
        I = torch.full((iters * K,), -1, dtype=torch.int32, device="cuda")
        X = torch.zeros((iters, n), dtype=torch.float64, device="cuda")
        dyn = torch.zeros(iters * 4, dtype=torch.int32, device="cuda")
        tr.capacity, tr.tau, tr.I, tr.x, tr.dyn = (iters, tau.data_ptr(), I.data_ptr(),
                                                   X.data_ptr(), dyn.data_ptr())
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        res = h.solve(_dev(s.b), x, tol=0.0, maxit=iters, seed=7, trace=tr)
        torch.cuda.synchronize()
    d = dyn.cpu().numpy().reshape(iters, 4)
    nS = d[:, 2]
    used = int((d[:, 3] == -2).sum())
    assert used >= 5, (used, nS)                       # the cluster path ran
    assert ((d[:, 3] == -2) == ((nS > 176) & (nS <= 512))).all()
    o = oracle.solve(s, maxit=iters, tol=0.0, seed=7, trace_tau=True, trace_I=True, trace_x=True)
    assert res.iters == o.iters == iters
    np.testing.assert_array_equal(tau.cpu().numpy().reshape(iters, 3), o.tau)
    np.testing.assert_array_equal(I.cpu().numpy().reshape(iters, K), o.I)
    Xg = X.cpu().numpy()
    worst = max(np.linalg.norm(Xg[j] - o.x_trace[j]) / np.linalg.norm(o.x_trace[j])
                for j in range(iters))
    assert worst <= 1e-9, worst
    np.testing.assert_array_equal(Xg, o.x_trace)


def test_cluster_factor_mixed_solve_reaches_tolerance(cuda_ok):
    """The mixed form (FP32 inner iterations, FP64 factor) on the same system
    reaches the tolerance, measured in FP64 on the host."""
    import scipy.sparse as sp
    s = W.powerlaw(n=1 << 16, num_blocks=256, seed=5, lam=1e-8, tol=1e-8)
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(_dev(s.b), x, tol=s.tol, maxit=200000, seed=1, precision=B.PREC_MIXED)
    A = sp.csr_matrix((s.values.astype(np.float64), s.col_idx, s.row_ptr), shape=(s.m, s.n))
    xh = x.cpu().numpy()
    assert res.converged
    assert np.linalg.norm(A @ xh - s.b) / np.linalg.norm(s.b) <= 1.001e-8
