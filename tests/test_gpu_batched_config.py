"""The batched configuration: power-law systems drawn as the benchmark draws
them (n ~ U[5000, 200000], 3-50 off-diagonals per row, blocks of 256 rows),
each a block of 16 right-hand sides, together with a dense wide system whose
limit is the minimum-norm solution (Lemma 2), in one graph launch.

- Two of the 256 systems (the first and the smallest) over 100 iterations in
  one launch: every column's iterate equals the FP64 oracle's one-column run
  of that right-hand side bit for bit (and within the 1e-9 parity bound), and
  the batch equals the blocks' own solves, whose traces give the draws and
  top-K sets of a column equal to the oracle's.
- The dense wide member (m = 512, n = 20,000, A = U diag(s) V^T with s from 1
  to 0.1), solved in the same launch to 1e-12 from x0 = 0: within 1e-8 of the
  minimum-norm solution A+ b (numpy lstsq) and in range(A^T).
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


def test_batched_configuration_members_follow_the_oracle(cuda_ok):
    sizes = W.batched_sizes(256)
    pick = [0, int(np.argmin(sizes))]
    systems = [W.batched_system(i, int(sizes[i])) for i in pick]
    nr, iters = 16, 100
    Bs = [W.rhs_block(q, nr, seed=500 + i) for q, i in zip(systems, pick)]
    d = W.dense_usv(512, 20_000, seed=6, smin=0.1, block_rows=256, lam=1e-12, tol=1e-12)
    hs = [B.Handle.from_system(q) for q in systems]
    blocks = [h.multi(nr) for h in hs]
    hd = B.Handle.from_system(d)
    try:
        xs = [torch.zeros((q.n, nr), dtype=torch.float64, device="cuda") for q in systems]
        xd = torch.zeros(d.n, dtype=torch.float64, device="cuda")
        with B.Batch(blocks + [hd]) as bt:
            st, res = bt.solve([_dev(b) for b in Bs] + [_dev(d.b)], xs + [xd], tol=0.0, maxit=iters,
                               seed=4)
        assert all(r.iters == iters for r in res)
        # each block equals its own solve, whose traces hold the draws and top-K sets
        for q, blk, Bm, xb in zip(systems, blocks, Bs, xs):
            K = blk.info.dyn_rows
            keep, trs = [], []
            for _ in range(nr):
                tau = torch.full((iters * 3,), -1, dtype=torch.int64, device="cuda")
                I = torch.full((iters * K,), -1, dtype=torch.int32, device="cuda")
                tr = B.Trace()
                tr.capacity, tr.tau, tr.I = iters, tau.data_ptr(), I.data_ptr()
                keep.append((tau, I))
                trs.append(tr)
            X = torch.zeros((q.n, nr), dtype=torch.float64, device="cuda")
            blk.solve_multi(_dev(Bm), X, tol=0.0, maxit=iters, seed=4, traces=trs)
            assert torch.equal(X, xb)
            for j in (0, 7, 15):
                o = oracle.solve(q, b=Bm[:, j], maxit=iters, tol=0.0, seed=4, trace_tau=True,
                                 trace_I=True)
                xj = xb[:, j].cpu().numpy()
                assert np.linalg.norm(xj - o.x) / np.linalg.norm(o.x) <= 1e-9
                np.testing.assert_array_equal(xj, o.x)
                np.testing.assert_array_equal(keep[j][0].cpu().numpy().reshape(iters, 3), o.tau)
                np.testing.assert_array_equal(keep[j][1].cpu().numpy().reshape(iters, K), o.I)
    finally:
        for blk in blocks:
            blk.close()
        for h in hs:
            h.close()
        hd.close()


def test_dense_wide_member_reaches_the_minimum_norm_solution(cuda_ok):
    """Lemma 2 in a batch: from x0 = 0 the dense wide member's iterates stay in
    range(A^T) and converge to A+ b."""
    s1 = W.batched_system(3, 5000)
    d = W.dense_usv(512, 20_000, seed=6, smin=0.1, block_rows=256, lam=1e-12, tol=1e-12)
    h1 = B.Handle.from_system(s1)
    b1 = h1.multi(4)
    hd = B.Handle.from_system(d)
    try:
        Bm = W.rhs_block(s1, 4, seed=2)
        x1 = torch.zeros((s1.n, 4), dtype=torch.float64, device="cuda")
        xd = torch.zeros(d.n, dtype=torch.float64, device="cuda")
        with B.Batch([b1, hd]) as bt:
            st, res = bt.solve([_dev(Bm), _dev(d.b)], [x1, xd], tol=1e-12, maxit=20000, seed=1)
        assert res[1].converged, res[1].rrn
        x = xd.cpu().numpy()
        xmn = np.linalg.lstsq(d.dense, d.b, rcond=None)[0]
        assert np.linalg.norm(x - xmn) / np.linalg.norm(xmn) <= 1e-8
        Q, _ = np.linalg.qr(d.dense.T)
        assert np.linalg.norm(x - Q @ (Q.T @ x)) <= 1e-10 * np.linalg.norm(x)
    finally:
        b1.close()
        h1.close()
        hd.close()
