"""Pins for the FP64 oracle against facts the paper and the mathematics fix.

None of these re-types the oracle's own formula: each compares it with a
closed form, an invariant, a library routine for a special case, or brute
force on a tiny input (see each test's docstring for the passage it pins).
"""
import os

import numpy as np
import pytest
import scipy.linalg
import scipy.sparse

import oracle
from paper_2510_02156_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------------- sampler
def test_philox_golden_kat():
    """Philox4x64-10 (Salmon et al. SC'11) published all-zero KAT."""
    for line in open(os.path.join(GOLDEN, "philox4x64_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        ctr = np.array([int(v) for v in f[0:4]], dtype=np.uint64)
        key = np.array([int(v) for v in f[4:6]], dtype=np.uint64)
        want = np.array([int(v, 16) for v in f[6:10]], dtype=np.uint64)
        assert (oracle.philox4x64_10(ctr, key) == want).all()


@pytest.mark.parametrize("seed", [0, 1, 12345])
def test_philox_matches_numpy(seed):
    """numpy.random.Philox is an independent Philox4x64-10; its counter is
    pre-incremented, so counter c-1 there gives block c here."""
    rng = np.random.default_rng(seed)
    for _ in range(50):
        ctr = [int(v) for v in rng.integers(0, 2**63, 4, dtype=np.int64)]
        ctr[0] = [0, 1, 2**64 - 1, ctr[0]][int(rng.integers(0, 4))]
        key = rng.integers(0, 2**63, 2, dtype=np.int64).astype(np.uint64)
        v = sum(c << (64 * i) for i, c in enumerate(ctr)) - 1
        v %= 2**256
        prev = np.array([(v >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
        ref = np.random.Philox(key=key, counter=prev).random_raw(4)
        got = oracle.philox4x64_10(np.array(ctr, dtype=np.uint64), key)
        assert (got == ref).all()


def test_sampler_distribution_chi2():
    """Algorithm 1 samples tau ~ P; a chi-square test over 200k counters."""
    import scipy.stats
    k = 7
    Pbar = np.array([0.5, 1.0, 2.0, 0.25, 3.0, 1.5, 0.75])
    cdf = np.cumsum(Pbar)
    n_draw = 200_000
    counts = np.zeros(k)
    lib = oracle.lib()
    c = np.ascontiguousarray(cdf)
    for it in range(n_draw // 2):
        for l in range(2):
            counts[lib.orc_sample(c.ctypes.data, k, 99, 3, it, l)] += 1
    expected = Pbar / Pbar.sum() * n_draw
    chi2 = ((counts - expected) ** 2 / expected).sum()
    assert scipy.stats.chi2.sf(chi2, k - 1) > 1e-4


def test_sampler_inverse_cdf_bruteforce():
    """tau is the first t with u * cdf[-1] < cdf[t], u from word 0 of the
    Philox block at counter (it, l, 0, 0), key (seed, sysid)."""
    cdf = np.cumsum(np.array([1.0, 0.0, 2.0, 0.5, 0.0, 1.0]))   # zero-mass blocks
    for it in range(300):
        for l in range(3):
            w = np.random.Philox(key=np.array([5, 9], dtype=np.uint64),
                                 counter=np.array([(it - 1) % 2**64 if it else 2**64 - 1,
                                                   l if it else (l - 1) % 2**64,
                                                   0 if (it or l) else 2**64 - 1,
                                                   0 if (it or l) else 2**64 - 1],
                                                  dtype=np.uint64)).random_raw(1)[0]
            u = float(int(w) >> 11) * 2.0 ** -53
            want = int(np.searchsorted(cdf, u * cdf[-1], side="right"))
            got = oracle.sample(cdf, 5, 9, it, l)
            assert got == want
            assert cdf[got] > (cdf[got - 1] if got else 0.0)   # never a zero-mass block


# --------------------------------------------------------------- partition
@pytest.mark.parametrize("m,k", [(2025, 32), (100, 7), (64, 64), (10, 1), (1 << 20, 4096)])
def test_partition_contiguous_uniform(m, k):
    """Algorithm 1's partition / Section 2: k contiguous blocks, each with at
    least floor(m/k) rows, covering all rows in order."""
    off = oracle.partition(m, k)
    sizes = np.diff(off)
    assert off[0] == 0 and off[-1] == m and len(sizes) == k
    assert (sizes >= m // k).all() and (sizes <= m // k + 1).all()
    assert (sizes[: m % k] == m // k + 1).all()


# ------------------------------------------------------- orthogonality / P
def _csr_system(Ad, k=2):
    sp = scipy.sparse.csr_matrix(Ad)
    sp.sort_indices()
    return W.System("t", Ad.shape[0], Ad.shape[1], row_ptr=sp.indptr.astype(np.int64),
                    col_idx=sp.indices.astype(np.int32), values=sp.data.astype(np.float64),
                    x_true=np.zeros(Ad.shape[1]), b=np.zeros(Ad.shape[0]), num_blocks=k)


def test_orthogonality_known_angles():
    """Section 2: C(i,j) is the |cosine| between block centroids (sums of the
    block's rows).  Centroids e1, e1+e2 and -e2 have cosines 1/sqrt2, 0, 1/sqrt2."""
    Ad = np.array([[1.0, 0, 0], [0.0, 0, 0],          # block 0 -> (1,0,0)
                   [0.5, 2, 0], [0.5, -1, 0],        # block 1 -> (1,1,0)
                   [0.0, -3, 0], [0.0, 1, 0]])       # block 2 -> (0,-2,0)
    Cm, rs = oracle.orthogonality(_csr_system(Ad), 3, full=True)
    h = 1 / np.sqrt(2)
    want = np.array([[1, h, 0], [h, 1, h], [0, h, 1]])
    np.testing.assert_allclose(Cm, want, rtol=0, atol=1e-15)
    np.testing.assert_allclose(rs, want.sum(1), rtol=1e-15)


def test_orthogonality_disjoint_supports_uniform_P():
    """Blocks with disjoint column supports are mutually orthogonal: C = I,
    so every Pbar_t = exp(-2/n) and P is uniform (Section 2 formula)."""
    rng = np.random.default_rng(0)
    k, s, n = 6, 4, 30
    Ad = np.zeros((k * s, n))
    for t in range(k):
        Ad[t * s:(t + 1) * s, t * 5:(t + 1) * 5] = rng.standard_normal((s, 5))
    Cm, rs = oracle.orthogonality(_csr_system(Ad, k), k, full=True)
    np.testing.assert_array_equal(Cm, np.eye(k))
    Pbar, P, cdf = oracle.proposal(rs, n)
    np.testing.assert_allclose(Pbar, np.exp(-2.0 / n), rtol=1e-15)
    np.testing.assert_allclose(P, 1.0 / k, rtol=1e-14)


def test_orthogonality_parallel_blocks():
    """Blocks whose centroids are (anti)parallel have C = all ones, so
    Pbar_t = exp(-2k/n)."""
    rng = np.random.default_rng(1)
    k, n = 5, 8
    v = rng.standard_normal(n)
    Ad = np.vstack([(t + 1) * (-1) ** t * v for t in range(k)])
    Cm, rs = oracle.orthogonality(_csr_system(Ad, k), k, full=True)
    np.testing.assert_allclose(Cm, np.ones((k, k)), rtol=1e-14)
    Pbar, P, _ = oracle.proposal(rs, n)
    np.testing.assert_allclose(Pbar, np.exp(-2.0 * k / n), rtol=1e-13)


def test_orthogonality_invariances_and_dense_equals_csr():
    """|cos| is invariant to a positive or negative scaling of a block and
    to the storage format; the zero centroid reads as orthogonal to all."""
    rng = np.random.default_rng(2)
    Ad = rng.standard_normal((12, 5)) * (rng.random((12, 5)) < 0.6)
    Ad[8:12] = 0.0                                     # block 2 has a zero centroid
    sysd = W.System("d", 12, 5, dense=Ad, x_true=np.zeros(5), b=np.zeros(12), num_blocks=3)
    C1, _ = oracle.orthogonality(_csr_system(Ad, 3), 3, full=True)
    C2, _ = oracle.orthogonality(sysd, 3, full=True)
    np.testing.assert_allclose(C1, C2, rtol=1e-14, atol=1e-15)
    Ad2 = Ad.copy()
    Ad2[0:4] *= -3.7
    C3, _ = oracle.orthogonality(_csr_system(Ad2, 3), 3, full=True)
    np.testing.assert_allclose(C1, C3, rtol=1e-13, atol=1e-15)
    assert C1[2, 2] == 1.0 and C1[2, 0] == 0.0 and C1[1, 2] == 0.0
    assert np.allclose(C1, C1.T) and (C1 >= 0).all() and (C1 <= 1 + 1e-15).all()


def test_proposal_normalised():
    """P = Pbar / sum(Pbar) sums to one; the cdf ends at sum(Pbar)."""
    rs = np.array([1.0, 3.5, 2.0, 1.25])
    Pbar, P, cdf = oracle.proposal(rs, 10)
    assert abs(P.sum() - 1) < 1e-15
    np.testing.assert_allclose(Pbar, [np.exp(-0.2), np.exp(-0.7), np.exp(-0.4), np.exp(-0.25)],
                               rtol=1e-15)
    assert cdf[-1] == pytest.approx(Pbar.sum(), rel=1e-15)


# ------------------------------------------------------------ residual/topk
def test_residual_matches_scipy():
    """r = b - A x against scipy.sparse's SpMV; ||r||^2 against numpy."""
    s = W.random_sparse(300, 200, 0.05, seed=3)
    x = np.random.default_rng(0).standard_normal(200)
    r, rr = oracle.residual(s, s.b, x)
    A = scipy.sparse.csr_matrix((s.values, s.col_idx, s.row_ptr), shape=(300, 200))
    np.testing.assert_allclose(r, s.b - A @ x, rtol=1e-13, atol=1e-13)
    assert rr == pytest.approx(float(r @ r), rel=1e-13)


@pytest.mark.parametrize("seed", range(5))
def test_topk_bruteforce_with_ties(seed):
    """Algorithm 1 top floor(m/k) of r_i^2; ties broken to the lower index,
    output ascending (brute force: stable sort on -|r|)."""
    rng = np.random.default_rng(seed)
    m = 500
    r = rng.integers(-20, 20, m).astype(np.float64)     # heavy exact ties, +-
    r[rng.choice(m, 40, replace=False)] = 0.0
    for K in [0, 1, 7, 63, 250, m]:
        got = oracle.topk(r, K)
        order = np.argsort(-np.abs(r), kind="stable")
        want = np.sort(order[:K])
        np.testing.assert_array_equal(got, want)


# ------------------------------------------------------------ factorisation
def test_cholesky_inverse_solve_match_lapack():
    """Cholesky, two triangular solves and the explicit inverse (Section 3.1
    stores (A A^T + mu I)^{-1}) against numpy/LAPACK."""
    rng = np.random.default_rng(4)
    B = rng.standard_normal((40, 60))
    G = B @ B.T + 1e-3 * np.eye(40)
    L = oracle.cholesky(G)
    np.testing.assert_allclose(L, np.linalg.cholesky(G), rtol=1e-11, atol=1e-12)
    assert np.all(np.triu(L, 1) == 0)
    r = rng.standard_normal(40)
    np.testing.assert_allclose(oracle.chol_solve(L, r), np.linalg.solve(G, r), rtol=1e-9)
    Wm = oracle.spd_inverse(L)
    np.testing.assert_allclose(Wm, np.linalg.inv(G), rtol=1e-9, atol=1e-11)
    np.testing.assert_array_equal(Wm, Wm.T)
    with pytest.raises(np.linalg.LinAlgError):
        oracle.cholesky(-np.eye(3))


def test_block_gram_is_AAT_plus_mu():
    rng = np.random.default_rng(5)
    s = W.random_sparse(50, 30, 0.2, seed=5)
    rows = np.array([3, 7, 8, 20, 41])
    Ad = s.to_dense()
    G = oracle.block_gram(s, rows, 0.25)
    np.testing.assert_allclose(G, Ad[rows] @ Ad[rows].T + 0.25 * np.eye(5), rtol=1e-14, atol=1e-15)


# --------------------------------------------------------- one block update
def _dense(Ad, k=1, lam=0.0):
    return W.System("d", Ad.shape[0], Ad.shape[1], dense=Ad, x_true=np.zeros(Ad.shape[1]),
                    b=np.zeros(Ad.shape[0]), num_blocks=k, lam=lam)


def test_update_mu0_projects_onto_block():
    """Eq. (3): with mu = 0 and a full-row-rank block, x+ satisfies
    A_B x+ = b_B, and x+ = x + pinv(A_B)(b_B - A_B x)."""
    rng = np.random.default_rng(6)
    A = rng.standard_normal((12, 30))
    b = rng.standard_normal(12)
    x = rng.standard_normal(30)
    rows = np.arange(4, 9)
    sysd = _dense(A)
    L = oracle.cholesky(oracle.block_gram(sysd, rows, 0.0))
    x1 = oracle.update_with_cholesky(sysd, rows, 0.0, b[rows] - A[rows] @ x, x)
    np.testing.assert_allclose(A[rows] @ x1, b[rows], rtol=0, atol=1e-12)
    np.testing.assert_allclose(x1, x + np.linalg.pinv(A[rows]) @ (b[rows] - A[rows] @ x),
                               rtol=1e-11, atol=1e-12)
    Wm = oracle.spd_inverse(L)
    x2 = oracle.update_with_inverse(sysd, rows, Wm, b, x)
    np.testing.assert_allclose(x2, x1, rtol=1e-11, atol=1e-12)


def test_update_single_row_is_kaczmarz():
    """Eq. (2): a one-row block with mu = 0 is the classical Kaczmarz step."""
    rng = np.random.default_rng(7)
    A = rng.standard_normal((5, 9))
    b = rng.standard_normal(5)
    x = rng.standard_normal(9)
    i = 3
    x1 = oracle.update_with_cholesky(_dense(A), np.array([i]), 0.0,
                                     np.array([b[i] - A[i] @ x]), x)
    want = x + (b[i] - A[i] @ x) / (A[i] @ A[i]) * A[i]
    np.testing.assert_allclose(x1, want, rtol=1e-13, atol=1e-14)


@pytest.mark.parametrize("mu", [1e-6, 1e-2, 3.0])
def test_update_regularised_closed_form_and_error_map(mu):
    """Lemma 1 / the proximal-point form: x+ = (A_B^T A_B + mu I)^{-1}
    (A_B^T b_B + mu x); Theorem 1's proof: for b = A x*, the error map is
    x+ - x* = mu (A_B^T A_B + mu I)^{-1} (x - x*), hence non-expansive.
    Both closed forms are evaluated through LAPACK's SVD of A_B
    (A_B = U S V^T), which stays accurate for small mu."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((20, 15))
    xs = rng.standard_normal(15)
    b = A @ xs
    x = rng.standard_normal(15)
    rows = np.array([2, 5, 6, 11, 17, 19])
    sysd = _dense(A)
    AB = A[rows]
    U, S, Vt = np.linalg.svd(AB, full_matrices=True)
    V = Vt.T
    Vr = V[:, : len(S)]
    Wm = oracle.spd_inverse(oracle.cholesky(oracle.block_gram(sysd, rows, mu)))
    x1 = oracle.update_with_inverse(sysd, rows, Wm, b, x)
    want = x + Vr @ ((S / (S ** 2 + mu)) * (U.T @ (b[rows] - AB @ x)))
    np.testing.assert_allclose(x1, want, rtol=1e-10, atol=1e-11)
    e = x - xs
    emap = Vr @ ((mu / (S ** 2 + mu)) * (Vr.T @ e)) + (e - Vr @ (Vr.T @ e))
    np.testing.assert_allclose(x1 - xs, emap, rtol=1e-9, atol=1e-10)
    assert np.linalg.norm(x1 - xs) <= np.linalg.norm(e) * (1 + 1e-12)
    x2 = oracle.update_with_cholesky(sysd, rows, mu, b[rows] - AB @ x, x)
    np.testing.assert_allclose(x2, x1, rtol=1e-10, atol=1e-11)


def test_update_sparse_equals_dense_storage():
    """The same block update on CSR and dense storage of one matrix."""
    s = W.random_sparse(40, 25, 0.15, seed=9)
    Ad = s.to_dense()
    x = np.random.default_rng(1).standard_normal(25)
    rows = np.array([0, 1, 2, 3, 4, 5, 6, 7])
    x1 = oracle.update_with_cholesky(s, rows, 1e-3, s.b[rows] - Ad[rows] @ x, x)
    x2 = oracle.update_with_cholesky(_dense(Ad), rows, 1e-3, s.b[rows] - Ad[rows] @ x, x)
    np.testing.assert_allclose(x1, x2, rtol=1e-13, atol=1e-14)


# ------------------------------------------------------------ whole solver
def test_solve_reaches_dense_lu_solution():
    """Algorithm 1 on a tiny consistent square system converges to the
    LU solution (scipy.linalg.lu_solve)."""
    rng = np.random.default_rng(10)
    n = 48
    A = rng.standard_normal((n, n)) + n ** 0.5 * np.eye(n)
    b = rng.standard_normal(n)
    sysd = W.System("sq", n, n, dense=A, x_true=None, b=b, num_blocks=6, lam=1e-8, tol=1e-13)
    res = oracle.solve(sysd, maxit=5000)
    assert res.converged
    x_lu = scipy.linalg.lu_solve(scipy.linalg.lu_factor(A), b)
    np.testing.assert_allclose(res.x, x_lu, rtol=1e-9, atol=1e-10)


def test_solve_sparse_recovers_x_true():
    """Consistent, full-column-rank sparse system: x -> x_true."""
    s = W.powerlaw(n=4096, num_blocks=16, seed=3, lam=1e-8, tol=1e-11)
    res = oracle.solve(s, maxit=4000)
    assert res.converged
    rel = np.linalg.norm(res.x - s.x_true) / np.linalg.norm(s.x_true)
    assert rel < 1e-7


def test_solve_underdetermined_min_norm_and_range():
    """Lemma 2: with x0 = 0 every iterate lies in R(A^T); for a consistent
    m < n system the limit is the minimum-norm solution pinv(A) b."""
    rng = np.random.default_rng(11)
    m, n = 30, 80
    A = rng.standard_normal((m, n))
    b = A @ rng.standard_normal(n)
    sysd = W.System("wide", m, n, dense=A, b=b, num_blocks=3, lam=1e-10, tol=1e-12)
    res = oracle.solve(sysd, maxit=3000, trace_x=True)
    assert res.converged
    np.testing.assert_allclose(res.x, np.linalg.pinv(A) @ b, rtol=1e-9, atol=1e-10)
    P_null = np.eye(n) - np.linalg.pinv(A) @ A
    for xj in res.x_trace[:: max(1, res.iters // 20)]:
        assert np.linalg.norm(P_null @ xj) <= 1e-10 * max(1.0, np.linalg.norm(xj))


def test_solve_error_non_increasing():
    """Theorem 1 (exact map, mu > 0): every block update is non-expansive
    in the error, so ||x_j - x*|| never increases across iterations."""
    s = W.random_sparse(120, 60, 0.1, seed=12, num_blocks=6, lam=1e-4)
    res = oracle.solve(s, maxit=60, tol=0.0, trace_x=True)
    xs = np.linalg.lstsq(s.to_dense(), s.b, rcond=None)[0]
    err = np.linalg.norm(res.x_trace - xs, axis=1)
    assert (np.diff(err) <= 1e-12 * err[:-1]).all()


def test_solve_trace_consistency_and_resume():
    """The tau trace is the sampler at (j, l); a solve stopped after 10
    iterations and resumed with start_iter = 10 equals a 20-iteration solve
    bit for bit (x is the whole state of Algorithm 1)."""
    s = W.laplace2d(g=12, num_blocks=8)
    full = oracle.solve(s, maxit=20, tol=0.0, seed=4, trace_tau=True, trace_rrn=True, trace_I=True)
    Pbar, P, cdf = oracle.proposal(oracle.orthogonality(s, 8), s.n)
    for j in range(20):
        for l in range(3):
            assert full.tau[j, l] == oracle.sample(cdf, 4, 0, j, l)
    a = oracle.solve(s, maxit=10, tol=0.0, seed=4)
    bb = oracle.solve(s, x0=a.x, maxit=10, tol=0.0, seed=4, start_iter=10)
    np.testing.assert_array_equal(bb.x, full.x)
    # the dynamic set is the top-K of the residual formed after the statics
    assert full.I.shape == (20, s.m // 8)


def test_solve_zero_rhs_and_immediate_convergence():
    s = W.laplace2d(g=6, num_blocks=4)
    res = oracle.solve(s, b=np.zeros(s.m), maxit=10)
    assert res.converged and res.iters == 0 and not res.x.any()
    res = oracle.solve(s, x0=s.x_true, maxit=10, tol=1e-10)
    assert res.converged and res.iters == 1


def test_solve_not_spd_with_zero_mu_and_dependent_rows():
    """mu = 0 with a rank-deficient block is the case regularisation exists
    for (Theorem 1 discussion): the Gram is singular and Cholesky fails."""
    A = np.ones((8, 3))
    sysd = W.System("sing", 8, 3, dense=A, b=A @ np.ones(3), num_blocks=2, lam=0.0)
    with pytest.raises(RuntimeError):
        oracle.solve(sysd, maxit=3)


# ------------------------------------------- residual-weighted proposal
# (not in the paper, whose P is static: the weighted variant draws block t with
# weight Pbar_t * ||r_{B_t}||^2 from the previous iteration's residual.)
def test_weighted_cdf_is_a_running_sum_of_the_weights():
    """cdf_t = sum_{i <= t} Pbar_i rho_i in block order: numpy's sequential
    accumulate of the rounded products gives the same numbers bit for bit, and
    the total agrees with an exactly rounded sum (math.fsum) within the
    sequential sum's error bound."""
    import math
    rng = np.random.default_rng(51)
    for k in (1, 63, 64, 65, 300, 4096):
        Pbar = rng.uniform(0.9, 1.0, k)
        rho = rng.uniform(0.0, 5.0, k) ** 3
        cdf = oracle.weighted_cdf(Pbar, rho)
        w = Pbar * rho
        np.testing.assert_array_equal(cdf, np.add.accumulate(w))
        exact = math.fsum(w.tolist())
        assert abs(cdf[-1] - exact) <= k * 2.0 ** -53 * exact
        assert np.all(np.diff(cdf) >= 0)


def test_threaded_residual_and_topk_equal_one_thread(monkeypatch):
    """The residual rows and the top-K scan run on several host threads above
    65536 rows; every number and the top-K set equal the one-thread run (and
    the top-K set equals a brute-force sort with planted ties)."""
    s = W.powerlaw(n=1 << 17, num_blocks=512, seed=5, lam=1e-8)
    rng = np.random.default_rng(53)
    x = rng.standard_normal(s.n)
    out = {}
    for t in ("1", "5"):
        monkeypatch.setenv("ORC_THREADS", t)
        assert oracle.thread_count(s.m) == int(t)
        r, rr = oracle.residual(s, s.b, x)
        r[[7, 70000, 130000]] = np.max(np.abs(r)) * 2.0     # a tie across thread ranges
        out[t] = (r, rr, oracle.topk(r, 256))
    np.testing.assert_array_equal(out["1"][0], out["5"][0])
    assert out["1"][1] == out["5"][1]
    np.testing.assert_array_equal(out["1"][2], out["5"][2])
    r = out["1"][0]
    order = np.lexsort((np.arange(r.size), -np.abs(r)))
    np.testing.assert_array_equal(out["5"][2], np.sort(order[:256]))


def test_block_norms_are_squared_block_residuals():
    rng = np.random.default_rng(52)
    r = rng.standard_normal(1000)
    off = np.array([0, 1, 300, 301, 700, 1000])
    rho = oracle.block_norms(r, off)
    ref = np.array([np.linalg.norm(r[off[t]:off[t + 1]]) ** 2 for t in range(5)])
    np.testing.assert_allclose(rho, ref, rtol=1e-13)


def test_weighted_draws_follow_the_weights():
    """Chi-square of 200k draws through the oracle's sampler on the weighted
    cdf against the normalised weights Pbar_t * rho_t."""
    import scipy.stats
    Pbar = np.array([0.9, 1.0, 0.95, 0.8, 1.0, 0.85, 0.9, 1.0])
    rho = np.array([4.0, 0.5, 2.0, 9.0, 0.25, 1.0, 3.0, 0.0])
    cdf = oracle.weighted_cdf(Pbar, rho)
    lib = oracle.lib()
    counts = np.zeros(8)
    for it in range(100_000):
        for l in range(2):
            counts[lib.orc_sample(cdf.ctypes.data, 8, 5, 1, it, l)] += 1
    w = Pbar * rho
    assert counts[7] == 0                         # zero residual: never drawn
    expected = w[:7] / w.sum() * counts.sum()
    chi2 = ((counts[:7] - expected) ** 2 / expected).sum()
    assert scipy.stats.chi2.sf(chi2, 6) > 1e-4


def test_weighted_first_draws_avoid_blocks_without_residual():
    """With x0 = 0 the first iteration's weights are Pbar_t ||b_{B_t}||^2, so a
    block whose right-hand side is zero is never drawn there."""
    s = W.random_sparse(400, 120, 0.3, seed=13, num_blocks=8, lam=1e-6)
    b = s.b.copy()
    b[0:50] = 0.0                                  # block 0 (50 rows)
    b[150:200] = 0.0                               # block 3
    for seed in range(40):
        res = oracle.solve(s, b=b, maxit=1, tol=0.0, seed=seed, trace_tau=True,
                           dist_mode=oracle.RESIDUAL_WEIGHTED)
        assert not set(res.tau[0]) & {0, 3}


def test_weighted_solve_recovers_x_true():
    """The weighting changes which blocks are drawn, not the fixed point: a
    consistent well-conditioned system still converges to x_true."""
    s = W.powerlaw(n=1 << 10, num_blocks=8, seed=3, lam=1e-8, tol=1e-10)
    res = oracle.solve(s, maxit=5000, seed=1, dist_mode=oracle.RESIDUAL_WEIGHTED)
    assert res.converged
    assert np.linalg.norm(res.x - s.x_true) / np.linalg.norm(s.x_true) < 1e-6


# --------------------------------------------- Algorithm 2: initial solution
def test_initial_solution_satisfies_the_remark():
    """The Remark after Algorithm 2: x0 = alpha y lies in range(A^T) (y is a
    sum of rows) and ||b - A x0|| <= ||b||.  Its proof fixes more: b - A x0 is
    orthogonal to b~ = A y, so ||b - A x0||^2 = ||b||^2 - <b, b~>^2/||b~||^2, and
    alpha minimises ||b - alpha A y|| (a least-squares fit in one unknown)."""
    for s, first, count in ((W.random_sparse(400, 120, 0.3, seed=13, num_blocks=8), 50, 50),
                            (W.gaussian_dense(300, 80, seed=4), 0, 300),
                            (W.laplace2d(g=12, num_blocks=4), 36, 36)):
        x0 = oracle.initial_solution(s, first, count)
        A = s.to_dense()
        y = A[first:first + count].sum(axis=0)
        bt = A @ y
        alpha = np.linalg.lstsq(bt[:, None], s.b, rcond=None)[0][0]
        np.testing.assert_allclose(x0, alpha * y, rtol=1e-12, atol=1e-14 * np.abs(alpha * y).max())
        r0 = s.b - A @ x0
        assert np.linalg.norm(r0) <= np.linalg.norm(s.b)
        assert abs(r0 @ bt) <= 1e-10 * np.linalg.norm(r0) * np.linalg.norm(bt) + 1e-300
        lhs = np.linalg.norm(r0) ** 2
        rhs = np.linalg.norm(s.b) ** 2 - (s.b @ bt) ** 2 / (bt @ bt)
        assert lhs == pytest.approx(rhs, rel=1e-9, abs=1e-12 * np.linalg.norm(s.b) ** 2)


def test_initial_solution_rejects_an_empty_set():
    s = W.random_sparse(40, 12, 0.3, seed=3, num_blocks=2)
    with pytest.raises(ValueError):
        oracle.initial_solution(s, 10, 0)


# --------------------------------- Algorithm 3: FAB-GMRES with ROR-BK inside
def test_fabgmres_with_exact_inner_solves_reaches_lu_solution():
    """When the inner ROR-BK solve is (nearly) exact, B ~ A^{-1}, so A z_1 =
    v_1 and the first outer step already holds the solution."""
    s = W.random_sparse(60, 60, 0.25, seed=21, num_blocks=3, lam=1e-12, tol=1e-12)
    A = s.to_dense() + 6.0 * np.eye(60)
    S = W.System("diag", 60, 60, dense=A, b=A @ s.x_true, x_true=s.x_true, num_blocks=3,
                 lam=1e-12, tol=1e-12)
    x, outer, inner, rrn, est, st = oracle.fabgmres(S, tol=1e-10, maxit=10, eta=1e-13,
                                                    lmax=200000)
    assert outer <= 2 and rrn <= 1e-10
    np.testing.assert_allclose(x, np.linalg.solve(A, S.b), rtol=1e-8, atol=1e-10)


def test_fabgmres_estimates_are_monotone_and_exact_at_the_end():
    """GMRES minimises the residual over a growing space: the estimates never
    increase, and the last equals ||b - A x|| / ||b|| of the returned x."""
    s = W.laplace2d(g=12, num_blocks=4)
    x, outer, inner, rrn, est, st = oracle.fabgmres(s, tol=1e-10, maxit=60, eta=1e-1, lmax=50)
    assert st == 0 and outer >= 3
    assert np.all(np.diff(est) <= 1e-14)
    true = np.linalg.norm(s.b - s.to_dense() @ x) / np.linalg.norm(s.b)
    assert true == pytest.approx(rrn, rel=1e-12)
    assert abs(est[-1] - rrn) <= 1e-3 * rrn + 1e-14


def test_fabgmres_wide_system_gives_min_norm_solution():
    """With x0 and the inner starts in range(A^T), the solution lies in
    range(A^T): on a wide system it is the minimum-norm solution."""
    s = W.gaussian_dense(80, 200, seed=6, num_blocks=4, lam=1e-10)
    x, outer, inner, rrn, est, st = oracle.fabgmres(s, tol=1e-11, maxit=40, eta=1e-2, lmax=200)
    assert st == 0
    x_mn = np.linalg.lstsq(s.dense, s.b, rcond=None)[0]
    assert np.linalg.norm(x - x_mn) / np.linalg.norm(x_mn) <= 1e-8


# ---- the s >= n form (Lemma 1, Section 3.1) ---------------------------------

def _ridge(A_B, b_B, x, mu):
    """The regularised block step in closed form: argmin ||A_B z - b_B||^2 +
    mu ||z - x||^2 = (A_B^T A_B + mu I)^{-1} (A_B^T b_B + mu x)."""
    n = A_B.shape[1]
    return np.linalg.solve(A_B.T @ A_B + mu * np.eye(n), A_B.T @ b_B + mu * x)


def _tall_sparse():
    s = W.random_sparse(400, 40, 0.3, seed=17, num_blocks=5, lam=1e-3)
    return s


def test_column_operator_is_the_inverse_of_the_column_gram():
    s = W.gaussian_dense(700, 120, seed=3, num_blocks=5, lam=1e-6)
    V = oracle.column_operator(s, 5, 2, 1e-6)
    A_B = s.dense[280:420]
    ref = np.linalg.inv(A_B.T @ A_B + 1e-6 * np.eye(120))
    assert np.max(np.abs(V - ref)) <= 1e-12 * np.max(np.abs(ref))
    np.testing.assert_allclose(oracle.column_gram(s, np.arange(280, 420), 1e-6),
                               A_B.T @ A_B + 1e-6 * np.eye(120), rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("kind", ["dense", "sparse"])
def test_woodbury_static_update_is_the_ridge_step_and_lemma1(kind):
    """One static update in the n x n form equals the ridge closed form, and
    the s < n form with W = (A_B A_B^T + mu I)^{-1} gives the same x (Lemma 1)
    up to its own rounding: with s > n, W carries 1/mu on the null space of
    A_B A_B^T, so that form's rounding grows like eps ||A_B||^2 / mu, which is
    why Section 3.1 stores the n x n inverse there.  The sparse block has
    columns that none of its rows holds."""
    if kind == "dense":
        s = W.gaussian_dense(700, 120, seed=3, num_blocks=5, lam=1e-6)
        mu, k, t = 1e-6, 5, 1
        A = s.dense
    else:
        s = _tall_sparse()
        mu, k, t = 1e-3, 5, 3
        A = s.to_dense()
    off = oracle.partition(s.m, k)
    rows = np.arange(off[t], off[t + 1])
    assert len(rows) >= s.n
    rng = np.random.default_rng(4)
    x = rng.standard_normal(s.n)
    b = s.b + 0.1 * rng.standard_normal(s.m)          # inconsistent block: a real step
    V = oracle.column_operator(s, k, t, mu)
    x_w = oracle.update_woodbury(s, rows, V, b, x)
    x_ref = _ridge(A[rows], b[rows], x, mu)
    assert np.linalg.norm(x_w - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    Wm = oracle.static_operator(s, k, t, mu)
    x_s = oracle.update_with_inverse(s, rows, Wm, b, x)
    A_B = A[rows]
    amp = np.finfo(float).eps * np.linalg.norm(A_B, 2) ** 2 / mu
    assert np.linalg.norm(x_s - x_ref) <= 100 * amp * np.linalg.norm(x_ref)
    assert np.linalg.norm(x_w - x_ref) <= np.linalg.norm(x_s - x_ref) + 1e-12 * np.linalg.norm(x_ref)


def test_woodbury_dynamic_update_is_the_ridge_step():
    s = _tall_sparse()
    rng = np.random.default_rng(5)
    I = np.sort(rng.choice(s.m, 80, replace=False))
    x = rng.standard_normal(s.n)
    r = s.b - s.to_dense() @ x
    x_w = oracle.update_woodbury_cholesky(s, I, 1e-3, r[I], x)
    x_ref = _ridge(s.to_dense()[I], s.b[I], x, 1e-3)
    assert np.linalg.norm(x_w - x_ref) <= 1e-9 * np.linalg.norm(x_ref)
    # and the K x K form agrees (Lemma 1), up to its eps ||A_I||^2 / mu rounding
    x_k = oracle.update_with_cholesky(s, I, 1e-3, r[I], x)
    amp = np.finfo(float).eps * np.linalg.norm(s.to_dense()[I], 2) ** 2 / 1e-3
    assert np.linalg.norm(x_k - x_ref) <= 100 * amp * np.linalg.norm(x_ref)


def test_tall_consistent_system_solved_by_one_full_rank_block():
    """With s >= n and a full-column-rank block, one regularised step on a
    consistent system lands within O(mu / sigma_min^2) of x_true."""
    s = W.gaussian_dense(700, 120, seed=3, num_blocks=5, lam=1e-10)
    r = oracle.solve(s, maxit=1, tol=0.0, seed=1)
    assert np.linalg.norm(r.x - s.x_true) <= 1e-8 * np.linalg.norm(s.x_true)
    sp = _tall_sparse()
    r2 = oracle.solve(sp, maxit=3000, tol=1e-12, seed=2)
    assert r2.status == 0 and r2.rrn <= 1e-12


def test_woodbury_at_the_boundary_s_equals_n():
    """s = n takes the n x n form (the rule is s >= n); the step is still the
    ridge closed form."""
    s = W.gaussian_dense(400, 80, seed=13, num_blocks=5, lam=1e-4)    # blocks of exactly 80 rows
    off = oracle.partition(s.m, 5)
    assert off[1] - off[0] == s.n
    rng = np.random.default_rng(14)
    x = rng.standard_normal(s.n)
    b = s.b + 0.05 * rng.standard_normal(s.m)
    V = oracle.column_operator(s, 5, 0, 1e-4)
    rows = np.arange(off[0], off[1])
    x_w = oracle.update_woodbury(s, rows, V, b, x)
    assert np.linalg.norm(x_w - _ridge(s.dense[rows], b[rows], x, 1e-4)) <= 1e-9 * np.linalg.norm(x_w)


def test_woodbury_sparse_and_dense_storage_give_the_same_bits():
    """Unstored entries count as zero in the column sums: the same tall block
    held as CSR and as a dense array gives the same V and the same update,
    bit for bit, and the same solve."""
    sp_sys = _tall_sparse()
    A = sp_sys.to_dense()
    de_sys = W.System("tall_dense", sp_sys.m, sp_sys.n, dense=A, b=sp_sys.b, x_true=sp_sys.x_true,
                      num_blocks=sp_sys.num_blocks, lam=sp_sys.lam, tol=sp_sys.tol)
    k = sp_sys.num_blocks
    off = oracle.partition(sp_sys.m, k)
    rows = np.arange(off[2], off[3])
    Vs = oracle.column_operator(sp_sys, k, 2, sp_sys.lam)
    Vd = oracle.column_operator(de_sys, k, 2, sp_sys.lam)
    np.testing.assert_array_equal(Vs, Vd)
    x0 = np.random.default_rng(15).standard_normal(sp_sys.n)
    np.testing.assert_array_equal(oracle.update_woodbury(sp_sys, rows, Vs, sp_sys.b, x0),
                                  oracle.update_woodbury(de_sys, rows, Vd, sp_sys.b, x0))
    r1 = oracle.solve(sp_sys, maxit=30, tol=0.0, seed=4)
    r2 = oracle.solve(de_sys, maxit=30, tol=0.0, seed=4)
    np.testing.assert_array_equal(r1.x, r2.x)


def test_woodbury_with_mu_zero_is_the_block_least_squares_solution():
    """mu = 0 and a full-column-rank tall block: x + (A_B^T A_B)^{-1} A_B^T
    (b_B - A_B x) is the block's least-squares solution, whatever x was."""
    s = W.gaussian_dense(600, 50, seed=16, num_blocks=4, lam=0.0)
    off = oracle.partition(s.m, 4)
    rows = np.arange(off[1], off[2])
    rng = np.random.default_rng(17)
    b = s.b + 0.1 * rng.standard_normal(s.m)
    V = oracle.column_operator(s, 4, 1, 0.0)
    x_ls = np.linalg.lstsq(s.dense[rows], b[rows], rcond=None)[0]
    for _ in range(2):
        x = rng.standard_normal(s.n)
        x_w = oracle.update_woodbury(s, rows, V, b, x)
        assert np.linalg.norm(x_w - x_ls) <= 1e-10 * np.linalg.norm(x_ls)


def test_recorded_oracle_solution_of_the_benchmark_workload():
    """oracle/record_iterations.py ran the FP64 oracle alone to the tolerance on
    the 2^20 power-law workload and stored the iteration count and the solution
    (which the benchmark compares the GPU results with).  The stored solution
    is the recorded file (checksum), and its residual, recomputed here with
    scipy from the generated system, is the recorded relative residual."""
    import hashlib
    import json
    import os
    import scipy.sparse as sp
    here = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle")
    rec = json.load(open(os.path.join(here, "iterations_to_tol.json")))
    key = "powerlaw_n1048576_k4096_lam1e-08_tol1e-08_seed1"
    meta = rec[key + "_meta"]
    assert rec[key] == 74252 and meta["converged"]
    x = np.load(os.path.join(here, meta["x_file"]))
    assert hashlib.sha256(x.tobytes()).hexdigest() == meta["x_sha256"]
    s = W.powerlaw(n=1 << 20, num_blocks=4096, seed=1, lam=1e-8, tol=1e-8)
    A = sp.csr_matrix((s.values.astype(np.float64), s.col_idx, s.row_ptr), shape=(s.m, s.n))
    rrn = np.linalg.norm(s.b - A @ x) / np.linalg.norm(s.b)
    assert rrn <= 1e-8
    assert abs(rrn - meta["rrn"]) <= 1e-6 * meta["rrn"]
