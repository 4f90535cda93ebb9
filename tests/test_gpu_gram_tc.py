"""The mixed-precision dense dynamic Gram on the tensor cores (tcgen05,
kind::tf32): G = A_I A_I^T + mu I from A's FP32 copy, TF32 products
accumulated in FP32 per 128-column chunk, chunks added in FP64.  Checked
against the FP64 product of the same FP32 values computed on the host: TF32
keeps 10 of FP32's 23 mantissa bits, so each factor is off by less than 2^-10
of itself (truncated; 2^-11 rounded) and each product by less than
(2^-9 + 2^-20) of itself; FP32 accumulation of a 128-column chunk adds at most
128 * 2^-24 of sum_j |a_aj a_bj|.  The test allows 1.1 * 2^-9 sum_j |a_aj a_bj|.  Inputs
whose values carry 10 significant bits or fewer are exact in TF32, and their
Gram is exact: that case checks the data movement bit for bit."""
import numpy as np
import pytest

from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gram(h, I, precision):
    K = len(I)
    G = torch.empty(K * (K + 1) // 2, dtype=torch.float64, device="cuda")
    h.dense_gram(torch.as_tensor(np.asarray(I, dtype=np.int32), device="cuda"), G, precision)
    P = G.cpu().numpy()
    out = np.zeros((K, K))
    a, b = np.tril_indices(K)
    out[a, b] = P            # tril_indices enumerates the packed row-major order
    return out


def _system(m, n, blocks, seed, integer=False):
    s = W.gaussian_dense(m, n, seed=seed, num_blocks=blocks, lam=1e-6)
    if integer:
        rng = np.random.default_rng(seed)
        A = rng.integers(-8, 9, size=(m, n)).astype(np.float64)
        s = W.System("int_dense", m, n, dense=A, b=A @ np.ones(n), x_true=np.ones(n),
                     num_blocks=blocks, lam=1e-6, tol=1e-8)
    return s


@pytest.mark.parametrize("m,n,blocks", [(4000, 402, 20), (9000, 640, 30), (12800, 2048, 50)])
def test_tensor_core_gram_within_tf32_bound(cuda_ok, m, n, blocks):
    """K = 200, 300, 256 rows (2 or 3 tiles of 128 on each side), n with a
    ragged last chunk and n % 4 != 0 (the scalar staging path)."""
    s = _system(m, n, blocks, seed=4)
    K = m // blocks
    I = np.sort(np.random.default_rng(5).choice(m, K, replace=False))
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h:
        g64 = _gram(h, I, B.PREC_FP64)
        gtc = _gram(h, I, B.PREC_MIXED)
    A = s.dense[I].astype(np.float32).astype(np.float64)
    exact = A @ A.T + s.lam * np.eye(K)
    bound = 1.1 * 2.0 ** -9 * (np.abs(A) @ np.abs(A).T) + 1e-12
    low = np.tril(np.ones((K, K), dtype=bool))
    assert np.all(np.abs(gtc - exact)[low] <= bound[low])
    # and the FP64 kernel is the FP64 product to rounding (n fused steps)
    A64 = s.dense[I]
    err64 = np.abs(g64 - (A64 @ A64.T + s.lam * np.eye(K)))
    assert np.all(err64[low] <= (n * 2.0 ** -52 * (np.abs(A64) @ np.abs(A64).T) + 1e-12)[low])


def test_tensor_core_gram_exact_on_tf32_representable_values(cuda_ok):
    """Integers in [-8, 8]: exact in TF32, every partial sum exact in FP32, so
    the tensor-core Gram equals the FP64 one bit for bit (the layout of the
    staged operands, the descriptors and the tile bookkeeping all matter)."""
    s = _system(6000, 520, 20, seed=9, integer=True)
    K = 300
    I = np.sort(np.random.default_rng(6).choice(6000, K, replace=False))
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h:
        g64 = _gram(h, I, B.PREC_FP64)
        gtc = _gram(h, I, B.PREC_MIXED)
    low = np.tril(np.ones((K, K), dtype=bool))
    np.testing.assert_array_equal(gtc[low], g64[low])


def test_mixed_dense_solve_with_tensor_core_gram_reaches_tolerance(cuda_ok):
    """Two tiles per side (K = 200) and a ragged, unaligned n: the mixed form
    with the tensor-core Gram still reaches 1e-10, measured in FP64."""
    s = _system(4000, 402, 20, seed=11)
    with B.Handle.from_system(s, precision=B.PREC_MIXED) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(torch.as_tensor(s.b, device="cuda"), x, tol=1e-10, maxit=50000, seed=3,
                      precision=B.PREC_MIXED)
    xh = x.cpu().numpy()
    assert res.converged
    assert np.linalg.norm(s.dense @ xh - s.b) / np.linalg.norm(s.b) <= 1.001e-10


def test_dense_gram_rejects(cuda_ok):
    s = _system(4000, 402, 20, seed=4)
    I = torch.arange(200, dtype=torch.int32, device="cuda")
    G = torch.empty(200 * 201 // 2, dtype=torch.float64, device="cuda")
    with B.Handle.from_system(s) as h:                     # FP64 handle: no tensor-core Gram
        with pytest.raises(B.RorbkError):
            h.dense_gram(I, G, B.PREC_MIXED)
        with pytest.raises(B.RorbkError):
            h.dense_gram(I, G, 9)
    sp = W.powerlaw(n=1 << 12, num_blocks=16, seed=3, lam=1e-8)
    with B.Handle.from_system(sp) as h:
        with pytest.raises(B.RorbkError):
            h.dense_gram(torch.arange(h.info.dyn_rows, dtype=torch.int32, device="cuda"), G)
