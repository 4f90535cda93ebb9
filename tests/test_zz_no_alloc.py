"""The residual entry point that allocates nothing (rorbk_csr_residual_noalloc).

Callers that cannot allocate device memory where they need a residual (code
inside an allocator or a memory-pool callback, processes whose memory a
framework reserved at start-up, real-time loops) use this entry point; its
scratch is a fixed array compiled into the library.  It must give the same
residual as the handle-based rorbk_residual, call after call: the scratch is
shared and keeps the previous call's contents, so two calls in a row check
that nothing leaks from one call into the next.
"""
import numpy as np
import pytest

from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp32_values", [False, True])
def test_noalloc_residual_matches_handle_residual_twice(cuda_ok, fp32_values):
    s = W.powerlaw(n=1 << 15, num_blocks=128, seed=5, lam=1e-8)
    if not fp32_values:
        s.values = s.values.astype(np.float64)
    rng = np.random.default_rng(11)
    dev = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dt)
    rp = dev(s.row_ptr, torch.int32)
    ci = dev(s.col_idx, torch.int32)
    vals = dev(s.values, torch.float32 if fp32_values else torch.float64)
    b = dev(s.b)
    with B.Handle.from_system(s) as h:
        for call in range(2):
            x = dev(rng.standard_normal(s.n) * (1 + call))
            r_ref = torch.empty(s.m, dtype=torch.float64, device="cuda")
            rr_ref = h.residual(b, x, r_ref)
            r = torch.full((s.m,), np.nan, dtype=torch.float64, device="cuda")
            rr = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
            B.csr_residual_noalloc(rp, ci, vals, s.m, s.n, b, x, r, rr)
            torch.cuda.synchronize()
            # same row arithmetic: identical residuals; the sum of squares is
            # a different (fixed) tree
            assert torch.equal(r, r_ref)
            assert float(rr.item()) == pytest.approx(rr_ref, rel=1e-12)


@pytest.mark.parametrize("m,blocks", [(257, 1), (3, 1), (65537, 128)])
def test_noalloc_ragged_row_counts(cuda_ok, m, blocks):
    """Row counts that leave the last thread block part-filled (a few rows, one
    more than a multiple of 256): r bit for bit and ||r||^2 as the handle's
    residual, twice in a row."""
    s = W.random_sparse(m, 97, 0.05, seed=m % 1000, num_blocks=blocks)
    rng = np.random.default_rng(m)
    dev = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dt)
    rp, ci, vals, b = dev(s.row_ptr, torch.int32), dev(s.col_idx, torch.int32), dev(s.values), dev(s.b)
    with B.Handle.from_system(s) as h:
        for call in range(2):
            x = dev(rng.standard_normal(s.n))
            r_ref = torch.empty(s.m, dtype=torch.float64, device="cuda")
            rr_ref = h.residual(b, x, r_ref)
            r = torch.full((s.m,), np.nan, dtype=torch.float64, device="cuda")
            rr = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
            B.csr_residual_noalloc(rp, ci, vals, s.m, s.n, b, x, r, rr)
            torch.cuda.synchronize()
            assert torch.equal(r, r_ref)
            assert float(rr.item()) == pytest.approx(rr_ref, rel=1e-12, abs=1e-300)


def test_noalloc_at_its_row_limit(cuda_ok):
    """m = 2^24 rows, the most the fixed scratch covers (65536 thread blocks),
    one stored entry per row: r_i = b_i - a_i x_{c_i} exactly, and ||r||^2 as
    a sum of the exact squares within its rounding."""
    m, n = 1 << 24, 4096
    g = torch.Generator(device="cuda").manual_seed(5)
    rp = torch.arange(m + 1, dtype=torch.int32, device="cuda")
    ci = torch.randint(0, n, (m,), dtype=torch.int32, device="cuda", generator=g)
    vals = torch.randn(m, dtype=torch.float64, device="cuda", generator=g)
    b = torch.randn(m, dtype=torch.float64, device="cuda", generator=g)
    x = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    for _ in range(2):
        r = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
        rr = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
        B.csr_residual_noalloc(rp, ci, vals, m, n, b, x, r, rr)
        torch.cuda.synchronize()
        ref = b - torch.addcmul(torch.zeros_like(b), vals, x[ci.long()])
        assert torch.equal(r, ref)
        tot = float((ref * ref).sum().item())
        assert float(rr.item()) == pytest.approx(tot, rel=1e-12)


def test_noalloc_rejects_sizes_beyond_its_scratch(cuda_ok):
    """More rows than the fixed scratch covers is an argument error, reported
    before anything is launched."""
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    idx = torch.zeros(2, dtype=torch.int32, device="cuda")
    st = B.lib().rorbk_csr_residual_noalloc((1 << 24) + 1, 1, 0, B._ptr(idx), None, None, B.F64,
                                            B._ptr(one), B._ptr(one), B._ptr(one), B._ptr(one),
                                            None)
    assert st == -1
    assert b"16777216" in B.lib().rorbk_last_error(None)
