"""Failure paths, triggered from the host without faulting the GPU.

- A NaN in b or in x0 reaches the residual and ends the solve with
  RORBK_ERR_NUMERIC (graph loop and host loop, FP64 and mixed precision);
  a NaN in A is refused by the set-up's validation.
- The bounded wait of the sampled updates, driven to give up by the
  RORBK_FAULT_WAIT_LIMIT option (a barrier that nothing completes, one poll),
  ends the solve with RORBK_ERR_DEVICE_TIMEOUT after the kernel has waited for
  its own copies; the handle then solves normally and matches the oracle.
- A dynamic update given row indices outside [0, m) or out of order is refused
  on the device with RORBK_ERR_BOUNDS before any row is read, leaving x as it was.
"""
import numpy as np
import pytest

import oracle
from paper_2510_02156_gb300 import binding as B
from paper_2510_02156_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NUMERIC, BOUNDS, TIMEOUT = -5, -6, -8


def _dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dt)


@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_MIXED])
@pytest.mark.parametrize("host_loop", [0, 1])
@pytest.mark.parametrize("where", ["b", "x0"])
def test_nan_input_reports_numeric(cuda_ok, precision, host_loop, where):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=3, lam=1e-8)
    b = s.b.copy()
    x0 = np.zeros(s.n)
    if where == "b":
        b[123] = np.nan
    else:
        x0[45] = np.nan
    with B.Handle.from_system(s, precision=precision) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        with pytest.raises(B.RorbkError) as e:
            h.solve(_dev(b), x, x0=_dev(x0), tol=1e-8, maxit=50, precision=precision,
                    host_loop=host_loop, poll=8)
        assert e.value.status == NUMERIC
        # the handle is still usable
        res = h.solve(_dev(s.b), x, tol=0.0, maxit=5, precision=precision)
        assert res.iters >= 5 and np.isfinite(res.rrn)


def test_nan_in_A_is_refused_at_setup(cuda_ok):
    s = W.powerlaw(n=1 << 10, num_blocks=8, seed=3, lam=1e-8)
    s.values = s.values.astype(np.float64)
    s.values[17] = np.nan
    with pytest.raises(B.RorbkError) as e:
        B.Handle.from_system(s)
    assert e.value.status == NUMERIC


@pytest.mark.parametrize("host_loop", [0, 1])
@pytest.mark.parametrize("precision", [B.PREC_FP64, B.PREC_MIXED])
def test_bounded_wait_gives_up_with_timeout_status(cuda_ok, host_loop, precision):
    s = W.powerlaw(n=1 << 13, num_blocks=32, seed=4, lam=1e-8)
    with B.Handle.from_system(s, precision=precision) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        with pytest.raises(B.RorbkError) as e:
            h.solve(_dev(s.b), x, tol=0.0, maxit=20, seed=5, precision=precision,
                    host_loop=host_loop, poll=4, fault_inject=B.FAULT_WAIT_LIMIT)
        assert e.value.status == TIMEOUT
        torch.cuda.synchronize()
        # nothing was left in flight: the same handle now runs the oracle's iterations
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(_dev(s.b), x, tol=0.0, maxit=20, seed=5)
    o = oracle.solve(s, maxit=20, tol=0.0, seed=5)
    assert res.iters == 20
    np.testing.assert_array_equal(x.cpu().numpy(), o.x)


def test_unknown_fault_mode_is_an_argument_error(cuda_ok):
    s = W.powerlaw(n=1 << 10, num_blocks=8, seed=3, lam=1e-8)
    with B.Handle.from_system(s) as h:
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        with pytest.raises(B.RorbkError) as e:
            h.solve(_dev(s.b), x, maxit=2, fault_inject=7)
        assert e.value.status == -1


@pytest.mark.parametrize("bad", ["negative", "beyond_m", "descending", "repeated"])
def test_dynamic_update_refuses_bad_rows(cuda_ok, bad):
    s = W.powerlaw(n=1 << 12, num_blocks=16, seed=6, lam=1e-8)
    K = s.m // 16
    rng = np.random.default_rng(3)
    I = np.sort(rng.choice(s.m, K, replace=False)).astype(np.int32)
    if bad == "negative":
        I[0] = -1
    elif bad == "beyond_m":
        I[-1] = s.m
    elif bad == "descending":
        I[[3, 4]] = I[[4, 3]]
    else:
        I[5] = I[4]
    x0 = rng.standard_normal(s.n)
    with B.Handle.from_system(s) as h:
        r = torch.empty(s.m, dtype=torch.float64, device="cuda")
        x = _dev(x0)
        h.residual(_dev(s.b), x, r)
        with pytest.raises(B.RorbkError) as e:
            h.dynamic_update(_dev(I, torch.int32), r, x)
        assert e.value.status == BOUNDS
        np.testing.assert_array_equal(x.cpu().numpy(), x0)
        # a valid set afterwards runs the oracle's update
        Iok = np.sort(rng.choice(s.m, K, replace=False)).astype(np.int32)
        h.dynamic_update(_dev(Iok, torch.int32), r, x)
    rr = oracle.residual(s, s.b, x0)[0]
    ref = oracle.update_with_cholesky(s, Iok.astype(np.int64), s.lam, rr[Iok], x0)
    xg = x.cpu().numpy()
    assert np.linalg.norm(xg - ref) / np.linalg.norm(ref) <= 1e-13
