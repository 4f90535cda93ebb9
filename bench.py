"""Benchmark: time to ||Ax-b||/||b|| <= 1e-8 with ROR-BK on one GB300.

Workload: the 2^20-row power-law CSR system (FP32-stored values; row nnz a
power law, alpha = 2.5, 3..200 off-diagonals plus the diagonal shift; rows
scaled log-uniform in [1e-4, 1]), 4096 contiguous row blocks of 256 rows,
lambda = 1e-8, tol = 1e-8, x0 = 0, Philox seed 1.  One benchmark step is one
whole solve from x0 = 0 to the tolerance: every iteration of Algorithm 1
(three sampled static block updates, the full residual, the residual top-K
selection and the dynamic block update).  The set-up (Algorithm 1's partition, orthogonality weights and stored inverses)
runs once before timing and is reported separately.

Headline value: the mixed-precision form (FP64 iterative refinement around
FP32 ROR-BK, the block Gram Cholesky in FP64); the plain FP64 form is timed on
the same inputs beside it.

Arms:
  (default)          the CUDA library through its C ABI
  --impl reference   the FP64 CPU oracle on the host cores: a bounded sample of
                     iterations per step, scaled to the iterations the solve
                     takes

Prints one JSON line (rank 0).  Under torchrun each rank solves its own
system (seed = rank): weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "time-to ||Ax-b||/||b||<=1e-8 & HBM GB/s: mixed-prec vs FP64 ROR-BK, 1 GB300"
L2_FLUSH_BYTES = 512 << 20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=1 << 20)
    p.add_argument("--blocks", type=int, default=4096)
    p.add_argument("--lam", type=float, default=1e-8)
    p.add_argument("--tol", type=float, default=1e-8)
    p.add_argument("--inner-tol", type=float, default=1e-4)
    p.add_argument("--maxit", type=int, default=2_000_000)
    p.add_argument("--fp64-steps", type=int, default=1)
    p.add_argument("--oracle-iters", type=int, default=60)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-dense", action="store_true",
                   help="skip the dense measurement (A = U diag(s) V^T, 200,000 x 2,048, "
                        "781 blocks of 256 rows; a fixed number of iterations)")
    p.add_argument("--dense-iters", type=int, default=100)
    p.add_argument("--no-fabgmres", action="store_true",
                   help="skip FAB-GMRES with ROR-BK inner solves (Algorithm 3) on the 262,144-unknown "
                        "power-law system, beside plain ROR-BK on it")
    p.add_argument("--no-incremental", action="store_true",
                   help="skip the incremental-residual variant (r -= A dx from the change "
                        "log, an exact residual every 50 iterations) on the main workload")
    p.add_argument("--no-weighted", action="store_true",
                   help="skip the comparison of the residual-weighted draws with the paper's "
                        "(FP64 to tolerance on the 262,144-unknown power-law system)")
    p.add_argument("--clone-batched", action="store_true",
                   help="also run the batches of one-column handles (16 clones of a 65,536-row "
                        "system, 16 systems of 5,000-200,000 rows, each in one launch), which the "
                        "block measurements below supersede")
    p.add_argument("--no-multi-rhs", action="store_true",
                   help="skip the block of 16 right-hand sides of the main workload (one residual "
                        "pass over A for all columns), mixed and FP64 to the tolerance")
    p.add_argument("--no-batched-scale", action="store_true",
                   help="skip the batched configuration at its stated size (256 power-law "
                        "systems of 5,000-200,000 rows with 16 right-hand sides each, plus a dense "
                        "2,048 x 100,000 minimum-norm system, in one graph launch)")
    p.add_argument("--batch-systems", type=int, default=256)
    p.add_argument("--multi-fp64-iters", type=int, default=2000)
    p.add_argument("--tune-iters", type=int, default=100,
                   help="iterations per candidate of rorbk_autotune before the timed solves")
    p.add_argument("--dense-wide-lam", type=float, default=1e-10)
    p.add_argument("--no-autograd", action="store_true",
                   help="skip the differentiable-solve measurement (forward + adjoint backward "
                        "on the 262,144-unknown power-law system)")
    p.add_argument("--profile", type=int, default=0,
                   help="profiling run: N iterations of each form, the loop driven from the "
                        "host (so that a profiler sees every kernel); prints no JSON")
    p.add_argument("--profile-dense", choices=("fp64", "mixed"), default=None,
                   help="profiling run of the dense path: two host-driven iterations on a "
                        "25,600 x 2,048 Gaussian system with 100 blocks of 256 rows (the K, s "
                        "and n of the 200,000 x 2,048 workload) in the given precision; "
                        "prints no JSON")
    p.add_argument("--profile-multi", type=int, default=0,
                   help="profiling run of a block of 16 right-hand sides of the main workload: "
                        "three block residuals alone in FP32 and three in FP64, then N host-driven "
                        "iterations of the mixed form; prints no JSON")
    p.add_argument("--cache", default=os.path.join(ROOT, ".cache"))
    return p.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(rank):
    """Generator seed of the system rank `rank` solves: every rank (replica)
    solves its own independent system, so per-GPU work is fixed as N grows."""
    return 1 + rank


def max_over_ranks(value, dist, device):
    """The step time of the job: the maximum over all ranks (a no-op for one
    process).  The only collective of a replicated run besides barriers."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload(args, rank):
    from paper_2510_02156_gb300 import workloads as W
    return W.powerlaw(n=args.n, num_blocks=args.blocks, seed=replica_seed(rank), lam=args.lam,
                      tol=args.tol, cache=args.cache)


def config(args, s, extra=None):
    c = {"workload": (f"power-law sparse square CSR, n={s.n}, nnz={s.nnz}, FP32-stored A, "
                      f"{s.num_blocks} row blocks of {s.m // s.num_blocks}, lambda={s.lam:g}, "
                      f"tol={s.tol:g}, x0=0, Philox seed 1"),
         "step": "one whole solve from x0 = 0 to the tolerance",
         "l2": "flushed (512 MiB write) between timed steps"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu, self.proc, self.lines = gpu_index, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_hbm_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p)).get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


def spmv_bytes(s, vbytes, xbytes):
    """Algorithmic bytes of one r = b - A x: A's values and column indices
    once, x read once, b read and r written."""
    return s.nnz * (vbytes + 4) + xbytes * s.n + 2 * xbytes * s.m


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic_k_residual_powerlaw_n1048576.txt")
MRES_TRAFFIC_FILE = os.path.join(ROOT, "profiles", "roofline_traffic_k_mres_powerlaw_n1048576_nr16.txt")
KERNEL_SOURCES = ("paper_2510_02156_gb300/csrc/kernels_iter.cu", "paper_2510_02156_gb300/csrc/common.cuh")
# the residual kernel's part of the first source: from its section marker to
# the next kernel's comment (the kernel and the helpers it calls)
RESIDUAL_REGION = ("// ---------------------------------------------------------------- residual",
                   "// Incremental residual, first kernel")
# the block residual's part: the section of a block of right-hand sides up to
# the kernel that unpermutes its columns
MRES_REGION = ("// ------------------------------------------------- a block of right-hand sides",
               "// Residual columns from the SELL order")


def region_sha256(region):
    """sha256 of one kernel's source region of kernels_iter.cu and of
    common.cuh: the code a traffic record was captured from."""
    import hashlib
    h = hashlib.sha256()
    for i, f in enumerate(KERNEL_SOURCES):
        with open(os.path.join(ROOT, f), "rb") as fh:
            data = fh.read()
        if i == 0:
            a = data.find(region[0].encode())
            z = data.find(region[1].encode())
            data = data[a:z] if 0 <= a < z else data
        h.update(data)
    return h.hexdigest()


def residual_sources_sha256():
    return region_sha256(RESIDUAL_REGION)


def mres_sources_sha256():
    return region_sha256(MRES_REGION)


def profiled_traffic(kernel, s):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, or
    None when the workload differs from the captured one or the kernel's
    source changed since the capture."""
    if kernel.startswith("k_mres<"):
        path, region = MRES_TRAFFIC_FILE, MRES_REGION
    else:
        path, region = TRAFFIC_FILE, RESIDUAL_REGION
    if (s.m, s.nnz) != (1 << 20, 9692830) or not os.path.exists(path):
        return None
    digest = region_sha256(region)
    rec = {}
    with open(path) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                k, v = ln.split()
                rec[k] = v
    if rec.get("sources_sha256") != digest or kernel not in rec:
        return None
    return int(rec[kernel])


def time_kernel(launch, flush, torch, reps=20):
    """Mean device time of one launch: each launch after an L2 flush (cold;
    the kernel's HBM-bound time), and back to back (warm)."""
    st = torch.cuda.current_stream()
    for _ in range(3):
        launch()
    torch.cuda.synchronize()
    cold = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        launch()
        e1.record(st)
        e1.synchronize()
        cold.append(e0.elapsed_time(e1))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        launch()
    e1.record(st)
    e1.synchronize()
    return float(np.mean(cold)), float(e0.elapsed_time(e1) / reps)


def run_solves(h, b, x, s, args, prec, steps, warmup, flush, torch, clocks=None):
    stream = torch.cuda.current_stream()
    kw = dict(tol=s.tol, maxit=args.maxit, seed=1, precision=prec, inner_tol=args.inner_tol)
    for _ in range(warmup):
        flush.zero_()
        h.solve(b, x, **kw)
    torch.cuda.synchronize()
    times, last = [], None
    ctx = clocks if clocks is not None else _Null()
    with ctx:
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            last = h.solve(b, x, **kw)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
    xh = x.cpu().numpy()
    out = {"time_s": float(np.mean(times)), "times_s": times, "iters": int(last.iters),
           "refinements": int(last.refinements), "rrn": float(last.rrn),
           "converged": bool(last.converged),
           "rel_err_vs_x_true": float(np.linalg.norm(xh - s.x_true) / np.linalg.norm(s.x_true))}
    xo = oracle_solution(s, args)
    if xo is not None:
        out["rel_err_vs_fp64_oracle"] = float(np.linalg.norm(xh - xo) / np.linalg.norm(xo))
    return out


def oracle_solution(s, args):
    """The FP64 oracle's converged solution of this workload, as recorded by
    oracle/record_iterations.py (an oracle-only script), or None when no
    record matches the workload (or its checksum)."""
    import hashlib
    key = (f"powerlaw_n{s.n}_k{s.num_blocks}_lam{args.lam:g}_tol{args.tol:g}_seed1")
    rec = os.path.join(ROOT, "oracle", "iterations_to_tol.json")
    if not os.path.exists(rec):
        return None
    meta = json.load(open(rec)).get(key + "_meta", {})
    path = os.path.join(ROOT, "oracle", meta.get("x_file", "-"))
    if not os.path.exists(path):
        return None
    xo = np.load(path)
    if hashlib.sha256(xo.tobytes()).hexdigest() != meta.get("x_sha256") or xo.shape != (s.n,):
        return None
    return xo


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


_T0 = time.time()


def note(msg):
    """A progress line on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.time() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def run_ours(args, rank, world, local):
    import torch
    from paper_2510_02156_gb300 import binding as B

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    s = workload(args, rank)
    t0 = time.time()
    h = B.Handle.from_system(s, precision=B.PREC_MIXED)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    b = torch.as_tensor(s.b, device="cuda")
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    # launch shapes chosen by measurement for the mixed form's inner iteration
    # (rorbk_autotune; grids that leave every result unchanged)
    tune = h.autotune(b, precision=B.PREC_MIXED, iters=args.tune_iters)
    tuning = tuning_dict(tune)
    if dist:
        dist.barrier()
    clk = ClockSampler(local)
    note("timed mixed solves")
    mixed = run_solves(h, b, x, s, args, B.PREC_MIXED, args.steps, args.warmup, flush, torch, clk)
    note("FP64 solves")
    t_step = mixed["time_s"]
    t_step = max_over_ranks(t_step, dist, "cuda")
    fp64 = run_solves(h, b, x, s, args, B.PREC_FP64, args.fp64_steps, 1, flush, torch)

    # end to end through the host-buffer entry point (H2D of b and D2H of x
    # inside the timed call)
    bh = np.ascontiguousarray(s.b)
    xo = np.zeros(s.n)
    flush.zero_()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    h.solve_host(bh, xo, tol=s.tol, maxit=args.maxit, seed=1, precision=B.PREC_MIXED,
                 inner_tol=args.inner_tol)
    e2e_s = time.perf_counter() - t1

    note("incremental residual")
    inc = None if args.no_incremental else incremental_measurement(args, s, h, b, x, flush)
    note("FAB-GMRES")
    fg = None if args.no_fabgmres else fabgmres_measurement(args)
    note("differentiable solve")
    ag = None if args.no_autograd else autograd_measurement(args)
    note("residual-weighted draws")
    weighted = None if args.no_weighted else weighted_measurement(args)
    batched = batched_measurement(args) if args.clone_batched else None
    note("block of 16 right-hand sides")
    multi = (None if args.no_multi_rhs else
             multi_rhs_measurement(args, s, flush, mixed["time_s"], fp64["time_s"]))
    note("batched configuration")
    scale = None if args.no_batched_scale else batched_scale_measurement(args, flush)
    note("dense system")
    dense = None if args.no_dense else dense_measurement(args, flush)
    note("done with the GPU measurements")

    # the sparse residual kernels timed alone, the same kernel and grid as in
    # the solve: FP32 (the inner solve, every iteration) and FP64
    x32 = (torch.as_tensor(s.x_true, device="cuda") * 0.5).float()
    b32 = b.float()
    r32 = torch.empty(s.m, dtype=torch.float32, device="cuda")
    cold32, warm32 = time_kernel(lambda: h.residual32(b32, x32, r32, wait=False), flush, torch)
    x64 = torch.as_tensor(s.x_true, device="cuda") * 0.5
    r64 = torch.empty(s.m, dtype=torch.float64, device="cuda")
    cold64, warm64 = time_kernel(lambda: h.residual_async(b, x64, r64), flush, torch)
    h.close()
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    peak, peak_kind = measured_hbm_peak()
    by32 = spmv_bytes(s, 4, 4)
    by64 = spmv_bytes(s, 4, 8)
    ach32 = by32 / (cold32 * 1e-3) / 1e9
    ach64 = by64 / (cold64 * 1e-3) / 1e9
    launches = 1 + mixed["refinements"] * 3 + 6 * mixed["iters"]
    line = {
        "metric": METRIC, "value": t_step, "unit": "s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 inner + f64 refinement",
        "data": "synthetic", "setup_s": setup_s,
        "config": config(args, s, {"precision": "mixed (headline) and fp64",
                                   "inner_tol": args.inner_tol,
                                   "solves_per_s_all_ranks": world / t_step}),
        "mixed": mixed, "fp64": fp64, "autotune": tuning,
        "speedup_mixed_vs_fp64": fp64["time_s"] / mixed["time_s"],
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": 8 * s.m,
                "d2h_bytes_per_step": 8 * s.n},
        "gpu_launches": launches * args.steps,
        "autograd": ag,
        "batched": batched,
        "multi_rhs": multi,
        "batched_scale": scale,
        "residual_weighted": weighted,
        "fabgmres": fg,
        "incremental_residual": inc,
        "dense": dense,
        "clocks": clk.summary(),
        "roofline": {"bound": "hbm", "achieved": ach32, "peak": peak, "unit": "GB/s",
                     "frac": ach32 / peak,
                     "traffic": profiled_traffic("k_residual<float,float>", s),
                     "kernel": "k_residual<float,float>: the FP32 SELL-32 sparse residual "
                               "r = b - A x of the inner solve (one launch per iteration)",
                     "bytes_per_launch": by32, "launch_ms_cold_l2": cold32,
                     "launch_ms_warm_l2": warm32,
                     "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs, burst copy)"},
        "roofline_fp64_residual": {"bound": "hbm", "achieved": ach64, "peak": peak,
                                   "unit": "GB/s", "frac": ach64 / peak,
                                   "traffic": profiled_traffic("k_residual<double,float>", s),
                                   "bytes_per_launch": by64, "launch_ms_cold_l2": cold64,
                                   "launch_ms_warm_l2": warm64},
    }
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(s, args, mixed["iters"])
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def _timed(fn, torch):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return time.perf_counter() - t0, out


def _batch_vs_sequential(handles, bs, tol, maxit, precision, torch, B, system_ids, seq=None):
    """One batched launch against the same solves one after another (each
    solve's own graph).  seq = how many of the solves to run one after another
    (None: all; fewer: the time is scaled to all of them, and said so; 0: no
    sequential run)."""
    xs = [torch.empty(h.info.n, dtype=torch.float64, device="cuda") for h in handles]
    with B.Batch(handles, precision=precision) as bt:
        bt.solve(bs, xs, tol=tol, maxit=maxit, seed=1, system_ids=system_ids)     # warm-up
        t_b, (st, res) = _timed(lambda: bt.solve(bs, xs, tol=tol, maxit=maxit, seed=1,
                                                 system_ids=system_ids), torch)
    out = {"batched_s": t_b, "iters": [int(r.iters) for r in res],
           "all_converged": bool(all(r.converged for r in res))}
    k = len(handles) if seq is None else seq
    if k:
        sel = list(zip(handles, bs, xs, system_ids))[:k]
        h0, b0, x0, s0 = sel[0]
        h0.solve(b0, x0, tol=tol, maxit=maxit, seed=1, system_id=s0, precision=precision)
        t_s, sq = _timed(lambda: [h.solve(b, x, tol=tol, maxit=maxit, seed=1, system_id=sid,
                                          precision=precision) for h, b, x, sid in sel], torch)
        scale = len(handles) / k
        out.update({"sequential_s": t_s * scale, "speedup": t_s * scale / t_b,
                    "sequential_measured": (f"all {k} solves" if k == len(handles) else
                                            f"{k} of {len(handles)} solves, scaled by {scale:g}"),
                    "same_iterations_as_single_solves":
                        bool(all(r.iters == q.iters for r, q in zip(res, sq)))})
    return out


def batched_measurement(args):
    """The batched form: (a) 16 right-hand sides of one power-law system
    (n = 65,536, 256 blocks of 256 rows; the source handle and 15 clones, one
    shared sampled block stream); (b) 16 power-law systems with n drawn
    uniformly from [5,000, 200,000] and 3-50 off-diagonals per row, blocks of
    256 rows, one right-hand side each.  Each form runs as one graph launch,
    in mixed precision and FP64; the same solves one after another are timed
    for comparison in mixed precision (for (a) 4 of the 16, scaled)."""
    import torch
    import scipy.sparse as sp
    from paper_2510_02156_gb300 import binding as B
    from paper_2510_02156_gb300 import workloads as W
    out = {}
    s = W.powerlaw(n=1 << 16, num_blocks=256, seed=5, lam=args.lam, tol=args.tol,
                   cache=args.cache)
    A = sp.csr_matrix((s.values.astype(np.float64), s.col_idx, s.row_ptr), shape=(s.m, s.n))
    rng = np.random.default_rng(41)
    bs = [torch.as_tensor(A @ rng.standard_normal(s.n), device="cuda") for _ in range(16)]
    h0 = B.Handle.from_system(s, precision=B.PREC_MIXED)
    hs = [h0] + [h0.clone() for _ in range(15)]
    rhs = {"workload": f"16 right-hand sides, power-law CSR n={s.n}, nnz={s.nnz}, 256 blocks of 256, "
                       f"lambda={s.lam:g}, tol={s.tol:g}"}
    rhs["mixed"] = _batch_vs_sequential(hs, bs, s.tol, args.maxit, B.PREC_MIXED, torch, B,
                                        [0] * 16, seq=4)
    rhs["fp64"] = _batch_vs_sequential(hs, bs, s.tol, args.maxit, B.PREC_FP64, torch, B,
                                       [0] * 16, seq=0)
    for h in hs:
        h.close()
    out["multi_rhs"] = rhs
    sizes = np.random.default_rng(42).integers(5000, 200001, 16)
    systems = [W.powerlaw(n=int(n), num_blocks=max(1, int(n) // 256), seed=100 + i, dmax=50,
                          lam=args.lam, tol=args.tol, cache=args.cache)
               for i, n in enumerate(sizes)]
    hs = [B.Handle.from_system(q, precision=B.PREC_MIXED) for q in systems]
    bs = [torch.as_tensor(q.b, device="cuda") for q in systems]
    ms = {"workload": (f"16 power-law CSR systems, n in [5000, 200000] (total {int(sizes.sum())} rows, "
                       f"{sum(q.nnz for q in systems)} nnz), 3-50 off-diagonals per row, blocks of "
                       f"256 rows, lambda={args.lam:g}, tol={args.tol:g}")}
    ms["mixed"] = _batch_vs_sequential(hs, bs, args.tol, args.maxit, B.PREC_MIXED, torch, B,
                                       list(range(16)))
    ms["fp64"] = _batch_vs_sequential(hs, bs, args.tol, args.maxit, B.PREC_FP64, torch, B,
                                      list(range(16)), seq=0)
    for h in hs:
        h.close()
    out["multi_system"] = ms
    return out


def tuning_dict(t):
    """The launch shapes rorbk_autotune chose, and its per-iteration times."""
    return {"topk_blocks": t.topk_blocks, "collect_blocks": t.collect_blocks,
            "dyn_mark_blocks": t.dyn_mark_blocks, "dyn_scatter_blocks": t.dyn_scatter_blocks,
            "residual_blocks": t.residual_blocks, "graph_unroll": t.graph_unroll,
            "us_per_iteration_default": t.us_default,
            "us_per_iteration_tuned": t.us_tuned}


def mres_bytes(s, nr, vbytes, xbytes):
    """Algorithmic bytes of one block residual R = B - A X for nr columns: A's
    values and column indices once, X read once, B read and R written."""
    return s.nnz * (vbytes + 4) + nr * xbytes * (s.n + 2 * s.m)


def multi_rhs_measurement(args, s, flush, t_single_mixed, t_single_fp64):
    """16 right-hand sides of the main workload as one block (B = A X_true,
    column 0 = b, X_true ~ N(0,1) seed 77): every column solved to the
    tolerance in one graph launch, mixed precision and FP64; each column's
    FP64 RRN re-checked on the host; the block residual k_mres timed alone
    (cold L2) against the HBM roofline.  The one-column solve times of the
    headline give the 16 solves one after another."""
    import torch
    import scipy.sparse as sp
    from paper_2510_02156_gb300 import binding as B
    from paper_2510_02156_gb300 import workloads as W
    nr = 16
    Bm = W.rhs_block(s, nr, seed=77)
    A = sp.csr_matrix((s.values.astype(np.float64), s.col_idx, s.row_ptr), shape=(s.m, s.n))
    h0 = B.Handle.from_system(s, precision=B.PREC_MIXED)
    h = h0.multi(nr)
    Bd = torch.as_tensor(Bm, device="cuda")
    out = {"workload": (f"{nr} right-hand sides of the power-law system n={s.n} (B = A X_true, "
                        f"X_true ~ N(0,1), column 0 = b), one block (rorbk_multi_create), tol={s.tol:g}")}
    out["autotune"] = tuning_dict(h.autotune(Bd, precision=B.PREC_MIXED, iters=args.tune_iters))
    # the mixed block to the tolerance (every column), checked on the host
    X = torch.zeros((s.n, nr), dtype=torch.float64, device="cuda")
    h.solve_multi(Bd, X, tol=s.tol, maxit=3, seed=1, precision=B.PREC_MIXED, inner_tol=args.inner_tol)
    flush.zero_()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = h.solve_multi(Bd, X, tol=s.tol, maxit=args.maxit, seed=1, precision=B.PREC_MIXED,
                        inner_tol=args.inner_tol)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    Xh = X.cpu().numpy()
    rrn_host = [float(np.linalg.norm(Bm[:, j] - A @ Xh[:, j]) / np.linalg.norm(Bm[:, j]))
                for j in range(nr)]
    its = [int(r.iters) for r in res]
    out["mixed"] = {"time_s": dt, "device_ms": float(res[0].time_ms), "iters_max": max(its),
                    "iters_min": min(its), "all_converged": bool(all(r.converged for r in res)),
                    "rrn_host_max": max(rrn_host), "us_per_iteration": dt * 1e6 / max(its),
                    "sequential_one_column_mixed_s": nr * t_single_mixed,
                    "sequential_one_column_fp64_s": nr * t_single_fp64,
                    "speedup_vs_sequential_mixed": nr * t_single_mixed / dt,
                    "speedup_vs_sequential_fp64": nr * t_single_fp64 / dt,
                    "sequential_note": f"{nr} x the one-column solve times (mixed, FP64) of this run"}
    # the FP64 block: a bounded sample of its iterations (the whole solve
    # takes minutes), scaled to the mixed block's iteration count
    X.zero_()
    k = args.multi_fp64_iters
    h.solve_multi(Bd, X, tol=0.0, maxit=3, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h.solve_multi(Bd, X, tol=0.0, maxit=k, seed=1)
    torch.cuda.synchronize()
    per = (time.perf_counter() - t0) / k
    out["fp64"] = {"us_per_iteration": per * 1e6, "sample_iterations": k,
                   "time_s_scaled": per * max(its),
                   "note": f"{k} FP64 block iterations timed, scaled to {max(its)} iterations"}
    out["speedup_mixed_vs_fp64_block"] = per * max(its) / dt
    Xm = torch.as_tensor(np.random.default_rng(3).standard_normal((s.n, nr)) * 0.5, device="cuda")
    B32, X32 = Bd.float(), Xm.float()
    c32, w32 = time_kernel(lambda: h.residual_multi(B32, X32, None, precision=B.PREC_MIXED, wait=False),
                           flush, torch)
    c64, w64 = time_kernel(lambda: h.residual_multi(Bd, Xm, None, wait=False), flush, torch)
    h.close()
    h0.close()
    peak, kind = measured_hbm_peak()
    by32, by64 = mres_bytes(s, nr, 4, 4), mres_bytes(s, nr, 4, 8)
    out["roofline_fp32"] = {"bound": "hbm", "kernel": f"k_mres<float,float,{nr}>",
                            "achieved": by32 / (c32 * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                            "frac": by32 / (c32 * 1e-3) / 1e9 / peak, "bytes_per_launch": by32,
                            "launch_ms_cold_l2": c32, "launch_ms_warm_l2": w32,
                            "traffic": profiled_traffic(f"k_mres<float,float,{nr}>", s),
                            "peak_source": f"{kind} (MEASURED_PEAKS.json hbm_gbs, burst copy)"}
    out["roofline_fp64"] = {"bound": "hbm", "kernel": f"k_mres<double,float,{nr}>",
                            "achieved": by64 / (c64 * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                            "frac": by64 / (c64 * 1e-3) / 1e9 / peak, "bytes_per_launch": by64,
                            "launch_ms_cold_l2": c64, "launch_ms_warm_l2": w64,
                            "traffic": profiled_traffic(f"k_mres<double,float,{nr}>", s)}
    return out


def _batched_system(a):
    i, n, lam, tol, cache = a
    from paper_2510_02156_gb300 import workloads as W
    return W.batched_system(i, n, lam=lam, tol=tol, cache=cache)


def batched_scale_measurement(args, flush):
    """The batched configuration at its stated size, in one graph launch:
    256 power-law systems (n ~ U[5000, 200000], 3-50 off-diagonals per row,
    blocks of 256 rows), each a block of 16 right-hand sides (B = A X_true,
    X_true ~ N(0,1), column 0 = b), plus a dense wide system m = 2,048,
    n = 100,000 (A = U diag(s) V^T, s geometric from 1 to 0.1, 8 blocks of 256
    rows) whose limit from x0 = 0 is the minimum-norm solution (Lemma 2).
    Every column and the dense system solved to the tolerance, mixed precision;
    the dense system's distance to A+ b and to range(A^T) is reported."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import torch
    from paper_2510_02156_gb300 import binding as B
    from paper_2510_02156_gb300 import workloads as W
    nr = 16
    sizes = W.batched_sizes(args.batch_systems)
    t0 = time.time()
    with cf.ProcessPoolExecutor(max_workers=max(1, min(16, os.cpu_count() or 1)),
                                mp_context=mp.get_context("spawn")) as ex:
        systems = list(ex.map(_batched_system, [(i, int(n), args.lam, args.tol, args.cache)
                                                 for i, n in enumerate(sizes)]))
    gen_s = time.time() - t0
    t0 = time.time()
    handles, blocks, Bs, Xs = [], [], [], []
    for i, q in enumerate(systems):
        h = B.Handle.from_system(q, precision=B.PREC_MIXED)
        blocks.append(h.multi(nr))
        handles.append(h)
        # B = A X_true formed on the device (input construction only)
        g = torch.Generator(device="cuda")
        g.manual_seed(1000 + i)
        Xt = torch.randn((q.n, nr), generator=g, device="cuda", dtype=torch.float64)
        At = torch.sparse_csr_tensor(torch.as_tensor(q.row_ptr, device="cuda"),
                                     torch.as_tensor(q.col_idx.astype(np.int64), device="cuda"),
                                     torch.as_tensor(q.values.astype(np.float64), device="cuda"),
                                     size=(q.m, q.n))
        Bq = (At @ Xt).contiguous()
        Bq[:, 0] = torch.as_tensor(q.b, device="cuda")
        Bs.append(Bq)
        Xs.append(torch.zeros((q.n, nr), dtype=torch.float64, device="cuda"))
        del At, Xt
    rows, nnz = int(sum(q.m for q in systems)), int(sum(q.nnz for q in systems))
    del systems
    d = W.dense_usv_cuda(2048, 100_000, seed=4, smin=0.1, block_rows=256, lam=args.dense_wide_lam,
                         tol=args.tol)
    hd = B.Handle.from_system(d, precision=B.PREC_MIXED)
    bd = torch.as_tensor(d.b, device="cuda")
    xd = torch.zeros(d.n, dtype=torch.float64, device="cuda")
    setup_s = time.time() - t0
    members = blocks + [hd]
    bs, xs = Bs + [bd], Xs + [xd]
    out = {"workload": (f"{len(blocks)} power-law CSR systems, n in [5000, 200000] ({rows} rows, {nnz} nnz "
                        f"in total), 3-50 off-diagonals per row, blocks of 256 rows, lambda={args.lam:g}, "
                        f"{nr} right-hand sides each; plus dense A = U diag(s) V^T, 2048 x 100000, s "
                        f"geometric 1..0.1, 8 blocks of 256 rows, lambda={args.dense_wide_lam:g}; "
                        f"tol={args.tol:g}; one graph launch"),
           "generation_s": gen_s, "setup_s": setup_s,
           "right_hand_sides": len(blocks) * nr + 1}
    with B.Batch(members, precision=B.PREC_MIXED) as bt:
        bt.solve(bs, xs, tol=args.tol, maxit=3, seed=1, inner_tol=args.inner_tol)     # warm-up
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        st, res = bt.solve(bs, xs, tol=args.tol, maxit=args.maxit, seed=1, inner_tol=args.inner_tol)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t1
    cols = [r for m in blocks for r in m.multi_results()]
    out["mixed"] = {"time_s": dt, "status": int(st),
                    "all_converged": bool(all(r.converged for r in cols) and res[-1].converged),
                    "iters_max": int(max(r.iters for r in cols)),
                    "iters_sum": int(sum(r.iters for r in cols)),
                    "rhs_solved_per_s": (len(cols) + 1) / dt,
                    "dense_member": {"iters": int(res[-1].iters), "rrn": float(res[-1].rrn),
                                     "refinements": int(res[-1].refinements)}}
    # Lemma 2: from x0 = 0 the iterates stay in range(A^T), so the limit is
    # the minimum-norm solution A+ b; both checked in FP64 on the device
    Ad = torch.as_tensor(d.dense, device="cuda")
    Q, Rf = torch.linalg.qr(Ad.T)               # A^T = Q R: Q spans range(A^T)
    # A x = R^T Q^T x = b with x = Q y: the minimum-norm solution
    xmn = (Q @ torch.linalg.solve_triangular(Rf.T, bd.unsqueeze(1), upper=False)).squeeze(1)
    out["mixed"]["dense_member"]["rel_err_vs_min_norm"] = float(torch.linalg.norm(xd - xmn) / torch.linalg.norm(xmn))
    out["mixed"]["dense_member"]["off_range_rel"] = float(torch.linalg.norm(xd - Q @ (Q.T @ xd)) / torch.linalg.norm(xd))
    del Ad, Q, Rf, xmn
    for m in blocks:
        m.close()
    for h in handles:
        h.close()
    hd.close()
    return out


def dense_measurement(args, flush):
    """The dense least-squares form: A = U diag(s) V^T, m = 200,000, n = 2,048,
    s_i geometric from 1 to 1e-8, 781 blocks of 256 rows, mu = 1e-6 * 256.
    Its condition number (1e8) puts RRN = 1e-8 out of reach of any row-action
    method in a practical number of iterations, so a fixed number of
    iterations is timed (FP64 and mixed) and the RRN reached is reported, with
    the dense residual kernel timed alone against the HBM roofline."""
    import torch
    from paper_2510_02156_gb300 import binding as B
    from paper_2510_02156_gb300 import workloads as W
    s = W.dense_usv_cuda(200_000, 2048, seed=2, block_rows=256, lam=2.56e-4, tol=args.tol)
    t0 = time.time()
    h = B.Handle.from_system(s, precision=B.PREC_MIXED)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    b = torch.as_tensor(s.b, device="cuda")
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    out = {"workload": (f"dense A = U diag(s) V^T, m={s.m}, n={s.n}, s geometric 1..1e-8, "
                        f"{s.num_blocks} blocks of 256 rows (781 = floor(m/256)), lambda=2.56e-4, "
                        f"x0=0, Philox seed 1"),
           "setup_s": setup_s, "iterations": args.dense_iters}
    for name, prec in (("fp64", B.PREC_FP64), ("mixed", B.PREC_MIXED)):
        h.solve(b, x, tol=0.0, maxit=5, seed=1, precision=prec)            # warm-up
        flush.zero_()
        torch.cuda.synchronize()
        r = h.solve(b, x, tol=0.0, maxit=args.dense_iters, seed=1, precision=prec)
        xh = x.cpu().numpy()
        out[name] = {"ms_per_iteration": r.time_ms / max(1, r.iters), "iters": int(r.iters),
                     "rrn": float(np.linalg.norm(s.dense @ xh - s.b) / np.linalg.norm(s.b)),
                     "refinements": int(r.refinements)}
    # the residual over the dense A (its CSR form) timed alone, cold L2
    x64 = torch.as_tensor(s.x_true, device="cuda") * 0.5
    r64 = torch.empty(s.m, dtype=torch.float64, device="cuda")
    cold64, warm64 = time_kernel(lambda: h.residual_async(b, x64, r64), flush, torch, reps=10)
    b32, x32 = b.float(), x64.float()
    r32 = torch.empty(s.m, dtype=torch.float32, device="cuda")
    cold32, warm32 = time_kernel(lambda: h.residual32(b32, x32, r32, wait=False), flush, torch,
                                 reps=10)
    peak, kind = measured_hbm_peak()
    mn = s.m * s.n
    by64 = mn * 8 + 8 * (s.n + 2 * s.m)       # a dense GEMV: A once, x, b, r
    by32 = mn * 4 + 4 * (s.n + 2 * s.m)
    out["residual_fp64"] = {"bound": "hbm", "launch_ms_cold_l2": cold64, "launch_ms_warm_l2": warm64,
                            "bytes_per_launch": by64, "achieved": by64 / (cold64 * 1e-3) / 1e9,
                            "peak": peak, "unit": "GB/s", "frac": by64 / (cold64 * 1e-3) / 1e9 / peak,
                            "note": "algorithmic bytes of a dense GEMV; the CSR form also reads "
                                    "4 bytes of column index per entry"}
    out["residual_fp32"] = {"bound": "hbm", "launch_ms_cold_l2": cold32, "launch_ms_warm_l2": warm32,
                            "bytes_per_launch": by32, "achieved": by32 / (cold32 * 1e-3) / 1e9,
                            "peak": peak, "unit": "GB/s", "frac": by32 / (cold32 * 1e-3) / 1e9 / peak}
    h.close()
    del s
    return out


def incremental_measurement(args, s, h, b, x, flush):
    """The main workload solved with the incremental residual (r -= A dx from
    the iteration's change log through a CSC copy of A; an exact residual every
    50 iterations and to confirm convergence), FP64 and mixed; the relative
    residual of the returned x is measured again on the host in FP64."""
    import scipy.sparse as sp
    import torch
    from paper_2510_02156_gb300 import binding as B
    A = sp.csr_matrix((s.values.astype(np.float64), s.col_idx, s.row_ptr), shape=(s.m, s.n))
    bn = float(np.linalg.norm(s.b))
    out = {"residual_mode": "incremental", "refresh": 50}
    for name, prec in (("mixed", B.PREC_MIXED), ("fp64", B.PREC_FP64)):
        kw = dict(seed=1, precision=prec, inner_tol=args.inner_tol,
                  residual_mode=B.RESIDUAL_INCREMENTAL)
        h.solve(b, x, tol=s.tol, maxit=20, **kw)                   # CSC copy, log, graph
        flush.zero_()
        torch.cuda.synchronize()
        r = h.solve(b, x, tol=s.tol, maxit=args.maxit, **kw)
        xh = x.cpu().numpy()
        out[name] = {"time_s": r.time_ms / 1e3, "iters": int(r.iters),
                     "us_per_iteration": r.time_ms / max(1, r.iters) * 1e3,
                     "rrn": float(r.rrn), "rrn_host_fp64": float(np.linalg.norm(A @ xh - s.b) / bn),
                     "converged": bool(r.converged)}
    return out


def fabgmres_measurement(args):
    """Algorithm 3 on the 262,144-unknown power-law system (1024 blocks of 256
    rows): flexible AB-GMRES whose preconditioner is a ROR-BK solve of at most
    200 iterations to a relative residual of 0.1, to tolerance 1e-8, with FP64
    and with mixed inner solves, beside plain ROR-BK on the same system.  (On
    the 2^20 system these inner solves are too short: 400 outer steps stop at
    a relative residual of 0.054.)"""
    import torch
    from paper_2510_02156_gb300 import binding as B
    from paper_2510_02156_gb300 import workloads as W
    s = W.powerlaw(n=1 << 18, num_blocks=1024, seed=1, lam=args.lam, tol=args.tol,
                   cache=args.cache)
    h = B.Handle.from_system(s, precision=B.PREC_MIXED)
    b = torch.as_tensor(s.b, device="cuda")
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    out = {"algorithm": "Algorithm 3 (flexible AB-GMRES, ROR-BK inner solves)",
           "workload": f"power-law sparse square CSR, n={s.n}, nnz={s.nnz}, 1024 blocks of 256, "
                       f"lambda={s.lam:g}, tol={s.tol:g}, seed 1",
           "eta": 0.1, "lmax": 200, "max_outer": 400}
    for name, prec in (("mixed", B.PREC_MIXED), ("fp64", B.PREC_FP64)):
        h.fabgmres(b, x, tol=s.tol, maxit=2, eta=0.1, lmax=20, seed=1, precision=prec)  # graphs
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = h.fabgmres(b, x, tol=s.tol, maxit=400, eta=0.1, lmax=200, seed=1, precision=prec)
        torch.cuda.synchronize()
        out[name] = {"time_s": time.perf_counter() - t0, "outer": int(r.iters),
                     "inner_iterations": int(r.refinements), "rrn": float(r.rrn),
                     "converged": bool(r.converged)}
    for name, prec in (("plain_rorbk_mixed", B.PREC_MIXED), ("plain_rorbk_fp64", B.PREC_FP64)):
        h.solve(b, x, tol=s.tol, maxit=20, seed=1, precision=prec, inner_tol=args.inner_tol)
        r = h.solve(b, x, tol=s.tol, maxit=args.maxit, seed=1, precision=prec,
                    inner_tol=args.inner_tol)
        out[name] = {"time_s": r.time_ms / 1e3, "iters": int(r.iters), "rrn": float(r.rrn),
                     "converged": bool(r.converged)}
    h.close()
    return out


def weighted_measurement(args):
    """Iterations and time to tolerance of the FP64 solve with the paper's
    static proposal and with residual-weighted draws (not in the paper), on
    the 262,144-unknown power-law system (1024 blocks of 256 rows)."""
    import torch
    from paper_2510_02156_gb300 import binding as B
    from paper_2510_02156_gb300 import workloads as W
    s = W.powerlaw(n=1 << 18, num_blocks=1024, seed=1, lam=args.lam, tol=args.tol,
                   cache=args.cache)
    h = B.Handle.from_system(s)
    b = torch.as_tensor(s.b, device="cuda")
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    out = {"workload": f"power-law sparse square CSR, n={s.n}, nnz={s.nnz}, 1024 blocks of 256, "
                       f"lambda={s.lam:g}, tol={s.tol:g}, FP64, seed 1"}
    for name, mode in (("paper", B.DIST_PAPER), ("residual_weighted", B.DIST_RESIDUAL_WEIGHTED)):
        h.solve(b, x, tol=s.tol, maxit=20, seed=1, dist_mode=mode)           # builds the graph
        r = h.solve(b, x, tol=s.tol, maxit=args.maxit, seed=1, dist_mode=mode)
        out[name] = {"iters": int(r.iters), "time_s": r.time_ms / 1e3,
                     "us_per_iteration": r.time_ms / max(1, r.iters) * 1e3,
                     "rrn": float(r.rrn), "converged": bool(r.converged)}
    h.close()
    return out


def autograd_measurement(args):
    """Forward solve and adjoint backward of L = 0.5 ||x - x_t||^2 on the
    262,144-unknown power-law system (1024 blocks of 256 rows), to the bench
    tolerance, through the torch.autograd.Function, twice on one SolveSpec:
    the first forward sets its handle up (from device copies of the pattern
    and values), the second, with every value changed by a relative 1e-3
    N(0,1), refreshes it on the device (rorbk_update_values).  Wall times
    include that set-up or refresh and the adjoint handle's set-up (device
    transpose); the solve times are the device loops'."""
    import torch
    from paper_2510_02156_gb300 import autograd as AG
    from paper_2510_02156_gb300 import workloads as W
    s = W.powerlaw(n=1 << 18, num_blocks=1024, seed=1, lam=args.lam, tol=args.tol,
                   cache=args.cache)
    x_t = torch.as_tensor(np.random.default_rng(26).standard_normal(s.n), device="cuda")
    v0 = s.values.astype(np.float64)
    v1 = v0 * (1.0 + 1e-3 * np.random.default_rng(28).standard_normal(v0.size))
    spec = AG.SolveSpec(np.asarray(s.row_ptr, np.int32), np.asarray(s.col_idx, np.int32), s.m, s.n,
                        s.num_blocks, s.lam, tol=s.tol, maxit=args.maxit)
    out = {"workload": f"power-law sparse square CSR, n={s.n}, nnz={s.nnz}, 1024 blocks of 256, "
                       f"lambda={s.lam:g}, tol={s.tol:g}; L = 0.5||x - x_t||^2"}
    for name, v in (("first", v0), ("second", v1)):
        vals = torch.tensor(v, device="cuda", requires_grad=True)
        b = torch.tensor(s.b, device="cuda", requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x = AG.RorbkSolve.apply(vals, b, spec)
        loss = 0.5 * ((x - x_t) ** 2).sum()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        loss.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        f, a = spec.last_forward, spec.last_adjoint
        out[name] = {"forward_s": t1 - t0, "backward_s": t2 - t1,
                     "forward_solve_s": f.time_ms / 1e3, "adjoint_solve_s": a.time_ms / 1e3,
                     "forward_iters": int(f.iters), "adjoint_iters": int(a.iters),
                     "forward_rrn": float(f.rrn), "adjoint_rrn": float(a.rrn),
                     "converged": bool(f.converged and a.converged)}
    out["handles_set_up"] = spec.setups
    out["second_forward_wall_over_solve"] = out["second"]["forward_s"] / out["second"]["forward_solve_s"]
    spec.close()
    return out


def cpu_model():
    """The host CPU's model name (lscpu), or the machine type."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def oracle_per_iteration(s, iters):
    """Seconds per iteration of the FP64 oracle on this solve (its residual and
    top-K on all host cores, the block solves on one), from a bounded run of
    `iters` iterations; the oracle's set-up (orthogonality) is timed
    separately and removed."""
    import oracle
    t0 = time.perf_counter()
    res = oracle.solve(s, maxit=iters, tol=0.0, seed=1)
    total = time.perf_counter() - t0
    t1 = time.perf_counter()
    oracle.orthogonality(s, s.num_blocks)
    setup = time.perf_counter() - t1
    return max(total - setup, 1e-9) / max(1, res.iters), res.iters


def cpu_baseline(s, args, iters_to_tol):
    import oracle
    per_it, done = oracle_per_iteration(s, args.oracle_iters)
    cores = oracle.thread_count(s.m)
    return {"value": per_it * iters_to_tol, "unit": "s", "cores": cores, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": (f"{done} FP64 oracle iterations of this solve from x0 = 0 (residual and "
                       f"top-K on {cores} host threads, block solves on one; "
                       f"{per_it * 1e3:.1f} ms/iteration, set-up excluded), scaled to the "
                       f"{iters_to_tol} iterations the solve takes")}


def reference_iterations(args):
    """Iterations the FP64 oracle needs on this workload, recorded by
    oracle/record_iterations.py (a run of the oracle alone)."""
    p = os.path.join(ROOT, "oracle", "iterations_to_tol.json")
    key = f"powerlaw_n{args.n}_k{args.blocks}_lam{args.lam:g}_tol{args.tol:g}_seed1"
    if os.path.exists(p):
        d = json.load(open(p))
        if key in d:
            return int(d[key]), "recorded by oracle/record_iterations.py"
    return None, "not recorded"


def run_reference(args, rank, world, local):
    if rank != 0:
        return
    s = workload(args, 0)
    iters, src = reference_iterations(args)
    import oracle
    per, walls = [], []
    for _ in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        per_it, done = oracle_per_iteration(s, args.oracle_iters)
        walls.append(time.perf_counter() - t0)
        per.append(per_it)
    per_it = float(np.mean(per[args.warmup:]))
    step_s = float(np.mean(walls[args.warmup:]))
    cores = oracle.thread_count(s.m)
    if iters is None:
        print(json.dumps({"impl": "reference",
                          "unavailable": "the oracle's iteration count on this workload is not "
                                         "recorded (run oracle/record_iterations.py)"}))
        return
    val = per_it * iters
    # a step is the bounded sample (its wall time is ms_per_step); value is the
    # time to tolerance it implies: the sample's seconds per iteration times
    # the oracle's own recorded iteration count
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3,
            "value_note": (f"{per_it * 1e3:.1f} ms per oracle iteration (each step a sample of "
                           f"{args.oracle_iters} iterations) x {iters} iterations to tolerance"),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args, s),
            "cpu_baseline": {"value": val, "unit": "s", "cores": cores, "kind": "oracle",
                             "cpu": cpu_model(),
                             "sample": (f"{args.oracle_iters} oracle iterations per step (residual "
                                        f"and top-K on {cores} host threads), "
                                        f"{per_it * 1e3:.1f} ms/iteration (set-up excluded), "
                                        f"scaled to {iters} iterations to tolerance ({src})")},
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_profile(args):
    import torch
    from paper_2510_02156_gb300 import binding as B
    s = workload(args, 0)
    h = B.Handle.from_system(s, precision=B.PREC_MIXED)
    b = torch.as_tensor(s.b, device="cuda")
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    for prec in (B.PREC_MIXED, B.PREC_FP64):
        res = h.solve(b, x, tol=s.tol, maxit=args.profile, seed=1, precision=prec,
                      inner_tol=args.inner_tol, host_loop=1, poll=args.profile)
        print(f"profile run: precision {prec}: {res.iters} iterations, "
              f"{res.time_ms / max(1, res.iters) * 1e3:.1f} us/iteration (host-driven loop)")
    h.close()


def run_profile_dense(args):
    import torch
    from paper_2510_02156_gb300 import binding as B
    from paper_2510_02156_gb300 import workloads as W
    prec = B.PREC_MIXED if args.profile_dense == "mixed" else B.PREC_FP64
    s = W.gaussian_dense(25_600, 2048, seed=8, num_blocks=100, lam=2.56e-4)
    with B.Handle.from_system(s, precision=prec) as h:
        b = torch.as_tensor(s.b, device="cuda")
        x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
        res = h.solve(b, x, tol=0.0, maxit=2, seed=1, precision=prec, host_loop=1)
        torch.cuda.synchronize()
    print(f"dense profile run ({args.profile_dense}): {res.iters} iterations, rrn {res.rrn:.4e}")


def run_profile_multi(args):
    import torch
    from paper_2510_02156_gb300 import binding as B
    from paper_2510_02156_gb300 import workloads as W
    s = workload(args, 0)
    nr = 16
    h0 = B.Handle.from_system(s, precision=B.PREC_MIXED)
    h = h0.multi(nr)
    Bd = torch.as_tensor(W.rhs_block(s, nr, seed=77), device="cuda")
    Xm = torch.as_tensor(np.random.default_rng(3).standard_normal((s.n, nr)) * 0.5, device="cuda")
    # three FP32 block residuals, then three FP64 ones (the launches a
    # traffic capture of k_mres takes), then the iterations
    for _ in range(3):
        h.residual_multi(Bd.float(), Xm.float(), None, precision=B.PREC_MIXED, wait=False)
    for _ in range(3):
        h.residual_multi(Bd, Xm, None, wait=False)
    X = torch.zeros((s.n, nr), dtype=torch.float64, device="cuda")
    res = h.solve_multi(Bd, X, tol=s.tol, maxit=args.profile_multi, seed=1, precision=B.PREC_MIXED,
                        inner_tol=args.inner_tol, host_loop=1, poll=args.profile_multi)
    torch.cuda.synchronize()
    print(f"profile run: {nr} columns, {res[0].iters} iterations, "
          f"{res[0].time_ms / max(1, res[0].iters) * 1e3:.1f} us/iteration (host-driven loop)")
    h.close()
    h0.close()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.profile:
        run_profile(args)
        return
    if args.profile_multi:
        run_profile_multi(args)
        return
    if args.profile_dense:
        run_profile_dense(args)
        return
    if args.impl == "reference":
        run_reference(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
