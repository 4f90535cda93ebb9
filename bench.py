"""Benchmark: time to ||Ax-b||/||b|| <= 1e-8 with ROR-BK on one GB300.

Workload (default): the 2^20-row power-law CSR system (FP32-stored values,
row nnz power law alpha=2.5 in [3,200] plus the diagonal, rows scaled
log-uniform [1e-4,1]), 4096 contiguous row blocks, lambda=1e-8, tol=1e-8,
x0 = 0.  One benchmark step is one whole solve from x0 = 0 to the tolerance
(every iteration of Algorithm 1: 3 sampled static updates, the full residual,
the top-K selection and the dynamic update).  The setup (Algorithm 1 steps
1-4) runs once before timing and is reported separately.

Arms:
  (default)          the CUDA library through its C ABI
  --impl reference   the FP64 CPU oracle on the host cores, a bounded sample
                     of iterations per step, extrapolated to the same solve

Prints one JSON line (rank 0).  Under torchrun every rank solves its own
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
    p.add_argument("--maxit", type=int, default=2_000_000)
    p.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "both"])
    p.add_argument("--oracle-iters", type=int, default=40)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cache", default=os.path.join(ROOT, ".cache"))
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args, rank):
    from paper_2510_02156_gb300 import workloads as W
    return W.powerlaw(n=args.n, num_blocks=args.blocks, seed=1 + rank, lam=args.lam,
                      tol=args.tol, cache=args.cache)


def config(args, s, extra=None):
    c = {"workload": f"powerlaw CSR n={s.n} nnz={s.nnz} k={s.num_blocks} blocks "
                     f"(s=K={s.m // s.num_blocks}), FP32-stored A, lambda={s.lam:g}, "
                     f"tol={s.tol:g}, x0=0, seed={1}",
         "step": "one whole solve to tolerance", "l2": "flushed between timed steps"}
    if extra:
        c.update(extra)
    return c


class ClockSampler:
    """nvidia-smi clocks/throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
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


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def residual_bytes(s, fp32_values):
    """Algorithmic bytes of one r = b - A x launch: the CSR arrays once,
    x once, b read, r written (FP64 vectors)."""
    vb = 4 if fp32_values else 8
    return s.nnz * (vb + 4) + 4 * (s.m + 1) + 8 * s.n + 8 * s.m + 8 * s.m


def time_residual(h, s, torch, flush, reps=20):
    """Average device time of the residual kernel (the same kernel and grid
    as inside the solve), each launch after an L2 flush (cold) and back to
    back without flush (warm, L2-resident working set)."""
    b = torch.as_tensor(s.b, device="cuda")
    x = torch.as_tensor(s.x_true, device="cuda") * 0.5
    r = torch.empty(s.m, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    for _ in range(3):
        h.residual(b, x, r)
    torch.cuda.synchronize()
    cold = []
    for _ in range(reps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        h.residual_async(b, x, r)
        e1.record(st)
        e1.synchronize()
        cold.append(e0.elapsed_time(e1))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        h.residual_async(b, x, r)
    e1.record(st)
    e1.synchronize()
    warm = e0.elapsed_time(e1) / reps
    return float(np.mean(cold)), float(warm)


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
    precs = {"fp64": [B.PREC_FP64], "mixed": [B.PREC_MIXED],
             "both": [B.PREC_FP64, B.PREC_MIXED]}[args.precision]
    h = B.Handle.from_system(s, precision=B.PREC_MIXED if B.PREC_MIXED in precs else B.PREC_FP64)
    torch.cuda.synchronize()
    setup_s = time.time() - t0
    b = torch.as_tensor(s.b, device="cuda")
    x = torch.zeros(s.n, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    results = {}
    for prec in precs:
        for _ in range(args.warmup):
            flush.zero_()
            h.solve(b, x, tol=s.tol, maxit=args.maxit, seed=1, precision=prec)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        times, iters, rrns, refs = [], [], [], []
        with ClockSampler(local) as clk:
            for _ in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                res = h.solve(b, x, tol=s.tol, maxit=args.maxit, seed=1, precision=prec)
                e1.record(stream)
                e1.synchronize()
                times.append(e0.elapsed_time(e1) / 1e3)
                iters.append(res.iters)
                rrns.append(res.rrn)
                refs.append(res.refinements)
        torch.cuda.synchronize()
        t_step = float(np.mean(times))
        if dist:
            tt = torch.tensor([t_step], device="cuda")
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t_step = float(tt.item())
        xh = x.cpu().numpy()
        # end to end through the host-buffer entry point
        bh = np.ascontiguousarray(s.b)
        xo = np.zeros(s.n)
        e2e = []
        for _ in range(max(1, min(args.steps, 2))):
            flush.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            h.solve_host(bh, xo, tol=s.tol, maxit=args.maxit, seed=1, precision=prec)
            e2e.append(time.perf_counter() - t1)
        results[prec] = {
            "time_s": t_step, "iters": int(iters[-1]), "rrn": float(rrns[-1]),
            "refinements": int(refs[-1]),
            "rel_err_vs_x_true": float(np.linalg.norm(xh - s.x_true) / np.linalg.norm(s.x_true)),
            "e2e_s": float(np.mean(e2e)), "clocks": clk.summary(),
            "launches_per_step": 1 + 5 * int(iters[-1]),
        }

    fp32_vals = s.values.dtype == np.float32
    cold_ms, warm_ms = time_residual(h, s, torch, flush)
    peak, peak_kind = measured_peaks()
    nbytes = residual_bytes(s, fp32_vals)
    h.close()
    if rank != 0:
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    head = results[B.PREC_MIXED] if B.PREC_MIXED in results else results[B.PREC_FP64]
    ach = nbytes / (cold_ms * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": head["time_s"], "unit": "s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["time_s"] * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if B.PREC_MIXED not in results else "f32+f64",
        "data": "synthetic", "setup_s": setup_s,
        "config": config(args, s, {"precision": args.precision, "solves_per_s_all_ranks": world / head["time_s"]}),
        "fp64": _public(results.get(B.PREC_FP64)), "mixed": _public(results.get(B.PREC_MIXED)),
        "e2e": {"value": head["e2e_s"], "unit": "s", "h2d_bytes_per_step": 8 * s.m,
                "d2h_bytes_per_step": 8 * s.n},
        "gpu_launches": head["launches_per_step"] * args.steps,
        "clocks": head["clocks"],
        "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                     "frac": ach / peak, "traffic": None,
                     "kernel": "k_residual (r = b - A x, FP64 accumulate, FP32-stored A)",
                     "bytes_per_launch": nbytes, "launch_ms_cold_l2": cold_ms,
                     "launch_ms_warm_l2": warm_ms, "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(s, args, head["iters"])
    print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def _public(r):
    if r is None:
        return None
    return {k: v for k, v in r.items() if k not in ("clocks",)}


def cpu_baseline(s, args, iters_to_tol):
    """The oracle, as it stands, on a bounded sample: args.oracle_iters
    iterations of the same solve (setup excluded), scaled to the GPU run's
    iteration count."""
    import oracle
    M = oracle.oracle.prepare(s)
    t0 = time.perf_counter()
    res = oracle.solve(s, maxit=args.oracle_iters, tol=0.0, seed=1)
    dt = time.perf_counter() - t0
    # subtract the oracle's own setup (orthogonality) measured separately
    t1 = time.perf_counter()
    oracle.orthogonality(s, s.num_blocks)
    setup = time.perf_counter() - t1
    per_it = max(dt - setup, 1e-9) / max(1, res.iters)
    del M
    return {"value": per_it * iters_to_tol, "unit": "s", "cores": 1, "kind": "oracle",
            "sample": f"{res.iters} FP64 oracle iterations of this solve on 1 host core "
                      f"({per_it * 1e3:.1f} ms/iteration, setup excluded), scaled to the "
                      f"{iters_to_tol} iterations the solve takes"}


def run_reference(args, rank, world, local):
    if rank != 0:
        return
    s = workload(args, 0)
    import oracle
    oracle.orthogonality(s, s.num_blocks)   # warm caches / page in
    per = []
    for _ in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        res = oracle.solve(s, maxit=args.oracle_iters, tol=0.0, seed=1)
        per.append((time.perf_counter() - t0) / max(1, res.iters))
    per_it = float(np.mean(per[args.warmup:]))
    iters = reference_iterations(args)
    val = per_it * iters
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": val * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args, s),
            "cpu_baseline": {"value": val, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.oracle_iters} oracle iterations per step (setup "
                                       f"included), {per_it * 1e3:.1f} ms/iteration, scaled to "
                                       f"{iters} iterations to tolerance"},
            "e2e": {"value": val, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reference_iterations(args):
    """Iterations Algorithm 1 needs on this workload (a property of the
    method and the seeded input, identical for every exact FP64
    implementation), recorded by the oracle's own full run."""
    p = os.path.join(ROOT, "oracle", "iterations_to_tol.json")
    if os.path.exists(p):
        d = json.load(open(p))
        key = f"powerlaw_n{args.n}_k{args.blocks}_lam{args.lam:g}_tol{args.tol:g}_seed1"
        if key in d:
            return int(d[key])
    return 1


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
