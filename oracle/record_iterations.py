"""Record how many iterations the FP64 oracle needs to reach the tolerance on
the benchmark workload (the 2^20-row power-law system, 4096 blocks,
lambda = 1e-8, tol = 1e-8, x0 = 0, seed 1).  Calls only the oracle; the
result is written to iterations_to_tol.json beside this file and is used by
the benchmark's reference arm to scale its bounded per-iteration sample.

    python oracle/record_iterations.py [--n 1048576] [--blocks 4096]
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import oracle  # noqa: E402
from paper_2510_02156_gb300 import workloads as W  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=1 << 20)
    ap.add_argument("--blocks", type=int, default=4096)
    ap.add_argument("--lam", type=float, default=1e-8)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=400000)
    ap.add_argument("--seed", type=int, default=1)
    args = ap.parse_args()
    s = W.powerlaw(n=args.n, num_blocks=args.blocks, seed=1, lam=args.lam, tol=args.tol)
    t0 = time.time()
    res = oracle.solve(s, maxit=args.maxit, seed=args.seed)
    dt = time.time() - t0
    key = f"powerlaw_n{args.n}_k{args.blocks}_lam{args.lam:g}_tol{args.tol:g}_seed{args.seed}"
    path = os.path.join(HERE, "iterations_to_tol.json")
    d = json.load(open(path)) if os.path.exists(path) else {}
    d[key] = res.iters
    d[key + "_meta"] = {"converged": bool(res.converged), "rrn": res.rrn,
                        "oracle_seconds": dt, "cores": 1}
    json.dump(d, open(path, "w"), indent=1, sort_keys=True)
    print(key, res.iters, res.converged, res.rrn, f"{dt:.0f}s")


if __name__ == "__main__":
    main()
