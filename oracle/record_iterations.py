"""Record how many iterations the FP64 oracle needs to reach the tolerance on
the benchmark workload (the 2^20-row power-law system, 4096 blocks,
lambda = 1e-8, tol = 1e-8, x0 = 0, seed 1), and the solution it reaches.
Calls only the oracle; the count is written to iterations_to_tol.json beside
this file (the benchmark's reference arm scales its bounded per-iteration
sample by it) and the solution to x_<key>.npy (the benchmark states the
mixed-precision result's distance to it).

    python oracle/record_iterations.py [--n 1048576] [--blocks 4096]
"""
import argparse
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402

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
    xfile = f"x_{key}.npy"
    np.save(os.path.join(HERE, xfile), res.x)
    d[key + "_meta"] = {"converged": bool(res.converged), "rrn": res.rrn,
                        "oracle_seconds": dt, "threads": oracle.thread_count(s.m),
                        "x_file": xfile, "x_sha256": hashlib.sha256(res.x.tobytes()).hexdigest()}
    json.dump(d, open(path, "w"), indent=1, sort_keys=True)
    print(key, res.iters, res.converged, res.rrn, f"{dt:.0f}s")


if __name__ == "__main__":
    main()
