"""Iteration counts of the benchmark sequence, solved by the oracle (writes bench_counts.json).

ORACLE / TEST INFRASTRUCTURE ONLY.  The CPU-baseline leg and the reference arm of bench.py time
the oracle on a bounded sample and convert seconds per iteration into solves per second with
the oracle's own iterations per pair over the whole sequence, which this script records once:
the 2-D convection-diffusion sequence (512 x 512 grid, 20 pairs, convection (10, 10) drifting
1 % per pair, seed 2000, b and bt ~ N(0, 1)) solved by Algorithm 2 with the Section 4 refresh,
k = 20, s = 40, tol 1e-8, with the same stagnation guard (1.5) as the library's default.

Usage: python -m oracle.bench_counts   (about two hours on eight cores)
"""
import json
import os
import sys
import time

import numpy as np

from . import rbicg_oracle as O

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "bench_counts.json")


def main():
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_1010_0762_gb300 import inputs as I

    grid, pairs, k, s, tol, guard = 512, 20, 20, 40, 1e-8, 1.5
    seq = I.convdiff_sequence(grid, [10.0, 10.0], pairs, 0.01, 2000, bt_kind="normal")
    t0 = time.perf_counter()
    done = []

    def on_pair(j, r):
        done.append(r)
        print("pair %d: %d iterations, status %d, fallback %s (%.0f s)"
              % (j, r.iters, r.status, r.hist["fallback"], time.perf_counter() - t0), flush=True)

    O.rbicg_sequence(seq, k=k, s=s, tol=tol, guard=guard, on_pair=on_pair)
    iters = [int(r.iters) for r in done]
    out = {"workload": "convdiff2d-%dx%d-seq%d-k%d" % (grid, grid, pairs, k),
           "params": {"k": k, "s": s, "tol": tol, "guard": guard, "svd_tol": 1e-6, "seed": 2000,
                      "drift": 0.01, "c0": [10.0, 10.0]},
           "iters_per_pair": iters, "mean_iters": float(np.mean(iters)),
           "statuses": [int(r.status) for r in done],
           "fallback": [bool(r.hist["fallback"]) for r in done],
           "oracle_seconds": round(time.perf_counter() - t0, 1)}
    with open(OUT, "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main()
