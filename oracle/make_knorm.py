"""Writes the stored spectral norms ||K||_2 of the synthetic solve operators.

Power iteration on K^T K in the CPU oracle (FP64), started from a seeded
Gaussian vector; the result is what ``inputs.scaled_operator`` divides by to
reach ||K||_2 = 0.5.  Calls only the oracle and the input generator.

    python oracle/make_knorm.py [--threads T] [--only d21_r48_s3 ...]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import oracle  # noqa: E402
from paper_1511_06029_gb300 import inputs  # noqa: E402

# (d, r_max, seed): mixed-precision refinement operator (d = 21, r_max = 48),
# the serving operators (one per d in 14..22, r_max = 32) and small ones used
# by the tests.
SERVE_SEED_BASE = 5000
ENTRIES = ([(21, 48, 3)]
           + [(d, 32, SERVE_SEED_BASE + d) for d in range(14, 23)]
           + [(d, 8, 7000 + d) for d in range(6, 13)])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--max-iter", type=int, default=40)
    ap.add_argument("--rtol", type=float, default=1e-4)
    ap.add_argument("--only", nargs="*", default=None)
    args = ap.parse_args()
    path = os.path.join(inputs._DATA, "knorm.json")
    os.makedirs(os.path.dirname(path), exist_ok=True)
    table = inputs.knorm_table()
    todo = sorted(ENTRIES, key=lambda e: (e[0], e[1]))
    for d, rmax, seed in todo:
        key = inputs.knorm_key(d, rmax, seed)
        if args.only and key not in args.only:
            continue
        if key in table and not args.only:
            continue
        K = inputs.synthetic_operator(d, rmax, seed)
        v0 = np.random.default_rng(seed + 99).standard_normal(K.N)
        t0 = time.time()
        sigma, it = oracle.power_norm(K, v0, max_iter=args.max_iter, rtol=args.rtol,
                                      threads=args.threads)
        table[key] = {"sigma": sigma, "iters": it, "max_iter": args.max_iter,
                      "rtol": args.rtol, "seconds": round(time.time() - t0, 1)}
        print(key, table[key], flush=True)
        with open(path + ".tmp", "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
        os.replace(path + ".tmp", path)


if __name__ == "__main__":
    main()
