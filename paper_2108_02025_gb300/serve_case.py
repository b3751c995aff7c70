"""Serve one seeded Poisson stream through the engine and print its summary.

    python -m paper_2108_02025_gb300.serve_case [--requests 2000] [--rate 1e7] [--bf16]

The stream is the serving workload (70% GEMV / 20% DOT / 10% GER, m and n
log-uniform in [32, 16384], 64 GB budget, 4 streams); with the default rate
every request arrives at once, which measures capacity.  Used to profile
the engine's kernels in isolation.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    p = argparse.ArgumentParser(description="one serving stream")
    p.add_argument("--requests", type=int, default=2000)
    p.add_argument("--rate", type=float, default=1e7)
    p.add_argument("--bf16", action="store_true")
    p.add_argument("--seed", type=int, default=1)
    args = p.parse_args(argv)
    import bench
    import paper_2108_02025_gb300 as gb
    r = bench.serve_once(args.requests, args.rate, gb.FORM_BF16 if args.bf16 else gb.FORM_F32, seed=args.seed,
                         sample=0)
    print(json.dumps(r))


if __name__ == "__main__":
    main()
