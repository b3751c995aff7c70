"""Serve one seeded Poisson stream through the engine and print its summary.

    python -m paper_2108_02025_gb300.serve_case [--requests 2000] [--rate 1e7] [--bf16]
        [--drawn] [--budget-gb 64] [--pool-log2 30] [--chunk-mb 256] [--loads]

The stream is the serving workload (70% GEMV / 20% DOT / 10% GER, m and n
log-uniform in [32, 16384], 4 streams), on resident operand pools of
2^pool-log2 FP32 and BF16 values (or with every operand drawn per request,
--drawn) under an HBM budget of --budget-gb GB; with the default rate every
request arrives at once, which measures capacity.  Pool GEMVs and GERs
moving more than --chunk-mb MB run in row chunks of about that size (0:
whole).  With --loads the stream is served at saturation and then, the same
requests, at 50%, 80% and 95% of the measured rate.  Used to profile the
engine's kernels in isolation (a small budget and pool keep the device
footprint of a profiler capture small) and to choose the chunk size.
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
    p.add_argument("--drawn", action="store_true", help="operands drawn per request, no pool")
    p.add_argument("--budget-gb", type=float, default=64.0)
    p.add_argument("--pool-log2", type=int, default=30)
    p.add_argument("--chunk-mb", type=float, default=None, help="row chunk size (default: the benchmark's)")
    p.add_argument("--loads", action="store_true", help="saturation, then 50/80/95%% of it")
    args = p.parse_args(argv)
    import bench
    import paper_2108_02025_gb300 as gb
    form = gb.FORM_BF16 if args.bf16 else gb.FORM_F32
    chunk = bench.SERVE_CHUNK if args.chunk_mb is None else int(args.chunk_mb * (1 << 20))
    if args.loads:
        r = bench.serve_loads(args.requests, form, seed=args.seed, chunk_bytes=chunk, pool=not args.drawn)
        r = {"chunk_bytes": chunk, "saturated": r["saturated"]["solves_per_s"],
             "loads": {f: (v["solves_per_s"], v["p50_us"], v["p99_us"]) for f, v in r["loads"].items()}}
    else:
        r = bench.serve_once(args.requests, args.rate, form, seed=args.seed, sample=0, pool=not args.drawn,
                             budget=int(args.budget_gb * (1 << 30)), pool_elems=1 << args.pool_log2,
                             chunk_bytes=chunk)
    print(json.dumps(r))


if __name__ == "__main__":
    main()
