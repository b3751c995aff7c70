"""Run one GEMV, DOT or GER case on the GPU and print its time and bandwidth.

    python -m paper_2108_02025_gb300.run_case gemv f32 row 64 1048576 [--reps 20]
    python -m paper_2108_02025_gb300.run_case dot f64 - 1 268435456
    python -m paper_2108_02025_gb300.run_case ger f64 col 16384 16384
    python -m paper_2108_02025_gb300.run_case gemvq e4m3 row 32768 32768
    python -m paper_2108_02025_gb300.run_case batch f32 row 256 0

Inputs are uniform[-1,1] from the synth generator (seed 0), written on the
device; for ``gemvq`` (A stored as BF16 or E4M3 with per-row scales) A is
N(0,1) with rows scaled by 10^U[-3,3], quantised before timing; for ``batch`` (one batched launch of m FP32 GEMVs,
sizes log-uniform in [32, 8192], the autotuned table) n is ignored.  Each call is timed with CUDA events on the launching stream; the
median is reported with the algorithmic bytes (every element touched once)
per second.  Used to profile one kernel in isolation.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    p = argparse.ArgumentParser(description="one GEMV / DOT / GER case")
    p.add_argument("op", choices=["gemv", "dot", "ger", "gemvq", "batch"])
    p.add_argument("dtype", choices=["f32", "f64", "bf16", "e4m3"])
    p.add_argument("layout", choices=["row", "col", "-"])
    p.add_argument("m", type=int)
    p.add_argument("n", type=int)
    p.add_argument("--reps", type=int, default=20)
    args = p.parse_args(argv)

    import torch
    import paper_2108_02025_gb300 as gb
    import synth

    dt = torch.float64 if args.dtype == "f64" else torch.float32
    e = 8 if args.dtype == "f64" else 4
    m, n = args.m, args.n
    lay = gb.COL_MAJOR if args.layout == "col" else gb.ROW_MAJOR

    def filled(numel, stream):
        t = torch.empty(max(numel, 1), dtype=dt, device="cuda")
        synth.fill_uniform(t, 0, stream)
        return t

    if args.op == "gemv":
        A, x, c = filled(m * n, 1), filled(n, 2), filled(m, 3)
        ld = n if lay == gb.ROW_MAJOR else m
        call = lambda: gb.gemv(A, x, c, 1.0, lay, m, n, ld)
        nbytes = e * (m * n + n + 2 * m)
    elif args.op == "gemvq":
        A = torch.empty((m, n), dtype=torch.float32, device="cuda")
        synth.fill_normal_rows(A, 0, 1, -3.0, 3.0)
        x, c = filled(n, 2), filled(m, 3)
        Q, sc = gb.quantize(A, args.dtype)
        del A
        call = lambda: gb.gemv_q(Q, sc, x, c, 1.0, n=n)
        nbytes = (2 if args.dtype == "bf16" else 1) * m * n + 4 * n + 8 * m + (4 * m if sc is not None else 0)
    elif args.op == "batch":
        import bench
        wl = bench.BatchWorkload(torch.device("cuda", torch.cuda.current_device()), count=m)
        b = gb.Batch(wl.problems, table=gb.load_tuning())
        call = lambda: b.launch()
        nbytes = wl.bytes
    elif args.op == "dot":
        x, y, a = filled(n, 4), filled(n, 5), filled(1, 6)
        call = lambda: gb.dot(x, y, a, n)
        nbytes = e * (2 * n + 2)
    else:
        C, x, y = filled(m * n, 7), filled(m, 8), filled(n, 9)
        ld = n if lay == gb.ROW_MAJOR else m
        call = lambda: gb.ger(x, y, C, 1.0, lay, m, n, ld)
        nbytes = e * (2 * m * n + m + n)

    for _ in range(3):
        call()
    torch.cuda.synchronize()
    st = torch.cuda.current_stream()
    times = []
    for _ in range(args.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        call()
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    med = statistics.median(times)
    print(json.dumps({"op": args.op, "dtype": args.dtype, "layout": args.layout, "m": m, "n": n,
                      "us_median": round(med * 1e6, 2), "us_min": round(min(times) * 1e6, 2),
                      "GB_s": round(nbytes / med / 1e9, 1), "bytes": nbytes}))


if __name__ == "__main__":
    main()
