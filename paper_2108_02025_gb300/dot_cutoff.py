"""Single-block versus multi-block DOT on the GPU: where the crossover lies.

    python -m paper_2108_02025_gb300.dot_cutoff [--out PATH] [--reps 200]

The paper runs DOT on one core below a cutoff and on all cores above it,
the cutoff being where one vector outgrows the L1 cache (Sec. 4.3.1, the
analysis of the two DOT forms; cutoff chosen at twice the L1 size).  On the
GPU the two forms are one block (Alg. 3) and a grid of blocks with a
combined sum (Alg. 4).  This study builds two copies of the library, one
that always takes the single block (up to 64 MiB per vector) and one that
always takes the grid, times gb_sdot and gb_ddot in each for vector sizes
from 1 KiB to 64 MiB (CUDA events around a graph of `reps` back-to-back
calls on the same vectors, so small sizes are L2-resident as in repeated
use and the host's issue rate does not count), and
reports per size both times and the crossover: the smallest size from
which the grid is never slower.  The library's GB_DOT_SMALL_BYTES is set
from it.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

SIZES_BYTES = [1 << k for k in range(10, 27)] + [3 << k for k in range(9, 25)]
VARIANTS = {"single": 1 << 26, "grid": 0}


def time_variant(reps):
    """In a process whose GBBLAS_LIB is one variant: {dtype: {bytes: us}}."""
    import torch
    import paper_2108_02025_gb300 as gb
    import synth
    out = {}
    st = torch.cuda.current_stream()
    for name, dt, e in (("f32", torch.float32, 4), ("f64", torch.float64, 8)):
        res = {}
        for nbytes in sorted(SIZES_BYTES):
            n = nbytes // e
            x = torch.empty(n, dtype=dt, device="cuda")
            y = torch.empty(n, dtype=dt, device="cuda")
            a = torch.zeros(1, dtype=dt, device="cuda")
            synth.fill_uniform(x, 0, 1)
            synth.fill_uniform(y, 0, 2)
            nb = gb.gb_workspace_bytes(gb.OP_DOT, gb.F32 if e == 4 else gb.F64, 0, 0, n)
            ws = torch.zeros(max(nb, 1), dtype=torch.uint8, device="cuda")
            f = gb.lib().gb_sdot if e == 4 else gb.lib().gb_ddot
            args = (n, x.data_ptr(), y.data_ptr(), a.data_ptr(), ws.data_ptr(), nb, st.cuda_stream)
            for _ in range(5):
                assert f(*args) == 0
            # the calls are replayed from a CUDA graph, so the host's issue
            # rate does not hide the kernels' own time
            cap = torch.cuda.Stream()
            cap.wait_stream(st)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap):
                cargs = args[:-1] + (cap.cuda_stream,)
                for _ in range(reps):
                    f(*cargs)
            st.wait_stream(cap)
            g.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            best = None
            for _ in range(3):
                e0.record(st)
                g.replay()
                e1.record(st)
                e1.synchronize()
                t = e0.elapsed_time(e1) * 1e3 / reps
                best = t if best is None else min(best, t)
            res[nbytes] = round(best, 3)
            del g
        out[name] = res
    return out


def main(argv=None):
    p = argparse.ArgumentParser(description="single-block vs grid DOT crossover")
    p.add_argument("--out", default=None, help="write the JSON result here")
    p.add_argument("--reps", type=int, default=200)
    p.add_argument("--child", default=None, help=argparse.SUPPRESS)
    args = p.parse_args(argv)
    if args.child:
        print(json.dumps(time_variant(args.reps)))
        return
    import paper_2108_02025_gb300.build as bld  # noqa: F401  (by path: importing the package needs the library)
    tmp = tempfile.mkdtemp(prefix="dot_cutoff_")
    times = {}
    for name, small in VARIANTS.items():
        lib = bld.build_variant(os.path.join(tmp, name), {"GB_DOT_SMALL_BYTES": small})
        env = dict(os.environ, GBBLAS_LIB=lib)
        r = subprocess.run([sys.executable, "-m", "paper_2108_02025_gb300.dot_cutoff", "--child", name,
                            "--reps", str(args.reps)], env=env, capture_output=True, text=True, cwd=ROOT)
        if r.returncode != 0:
            raise RuntimeError(r.stderr)
        times[name] = json.loads(r.stdout.strip().splitlines()[-1])
    result = {"sizes_bytes": sorted(SIZES_BYTES), "us": times, "crossover_bytes": {}}
    for dt in ("f32", "f64"):
        s, g = times["single"][dt], times["grid"][dt]
        cross = None
        for nbytes in sorted(SIZES_BYTES):
            k = str(nbytes)
            if all(g[str(b)] <= s[str(b)] for b in sorted(SIZES_BYTES) if b >= nbytes):
                cross = nbytes
                break
        result["crossover_bytes"][dt] = cross
        print(f"{dt}: crossover at {cross} bytes per vector")
        for nbytes in sorted(SIZES_BYTES):
            print(f"  {nbytes:>10d} B  single {s[str(nbytes)]:9.2f} us  grid {g[str(nbytes)]:9.2f} us")
    if args.out:
        with open(args.out, "w") as f:
            json.dump(result, f, indent=1)


if __name__ == "__main__":
    main()
