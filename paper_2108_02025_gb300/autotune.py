"""Autotuner of the batched FP32 GEMV (gb_sgemv_batch) tiling table.

    python -m paper_2108_02025_gb300.autotune [--out PATH] [--gb 1.0] [--reps 5]

The batched kernel takes, per bucket ceil(log2 n) of a problem's column
count, three parameters: lanes per row, 16-byte packs per lane in flight,
and the bytes of A per tile.  For every bucket b in [--lo, --hi] (default
5..13, n from 17 to 8192) this tool builds a synthetic batch on the GPU --
n uniform in (2^(b-1), 2^b], m log-uniform in [32, 8192], about --gb GB of
A, uniform[-1,1] -- times one launch of it under every candidate with CUDA
events (median of --reps after a warm-up launch), and keeps the fastest.
The result is a JSON table {"buckets": {b: [lanes, packs, tile_bytes]}, ...}
with the measured GB/s of the winner and of the built-in entry; the binding
(``load_tuning``) reads it from ``batch_tuning.json`` beside this file.

With --mix N the table is tuned on a whole mixed batch instead: N problems
drawn like the batched benchmark's (m, n log-uniform in [32, 8192]) but
with another seed, starting from the current table, one bucket at a time
in order of its share of the bytes, keeping a candidate only when the whole
batch gets at least 0.5% faster (buckets interact through the load balance
of the shared launch, which a per-bucket batch does not see).

Tuning changes the summation order of a row (lanes per row, packs per
iteration), so results are bit-reproducible for a fixed table, and every
candidate stays within the FP32 tolerance of the oracle (the GPU tests run
all kernel variants).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

LANES = (1, 2, 4, 8, 16, 32)
PACKS = (1, 2, 4)
TILE_BYTES = (32 << 10, 128 << 10, 512 << 10, 2 << 20)


def bucket_batch(b, gbytes, seed, device):
    """Problems of bucket b (n in (2^(b-1), 2^b]) totalling about `gbytes` GB of A."""
    import numpy as np
    import torch
    import synth
    lo_n, hi_n = (1 << (b - 1)) + 1, 1 << b
    budget = int(gbytes * 1e9) // 4   # elements of A
    draw = 1 << 16
    m_all = synth.log_uniform_integers(draw, seed, 401 + b, 32, 8192)
    n_all = synth.integers(draw, seed, 432 + b, lo_n, hi_n, np.int64)
    cum = np.cumsum(m_all * ((n_all + 3) // 4 * 4))
    k = max(1, int(np.searchsorted(cum, budget)))
    ms, ns = m_all[:k].tolist(), n_all[:k].tolist()
    m = np.array(ms, np.int64)
    n = np.array(ns, np.int64)
    lda = (n + 3) // 4 * 4

    def offsets(sizes):
        padded = (sizes + 63) // 64 * 64
        return np.concatenate([[0], np.cumsum(padded)[:-1]]).astype(np.int64), int(padded.sum())

    a_off, na = offsets(m * lda)
    x_off, nx = offsets(n)
    c_off, nc = offsets(m)
    A = torch.empty(na, dtype=torch.float32, device=device)
    x = torch.empty(nx, dtype=torch.float32, device=device)
    c = torch.empty(nc, dtype=torch.float32, device=device)
    synth.fill_uniform(A, seed, 403)
    synth.fill_uniform(x, seed, 404)
    synth.fill_uniform(c, seed, 405)
    probs = [(A.data_ptr() + 4 * int(a_off[p]), x.data_ptr() + 4 * int(x_off[p]),
              c.data_ptr() + 4 * int(c_off[p]), 1.0, int(m[p]), int(n[p]), int(lda[p]))
             for p in range(len(m))]
    nbytes = int((4 * (m * n + n + 2 * m)).sum())
    return probs, nbytes, (A, x, c)


def time_table(probs, table, stream, reps):
    import torch
    import paper_2108_02025_gb300 as gb
    batch = gb.Batch(probs, table=table)
    batch.launch(stream)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        batch.launch(stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return statistics.median(times)


def candidates(b):
    packs_row = max(1, (1 << b) // 4)  # 16-byte packs in the bucket's longest row
    for lpr in LANES:
        if lpr > 2 * packs_row and lpr > 1:
            continue
        for u in PACKS:
            for tb in TILE_BYTES:
                yield lpr, u, tb


def tune(lo=5, hi=13, gbytes=1.0, reps=5, seed=0, log=print):
    import torch
    import paper_2108_02025_gb300 as gb
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    default = gb.tuning_table()
    out = {"buckets": {}, "measured": {}, "device": torch.cuda.get_device_name(dev),
           "sms": torch.cuda.get_device_properties(dev).multi_processor_count,
           "gb_per_bucket": gbytes, "reps": reps}
    for b in range(lo, hi + 1):
        probs, nbytes, keep = bucket_batch(b, gbytes, seed, dev)
        d = default[b]
        t_def = time_table(probs, default, stream, reps)
        best = ((d.lanes_per_row, d.packs_per_iter, d.tile_bytes), t_def)
        tried = 0
        for cand in candidates(b):
            t = time_table(probs, gb.tuning_table({b: cand}), stream, reps)
            tried += 1
            if t < best[1]:
                best = (cand, t)
        out["buckets"][str(b)] = list(best[0])
        out["measured"][str(b)] = {"problems": len(probs), "bytes": nbytes, "candidates": tried,
                                   "best_GB_s": round(nbytes / best[1] / 1e9, 1),
                                   "default_GB_s": round(nbytes / t_def / 1e9, 1),
                                   "default": [d.lanes_per_row, d.packs_per_iter, d.tile_bytes]}
        log(f"bucket {b}: {len(probs)} problems, {nbytes / 1e9:.2f} GB, best {best[0]} "
            f"{nbytes / best[1] / 1e9:.1f} GB/s, built-in {nbytes / t_def / 1e9:.1f} GB/s")
        del probs, keep
        torch.cuda.empty_cache()
    return out


def tune_mix(count=4096, seed=1, reps=3, passes=1, start=None, log=print):
    """Coordinate descent on a mixed batch: the batched benchmark's recipe
    (m, n log-uniform in [32, 8192]) drawn with another seed, timed whole.
    Buckets are visited by their share of the batch's bytes, and a bucket's
    entry changes only when the whole batch gets at least 0.5% faster."""
    import numpy as np
    import torch
    import bench
    import paper_2108_02025_gb300 as gb
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    wl = bench.BatchWorkload(dev, count=count, seed=seed)
    table = gb.tuning_table() if start is None else start
    entries = {b: (table[b].lanes_per_row, table[b].packs_per_iter, table[b].tile_bytes)
               for b in range(gb.BATCH_BUCKETS)}
    buckets = np.array([max(0, int(np.ceil(np.log2(max(int(v), 1))))) for v in wl.n])
    weight = {int(b): int((wl.m * wl.n)[buckets == b].sum()) for b in np.unique(buckets)}
    order = sorted(weight, key=lambda b: -weight[b])
    best_t = time_table(wl.problems, gb.tuning_table(entries), stream, reps)
    t_start = best_t
    log(f"mix of {count} problems: start {best_t * 1e3:.3f} ms")
    for _ in range(passes):
        for b in order:
            for cand in candidates(b):
                if cand == entries[b]:
                    continue
                trial = dict(entries)
                trial[b] = cand
                t = time_table(wl.problems, gb.tuning_table(trial), stream, reps)
                if t < best_t * 0.995:
                    best_t, entries = t, trial
            log(f"bucket {b}: {entries[b]}, batch {best_t * 1e3:.3f} ms")
    out = {"buckets": {str(b): list(entries[b]) for b in order},
           "mix": {"problems": count, "seed": seed, "bytes": wl.bytes, "start_ms": round(t_start * 1e3, 3),
                   "tuned_ms": round(best_t * 1e3, 3)},
           "device": torch.cuda.get_device_name(dev)}
    del wl
    torch.cuda.empty_cache()
    return out


def main(argv=None):
    import paper_2108_02025_gb300 as gb
    p = argparse.ArgumentParser(description="autotune the batched GEMV tiling table")
    p.add_argument("--out", default=gb.TUNING_PATH)
    p.add_argument("--lo", type=int, default=5)
    p.add_argument("--hi", type=int, default=13)
    p.add_argument("--gb", type=float, default=1.0, help="GB of A per bucket's batch")
    p.add_argument("--reps", type=int, default=5)
    p.add_argument("--mix", type=int, default=0,
                   help="tune on a mixed batch of this many problems (coordinate descent) instead of per bucket")
    args = p.parse_args(argv)
    t0 = time.time()
    if args.mix:
        out = tune_mix(args.mix, reps=3, start=gb.load_tuning())
    else:
        out = tune(args.lo, args.hi, args.gb, args.reps)
    out["seconds"] = round(time.time() - t0, 1)
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
    print(f"wrote {args.out} in {out['seconds']} s")


if __name__ == "__main__":
    main()
