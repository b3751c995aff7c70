"""Benchmark of the GEMV / DOT / GER hot path on GB300.

One step = one pass of the plain-method sweep through the C ABI, inputs
uniform[-1,1] from the counter-based generator, resident in HBM:

    for FP32 and FP64:
      GEMV c += A x, A 16384x16384, 1048576x64 and 64x1048576, row-major
      DOT  alpha += x.y, n = 2^28
      GER  C += x y^T, 16384x16384, row-major
      GEMV (the same three shapes), column-major
      GER  16384x16384, column-major

(18 kernel launches).  Every large operand (A, C, the DOT vectors) is bigger
than the 129 MB L2 and consecutive calls touch different buffers, so no
call starts with its operand in L2.  The metric is algorithmic HBM bytes
(every element of A / C / x / y / c touched once) per second over the whole
step; per-operation figures and the roofline of the dominant kernel are
reported beside it.

Beside the device-timed value the line carries: `e2e` (the same step with
inputs uploaded from pinned host memory and results downloaded every step,
with the host link measured in the same run and the step bound it sets),
`cpu_baseline` (the CPU oracle on a bounded sample: all cores, one core,
and the compensated oracle), and the growth legs `precision` (BF16 / E4M3
GEMV), `batched` (4096 GEMVs in one persistent launch) and `serving` (the
engine on resident operand pools: saturated throughput, p50 / p99 at 50%,
80% and 95% load, and the same stream with operands drawn per request).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs its own replica on its own GPU (the operations
do not shard: "replicas only"); the step time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "GEMV/DOT/GER HBM GB/s vs peak; served solves/s + p99 at stated error"
WORKLOAD = ("plain-method sweep, FP32 and FP64: GEMV 16384x16384, 1048576x64, 64x1048576 "
            "(row- and column-major), DOT n=2^28, GER 16384x16384 (row- and column-major); "
            "inputs uniform[-1,1]")
SQ, TALL, WIDE = (16384, 16384), (1048576, 64), (64, 1048576)
NDOT = 1 << 28
HBM_FALLBACK_GBS = 6800.0
CPU_FRACTION = 16    # cpu_baseline sample: 1/16 of a step
NOMINAL_HBM_GBS = 8000.0   # HBM3e data-sheet bandwidth, for a second fraction beside the measured peak
REF_FRACTION = 32    # reference arm: 1/32 of a step per step
OP_CALLS, OP_REPS = 10, 3   # per-operation timing: calls back to back per event pair, pairs
SMS, DP_FMA_PER_CLK_SM, SM_MAX_MHZ = 152, 2, 2070.0   # FP64 pipe: 2 FMA/clk/SM (1.26 TFLOP/s at 2.07 GHz)


# --------------------------------------------------------------- workload --

def op_list():
    """(name, kind, dtype, layout, m, n) in launch order; dtype 'f32'/'f64'."""
    ops = []
    for dt in ("f32", "f64"):
        for lay, tag in ((0, "row"), (1, "col")):
            for (m, n), sh in ((SQ, "sq"), (TALL, "tall"), (WIDE, "wide")):
                ops.append((f"gemv_{tag}_{sh}_{dt}", "gemv", dt, lay, m, n))
            if lay == 0:
                ops.append((f"dot_{dt}", "dot", dt, 0, 1, NDOT))
            ops.append((f"ger_{tag}_{dt}", "ger", dt, lay, SQ[0], SQ[1]))
    return ops


def esize(dt):
    return 4 if dt == "f32" else 8


def alg_bytes(kind, dt, m, n):
    """Compulsory HBM bytes of one call: every element touched once."""
    e = esize(dt)
    if kind == "gemv":
        return e * (m * n + n + 2 * m)          # A, x read; c read and written
    if kind == "dot":
        return e * (2 * n + 2)                  # x, y read; alpha read and written
    return e * (2 * m * n + m + n)              # C read and written; x, y read


def alg_flops(kind, m, n):
    return 2 * m * n if kind in ("gemv", "ger") else 2 * n


class Workload:
    """Device buffers of one step and a launcher for every operation."""

    def __init__(self, device):
        import torch
        import synth
        import paper_2108_02025_gb300 as gb
        self.gb = gb
        self.lib = gb.lib()
        self.dev = device
        self.ops = op_list()
        self.buf = {}
        tdt = {"f32": torch.float32, "f64": torch.float64}

        def make(key, numel, dt, stream):
            t = torch.empty(numel, dtype=tdt[dt], device=device)
            synth.fill_uniform(t, 0, stream)
            self.buf[key] = t
            return t

        st = gen_streams()
        for dt in ("f32", "f64"):
            for (m, n), sh in ((SQ, "sq"), (TALL, "tall"), (WIDE, "wide")):
                make(("A", sh, dt), m * n, dt, st[("A", sh, dt)])
                make(("x", sh, dt), n, dt, st[("x", sh, dt)])
                make(("c", sh, dt), m, dt, st[("c", sh, dt)])
            make(("dx", dt), NDOT, dt, st[("dx", dt)])
            make(("dy", dt), NDOT, dt, st[("dy", dt)])
            make(("alpha", dt), 1, dt, st[("alpha", dt)])
            for tag in ("row", "col"):
                make(("C", tag, dt), SQ[0] * SQ[1], dt, st[("C", tag, dt)])
            make(("gx", dt), SQ[0], dt, st[("gx", dt)])
            make(("gy", dt), SQ[1], dt, st[("gy", dt)])
        # one zeroed workspace per operation (each call leaves it zeroed)
        self.ws = {}
        for (name, kind, dt, lay, m, n) in self.ops:
            code = gb.F32 if dt == "f32" else gb.F64
            op = gb.OP_GEMV if kind == "gemv" else gb.OP_DOT if kind == "dot" else gb.OP_GER
            nb = gb.gb_workspace_bytes(op, code, lay, m, n)
            self.ws[name] = (torch.zeros(max(nb, 1), dtype=torch.uint8, device=device), nb)
        torch.cuda.synchronize(device)

    def shape_key(self, m, n):
        return "sq" if (m, n) == SQ else "tall" if (m, n) == TALL else "wide"

    def launch(self, op, stream_handle):
        name, kind, dt, lay, m, n = op
        lib, b = self.lib, self.buf
        ws, nb = self.ws[name]
        if kind == "gemv":
            sh = self.shape_key(m, n)
            f = lib.gb_sgemv if dt == "f32" else lib.gb_dgemv
            lda = n if lay == 0 else m
            st = f(lay, m, n, 1.0, b[("A", sh, dt)].data_ptr(), lda, b[("x", sh, dt)].data_ptr(),
                   b[("c", sh, dt)].data_ptr(), ws.data_ptr(), nb, stream_handle)
        elif kind == "dot":
            f = lib.gb_sdot if dt == "f32" else lib.gb_ddot
            st = f(n, b[("dx", dt)].data_ptr(), b[("dy", dt)].data_ptr(), b[("alpha", dt)].data_ptr(),
                   ws.data_ptr(), nb, stream_handle)
        else:
            tag = "row" if lay == 0 else "col"
            f = lib.gb_sger if dt == "f32" else lib.gb_dger
            st = f(lay, m, n, 1.0, b[("gx", dt)].data_ptr(), b[("gy", dt)].data_ptr(),
                   b[("C", tag, dt)].data_ptr(), n if lay == 0 else m, stream_handle)
        if st != 0:
            raise RuntimeError(f"{name}: status {st} ({self.gb.gb_status_string(st)})")

    # tensors each step reads from the host (e2e) and the results it returns
    def inputs(self):
        return [t for k, t in self.buf.items()]

    def results(self):
        b = self.buf
        out = []
        for dt in ("f32", "f64"):
            out += [b[("c", sh, dt)] for sh in ("sq", "tall", "wide")]
            out += [b[("alpha", dt)], b[("C", "row", dt)], b[("C", "col", dt)]]
        return out


# ----------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi clock / throttle samples taken every 100 ms."""

    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.samples = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.5)

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append((time.time(), parts))

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)

    def summary(self, t0, t1):
        inside = [p for (t, p) in self.samples if t0 <= t <= t1]
        window = "timed region"
        if len(inside) < 3:
            inside = [p for (_, p) in self.samples]
            window = "warm-up and timed region"
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(p[1]) for p in inside if num(p[1]) is not None]
        smax = [num(p[2]) for p in inside if num(p[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for p in inside for i in range(4) if p[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(inside), "window": window}


# -------------------------------------------------------------- multi-GPU --

def dist_info():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return world, rank, local


def init_dist(backend):
    import torch.distributed as dist
    world, rank, _ = dist_info()
    if world > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend, world_size=world, rank=rank)
    return world, rank


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over all ranks (the value itself without a group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(bytes_per_step: float, steps: int, world: int, max_seconds: float) -> float:
    """GB/s of all replicas together: every rank moved bytes_per_step each step."""
    return bytes_per_step * steps * world / max_seconds / 1e9


# ------------------------------------------------------------ CPU oracle --

def gen_streams():
    """Generator stream of every buffer, in the order Workload fills them."""
    st, s = {}, 1
    for dt in ("f32", "f64"):
        for sh in ("sq", "tall", "wide"):
            st[("A", sh, dt)], st[("x", sh, dt)], st[("c", sh, dt)] = s, s + 1, s + 2
            s += 3
        st[("dx", dt)], st[("dy", dt)], st[("alpha", dt)] = s, s + 1, s + 2
        s += 3
        st[("C", "row", dt)], st[("C", "col", dt)] = s, s + 1
        s += 2
        st[("gx", dt)], st[("gy", dt)] = s, s + 1
        s += 2
    return st


def oracle_sample(fraction: int, seed: int = 0, acc: bool = False):
    """A bounded sample of one step for the CPU oracle: 1/fraction of the
    rows of each row-major GEMV/GER (at least one), of the columns of each
    column-major one, and of the DOT vectors, with the same generator values
    the GPU step uses; GEMV and DOT by the plain definitions, or by the
    compensated (Dot2) oracle with acc.  Returns [(callable, algorithmic
    bytes)]."""
    import numpy as np
    import oracle
    import synth
    st = gen_streams()
    work = []
    for (name, kind, dt, lay, m, n) in op_list():
        npdt = np.float32 if dt == "f32" else np.float64
        if kind == "gemv":
            sh = "sq" if (m, n) == SQ else "tall" if (m, n) == TALL else "wide"
            if lay == 0:
                k = max(1, m // fraction)
                A = synth.uniform(k * n, seed, st[("A", sh, dt)], npdt)
                x = synth.uniform(n, seed, st[("x", sh, dt)], npdt)
                c = synth.uniform(k, seed, st[("c", sh, dt)], npdt)
                work.append((lambda A=A, x=x, c=c, k=k, n=n: oracle.gemv(0, k, n, 1.0, A, n, x, c, acc=acc),
                             alg_bytes("gemv", dt, k, n)))
            else:
                k = max(1, n // fraction)
                A = synth.uniform(m * k, seed, st[("A", sh, dt)], npdt)
                x = synth.uniform(k, seed, st[("x", sh, dt)], npdt)
                c = synth.uniform(m, seed, st[("c", sh, dt)], npdt)
                work.append((lambda A=A, x=x, c=c, k=k, m=m: oracle.gemv(1, m, k, 1.0, A, m, x, c, acc=acc),
                             alg_bytes("gemv", dt, m, k)))
        elif kind == "dot":
            k = max(1, n // fraction)
            x = synth.uniform(k, seed, st[("dx", dt)], npdt)
            y = synth.uniform(k, seed, st[("dy", dt)], npdt)
            work.append((lambda x=x, y=y, k=k: oracle.dot(k, x, y, 0.0, acc=acc),
                         alg_bytes("dot", dt, 1, k)))
        else:
            tag = "row" if lay == 0 else "col"
            k = max(1, (m if lay == 0 else n) // fraction)
            C = synth.uniform(k * (n if lay == 0 else m), seed, st[("C", tag, dt)], npdt)
            x = synth.uniform(m, seed, st[("gx", dt)], npdt)
            y = synth.uniform(n, seed, st[("gy", dt)], npdt)
            if lay == 0:
                work.append((lambda C=C, x=x, y=y, k=k: oracle.ger(0, k, n, 1.0, x[:k], y, C, n),
                             alg_bytes("ger", dt, k, n)))
            else:
                work.append((lambda C=C, x=x, y=y, k=k: oracle.ger(1, m, k, 1.0, x, y[:k], C, m),
                             alg_bytes("ger", dt, m, k)))
    return work


def time_sample(work):
    """Seconds the oracle takes over one pass of the sample, and its bytes."""
    t, b = 0.0, 0
    for f, by in work:
        t0 = time.perf_counter()
        f()
        t += time.perf_counter() - t0
        b += by
    return t, b


# -------------------------------------------------------------- roofline --

def code_of(text: str) -> str:
    """C/C++ source without its comments and blank space, so that a change
    of comments alone does not count as a change of the kernel."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def source_sha(files=None):
    """sha256 of the code of the kernel sources (all of csrc/, or the named
    files), comments left out."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2108_02025_gb300", "csrc")
    names = sorted(files) if files else sorted(f for f in os.listdir(csrc) if f.endswith((".cu", ".cuh", ".h")))
    for f in names:
        h.update(f.encode())
        with open(os.path.join(csrc, f), encoding="utf-8") as fh:
            h.update(code_of(fh.read()).encode())
    return h.hexdigest()


def measured_traffic(op_name):
    """DRAM bytes per launch of `op_name` from the committed ncu summary
    (profiles/dram_traffic.json), or None when absent or when the kernel's
    sources changed since the capture."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except (OSError, ValueError):
        return None
    k = d.get("kernels", {}).get(op_name)
    if k is None or k.get("sha") != source_sha(k.get("sources")):
        return None
    return k.get("dram_bytes_per_launch")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return HBM_FALLBACK_GBS, "fallback"


def roofline_of(op, avg_s, hbm_gbs, src):
    name, kind, dt, lay, m, n = op
    by = alg_bytes(kind, dt, m, n)
    t_hbm = by / (hbm_gbs * 1e9)
    dp_peak_tflops = SMS * DP_FMA_PER_CLK_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    t_alu = alg_flops(kind, m, n) / (dp_peak_tflops * 1e12) if dt == "f64" else 0.0
    if t_alu > t_hbm:
        ach = alg_flops(kind, m, n) / avg_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": round(ach, 4),
                "peak": round(dp_peak_tflops, 4), "unit": "TFLOP/s", "frac": round(ach / dp_peak_tflops, 4),
                "traffic": measured_traffic(name),
                "note": "FP64 FMA pipe, 152 SMs x 2 FMA/clk x 2.07 GHz; HBM frac "
                        f"{by / avg_s / 1e9 / hbm_gbs:.3f} of {src}"}
    ach = by / avg_s / 1e9
    return {"kernel": name, "bound": "hbm", "achieved": round(ach, 1), "peak": hbm_gbs,
            "unit": "GB/s", "frac": round(ach / hbm_gbs, 4), "peak_source": src,
            "traffic": measured_traffic(name), "algorithmic_bytes": by}


# ------------------------------------------------------- precision leg --

PREC_N = 32768
PREC_WORKLOAD = ("GEMV 32768x32768 row-major, A = N(0,1) with row i scaled by 10^U[-3,3] (FP32 "
                 "master), stored as FP32 / BF16 / FP8-E4M3 with per-row FP32 scales; x uniform[-1,1] "
                 "FP32; c FP32")
PREC_BOUND = {"fp32": 2.0 ** -20, "bf16": 2.0 ** -9, "e4m3": 2.0 ** -4}


def precision_bytes(form, m, n):
    """Compulsory bytes of one reduced-precision GEMV: A's codes (and scales), x, c."""
    a = {"fp32": 4, "bf16": 2, "e4m3": 1}[form] * m * n
    return a + 4 * n + 8 * m + (4 * m if form == "e4m3" else 0)


def quantize_bytes(form, m, n):
    """Compulsory bytes of one quantiser call: the FP32 master read, the codes
    (and row scales) written."""
    return 4 * m * n + (2 * m * n if form == "bf16" else m * n + 4 * m)


def run_precision(device, stream, reps=20, sample_rows=64):
    """Solves/s of the 32768^2 GEMV with A stored as FP32 (plain method), BF16
    and E4M3, timed with CUDA events (median of `reps` calls; A is larger
    than L2), and the error of each form against an FP64 evaluation (numpy)
    of the FP32 master on `sample_rows` seeded rows, relative to
    sum_j |A_ij x_j|.  Beside each reduced form: the time of the quantiser
    that prepares A in it (quantize_us) and its compulsory GB/s."""
    import numpy as np
    import torch
    import synth
    import paper_2108_02025_gb300 as gb
    m = n = PREC_N
    A = torch.empty((m, n), dtype=torch.float32, device=device)
    synth.fill_normal_rows(A, 0, 201, -3.0, 3.0)
    x = torch.empty(n, dtype=torch.float32, device=device)
    synth.fill_uniform(x, 0, 203)
    c = torch.zeros(m, dtype=torch.float32, device=device)
    rows = np.unique(synth.integers(sample_rows, 0, 204, 0, m - 1, np.int64))
    A_rows = A[torch.from_numpy(rows).to(device)].double().cpu().numpy()
    xh = x.double().cpu().numpy()
    want = A_rows @ xh
    mag = np.abs(A_rows) @ np.abs(xh)
    out = {"workload": PREC_WORKLOAD, "error": "max over sampled rows of |c_i - (A x)_i| / "
           "sum_j |A_ij x_j|, FP64 numpy on the FP32 master", "sampled_rows": int(rows.size)}
    forms = {}
    for form in ("fp32", "bf16", "e4m3"):
        if form == "fp32":
            call = lambda: gb.gemv(A, x, c, 1.0, gb.ROW_MAJOR, stream=stream)
        else:
            Q, sc = gb.quantize(A, form, stream=stream)
            call = lambda Q=Q, sc=sc: gb.gemv_q(Q, sc, x, c, 1.0, n=n, stream=stream)
        c.zero_()
        call()
        got = c[torch.from_numpy(rows).to(device)].double().cpu().numpy()
        err = float(np.max(np.abs(got - want) / mag))
        for _ in range(3):
            call()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            gpu_lead(stream)
            e0.record(stream)
            call()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3)
        t = statistics.median(times)
        forms[form] = {"us": round(t * 1e6, 2), "solves_per_s": round(1.0 / t, 1),
                       "GB_s": round(precision_bytes(form, m, n) / t / 1e9, 1),
                       "max_rel_err": float(f"{err:.3e}"), "bound": PREC_BOUND[form]}
        if form != "fp32":
            # the preparation of A in this form: one quantiser call into the
            # same code buffers, timed alone (A larger than L2)
            if form == "bf16":
                qcall = lambda Q=Q: gb.lib().gb_quantize_bf16(m, n, A.data_ptr(), n, Q.data_ptr(), Q.stride(0),
                                                              stream.cuda_stream)
            else:
                qcall = lambda Q=Q, sc=sc: gb.lib().gb_quantize_e4m3(m, n, A.data_ptr(), n, Q.data_ptr(),
                                                                     Q.stride(0), sc.data_ptr(), stream.cuda_stream)
            assert qcall() == 0
            qt = []
            for _ in range(max(5, reps // 2)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                gpu_lead(stream)
                e0.record(stream)
                qcall()
                e1.record(stream)
                e1.synchronize()
                qt.append(e0.elapsed_time(e1) / 1e3)
            tq = statistics.median(qt)
            qbytes = quantize_bytes(form, m, n)
            forms[form].update({"quantize_us": round(tq * 1e6, 2), "quantize_GB_s": round(qbytes / tq / 1e9, 1),
                                "quantize_bytes": qbytes})
            del Q, sc
    for form in ("bf16", "e4m3"):
        forms[form]["speedup_vs_fp32"] = round(forms[form]["solves_per_s"] / forms["fp32"]["solves_per_s"], 3)
    out["forms"] = forms
    del A
    torch.cuda.empty_cache()
    return out


# --------------------------------------------------------- batched leg --

BATCH_COUNT = 4096
BATCH_WORKLOAD = ("4096 independent FP32 GEMVs c += A x, m and n log-uniform in [32, 8192] "
                  "(synth.log_uniform_integers, seed 0), row-major with lda = n rounded up to a "
                  "multiple of 4, A, x, c uniform[-1,1]")


class BatchWorkload:
    """The batched-GEMV workload resident on the device: one arena each for
    the A's, x's and c's, every operand 256-byte aligned."""

    def __init__(self, device, count=BATCH_COUNT, seed=0, lo=32, hi=8192):
        import numpy as np
        import torch
        import synth
        self.m = synth.log_uniform_integers(count, seed, 301, lo, hi)
        self.n = synth.log_uniform_integers(count, seed, 302, lo, hi)
        self.lda = (self.n + 3) // 4 * 4

        def offsets(sizes):
            padded = (sizes + 63) // 64 * 64          # 256-byte aligned starts
            off = np.concatenate([[0], np.cumsum(padded)[:-1]]).astype(np.int64)
            return off, int(padded.sum())

        self.a_off, na = offsets(self.m * self.lda)
        self.x_off, nx = offsets(self.n)
        self.c_off, nc = offsets(self.m)
        self.A = torch.empty(max(na, 1), dtype=torch.float32, device=device)
        self.x = torch.empty(max(nx, 1), dtype=torch.float32, device=device)
        self.c = torch.empty(max(nc, 1), dtype=torch.float32, device=device)
        synth.fill_uniform(self.A, seed, 303)
        synth.fill_uniform(self.x, seed, 304)
        synth.fill_uniform(self.c, seed, 305)
        a0, x0, c0 = self.A.data_ptr(), self.x.data_ptr(), self.c.data_ptr()
        self.problems = [(a0 + 4 * int(self.a_off[p]), x0 + 4 * int(self.x_off[p]),
                          c0 + 4 * int(self.c_off[p]), 1.0, int(self.m[p]), int(self.n[p]),
                          int(self.lda[p])) for p in range(count)]
        self.bytes = int((4 * (self.m * self.n + self.n + 2 * self.m)).sum())
        torch.cuda.synchronize(device)

    def operands(self, p):
        """(A as an m x lda view, x, c) of problem p."""
        m, n, ld = int(self.m[p]), int(self.n[p]), int(self.lda[p])
        a = self.A[self.a_off[p]:self.a_off[p] + m * ld].view(m, ld)
        return a, self.x[self.x_off[p]:self.x_off[p] + n], self.c[self.c_off[p]:self.c_off[p] + m]


LEAD_CYCLES = 1_000_000   # ~0.5 ms of GPU spin ahead of each timed region


def gpu_lead(stream):
    """Keep the GPU busy (a bounded spin kernel) while the host issues the
    calls that a timed region starts with: otherwise the start event is
    taken on an idle GPU, and the host's time to issue the first call (tens
    of microseconds through ctypes) is counted as GPU time."""
    import torch
    with torch.cuda.stream(stream):
        torch.cuda._sleep(LEAD_CYCLES)


def _time_events(fn, stream, reps):
    import torch
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        gpu_lead(stream)
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1) / 1e3)
    return statistics.median(times)


def run_batched(device, stream, hbm, reps=5):
    """The 4096 GEMVs as 4096 separate plain launches (gb_sgemv; host loop,
    then the same calls captured in one CUDA graph) and as one persistent
    batched launch (gb_sgemv_batch; direct, then replayed from a graph),
    each timed with CUDA events on the launching stream (median of `reps`;
    35 GB of operands, far above L2)."""
    import torch
    import paper_2108_02025_gb300 as gb
    wl = BatchWorkload(device)
    lib = gb.lib()
    sh = stream.cuda_stream
    nb = max(gb.gb_workspace_bytes(gb.OP_GEMV, gb.F32, gb.ROW_MAJOR, m, n) for
             (_, _, _, _, m, n, _) in wl.problems)
    ws = torch.zeros(max(nb, 1), dtype=torch.uint8, device=device)
    wsp = ws.data_ptr()
    f = lib.gb_sgemv

    def separate(st):
        for (a, x, c, al, m, n, ld) in wl.problems:
            if f(0, m, n, al, a, ld, x, c, wsp, nb, st) != 0:
                raise RuntimeError("gb_sgemv failed")

    table = gb.load_tuning()
    batch = gb.Batch(wl.problems, table=table, device=device)

    def batched(st):
        batch.launch(st)

    out = {"workload": BATCH_WORKLOAD, "problems": len(wl.problems), "bytes": wl.bytes,
           "tiles": batch.tiles,
           "tuning": "autotuned table" if os.path.exists(gb.TUNING_PATH) else "built-in table"}
    cap = torch.cuda.Stream(device)  # graphs are captured on a side stream
    for name, fn in (("separate", separate), ("batched", batched)):
        fn(sh)
        torch.cuda.synchronize(device)
        t = _time_events(lambda: fn(sh), stream, reps)
        g = torch.cuda.CUDAGraph()
        cap.wait_stream(stream)
        with torch.cuda.graph(g, stream=cap):
            fn(cap.cuda_stream)
        stream.wait_stream(cap)
        g.replay()
        torch.cuda.synchronize(device)
        tg = _time_events(g.replay, stream, reps)
        del g
        for key, tt in ((name, t), (name + "_graph", tg)):
            out[key] = {"ms": round(tt * 1e3, 3), "GB_s": round(wl.bytes / tt / 1e9, 1),
                        "frac_hbm": round(wl.bytes / tt / 1e9 / hbm, 4),
                        "solves_per_s": round(len(wl.problems) / tt, 1),
                        "launches": 1 if name == "batched" else len(wl.problems)}
    out["speedup_vs_separate"] = round(out["separate"]["ms"] / out["batched_graph"]["ms"], 3)
    del batch, ws
    out["bf16"] = batched_bf16(wl, device, stream, hbm, table, reps, out["batched_graph"]["ms"])
    del wl
    torch.cuda.empty_cache()
    return out


# --------------------------------------------------------- serving leg --

SERVE_WORKLOAD = ("Poisson request stream, 70% GEMV / 20% DOT / 10% GER, m and n log-uniform in "
                  "[32, 16384], alpha 1, operands resident on the device (pools of 2^30 FP32 and "
                  "2^30 BF16 values from the counter-based generator, filled once), each request's "
                  "output allocated under a 64 GB HBM admission budget, 4 streams, GEMVs and GERs "
                  "above 256 MB launched in row chunks of about 256 MB; for comparison the same "
                  "stream with every operand drawn on the device per request")
SERVE_BUDGET = 64 << 30
SERVE_POOL = 1 << 30
SERVE_POOL_SEED = 2108
SERVE_CHUNK = 256 << 20   # pool GEMVs / GERs above this many bytes run in row chunks of about this size


def serve_stream(count, rate, seed, lo=32, hi=16384):
    """Arrival offsets (ns), ops, m, n of a seeded Poisson stream."""
    import numpy as np
    import synth
    u = (synth.uniform(count, seed, 501) + 1.0) / 2.0
    t = np.cumsum(-np.log1p(-u) / rate * 1e9).astype(np.int64)
    pick = (synth.uniform(count, seed, 502) + 1.0) / 2.0
    ops = np.where(pick < 0.7, 0, np.where(pick < 0.9, 1, 2))
    m = synth.log_uniform_integers(count, seed, 503, lo, hi)
    n = synth.log_uniform_integers(count, seed, 504, lo, hi)
    return t, ops, m, n


def serve_once(count, rate, form, seed=0, sample=8, pool=True, budget=SERVE_BUDGET, pool_elems=SERVE_POOL,
               chunk_bytes=SERVE_CHUNK):
    """Serve one stream (operands from the resident pools, or drawn per
    request); returns throughput, latency percentiles and the measured error
    of `sample` GEMV results (numpy FP64 on the generator's FP32 values,
    relative to sum_j |A_ij x_j| + |c0_i|)."""
    import numpy as np
    import torch
    import synth
    import paper_2108_02025_gb300 as gb
    t, ops, m, n = serve_stream(count, rate, seed)
    gemv_idx = [i for i in range(count) if ops[i] == 0 and m[i] * n[i] <= 1 << 22]
    picks = set(gemv_idx[::max(1, len(gemv_idx) // sample)][:sample]) if sample > 0 else set()
    outs = {}
    with gb.Engine(budget, streams=4, max_inflight=16384, max_step_requests=512,
                   table=gb.load_tuning(), pool_elems=pool_elems if pool else 0,
                   pool_seed=SERVE_POOL_SEED, chunk_bytes=chunk_bytes) as e:
        t0 = e.now_ns() + int(0.2e9) + count * 20000   # every request is queued before the first arrives
        for i in range(count):
            out = None
            if i in picks:
                out = torch.empty(int(m[i]), dtype=torch.float32, pin_memory=True)
                outs[i] = out
            fi = form if ops[i] == 0 else gb.FORM_F32
            st = e.submit(i, int(ops[i]), int(m[i]), int(n[i]), 1.0, seed * 1000003 + i, out,
                          arrival_ns=int(t0 + t[i]), form=fi, pool=pool)
            if st != gb.GB_OK:
                raise RuntimeError(f"submit {i}: {st}")
        if e.drain(600000) != gb.GB_OK:
            raise RuntimeError("serving stream did not drain")
        done = e.poll(count)
        stats = e.stats()
    bad = [c for c in done if c["status"] != gb.GB_OK]
    if bad or len(done) != count:
        raise RuntimeError(f"{len(bad)} failed requests, {len(done)} of {count} completed")
    arr = np.array([c["arrival_ns"] for c in done], np.float64)
    fin = np.array([c["done_ns"] for c in done], np.float64)
    lat = (fin - arr) / 1e3
    span = (fin.max() - arr.min()) / 1e9
    steps = np.bincount([c["step"] for c in done])
    err = 0.0
    for i, out in outs.items():
        mi, ni = int(m[i]), int(n[i])
        ld = (ni + 7) // 8 * 8 if form == gb.FORM_BF16 else (ni + 3) // 4 * 4
        s0 = seed * 1000003 + i
        if pool:    # windows of the pools; the BF16 pool rounds stream 2 of the pool seed
            def win(s, L, stream):
                o = synth.pool_offset(s0, s, L, pool_elems)
                return synth.uniform_pairs(L, SERVE_POOL_SEED, stream, offset=o)
            A = win(1, mi * ld, 2 if form == gb.FORM_BF16 else 1)
            x, c0 = win(2, ni, 1), win(3, mi, 1)
        else:
            A = synth.uniform_pairs(mi * ld, s0, 1)
            x, c0 = synth.uniform_pairs(ni, s0, 2), synth.uniform_pairs(mi, s0, 3)
        A = A.reshape(mi, ld)[:, :ni].astype(np.float64)
        x, c0 = x.astype(np.float64), c0.astype(np.float64)
        want = c0 + A @ x
        scale = np.abs(c0) + np.abs(A) @ np.abs(x)
        err = max(err, float(np.max(np.abs(out.numpy().astype(np.float64) - want) / scale)))
    fp_bytes = np.where(ops == 0, (2 if form == gb.FORM_BF16 else 4) * m * n + 4 * n + 8 * m,
                        np.where(ops == 1, 8 * n + 8, 8 * m * n + 4 * m + 4 * n)).sum()
    return {"requests": count, "offered_per_s": rate, "solves_per_s": round(count / span, 1),
            "p50_us": round(float(np.percentile(lat, 50)), 1),
            "p99_us": round(float(np.percentile(lat, 99)), 1),
            "compute_GB_s": round(float(fp_bytes) / span / 1e9, 1),
            "steps": int(stats["steps"]), "mean_step_requests": round(float(steps.mean()), 1),
            "steps_inflight_peak": int(stats["steps_inflight_peak"]),
            "bytes_peak_GB": round(stats["bytes_peak"] / 1e9, 2),
            "gemv_max_rel_err": float(f"{err:.3e}"), "gemv_err_sampled": len(outs)}


SERVE_LOADS = (0.5, 0.8, 0.95)


def serve_loads(count, form, seed=1, chunk_bytes=SERVE_CHUNK, pool=True):
    """One stream at saturation, then the same requests (same sizes, same
    order) arriving at 50%, 80% and 95% of the measured rate."""
    sat = serve_once(count, 1e7, form, seed=seed, chunk_bytes=chunk_bytes, pool=pool)
    loads = {str(f): serve_once(count, sat["solves_per_s"] * f, form, seed=seed, chunk_bytes=chunk_bytes, pool=pool)
             for f in SERVE_LOADS}
    return {"saturated": sat, "loads": loads}


def run_serving(count=20000):
    """Saturating streams (throughput) for FP32 and BF16-stored A, then the
    same streams at 50%, 80% and 95% of their measured throughput (latency
    under load)."""
    import paper_2108_02025_gb300 as gb
    out = {"workload": SERVE_WORKLOAD, "budget_bytes": SERVE_BUDGET,
           "error_bound": {"fp32": "1e-5 of sum|A x| + |c0| (FP32 accumulation)",
                           "bf16": "2^-9 of sum|A x| + |c0| (BF16 rounding of A) + FP32 accumulation"}}
    out["chunk_bytes"] = SERVE_CHUNK
    for name, form in (("fp32", gb.FORM_F32), ("bf16", gb.FORM_BF16)):
        out[name] = serve_loads(count, form)
    out["bf16_speedup_solves"] = round(out["bf16"]["saturated"]["solves_per_s"] /
                                       out["fp32"]["saturated"]["solves_per_s"], 3)
    out["drawn_operands"] = {name: serve_once(count, 1e7, form, seed=1, pool=False, chunk_bytes=0)
                             for name, form in (("fp32", gb.FORM_F32), ("bf16", gb.FORM_BF16))}
    return out


def batched_bf16(wl, device, stream, hbm, table, reps, fp32_ms, sample=6):
    """The same 4096 GEMVs with every A stored as BF16 (rows padded to 8
    elements), one batched launch from a CUDA graph; error of sampled
    problems against numpy FP64 on the FP32 master, relative to
    sum_j |A_ij x_j| + |c0_i|."""
    import numpy as np
    import torch
    import paper_2108_02025_gb300 as gb
    ldq = (wl.n + 7) // 8 * 8
    padded = (wl.m * ldq + 127) // 128 * 128          # 256-byte aligned starts
    q_off = np.concatenate([[0], np.cumsum(padded)[:-1]]).astype(np.int64)
    Q = torch.empty(int(padded.sum()), dtype=torch.int16, device=device)
    for p in range(len(wl.problems)):
        a, _, _ = wl.operands(p)
        st = gb.gb_quantize_bf16(int(wl.m[p]), int(wl.n[p]), a, int(wl.lda[p]),
                                 Q[int(q_off[p]):].data_ptr(), int(ldq[p]), stream)
        if st != 0:
            raise RuntimeError(f"quantize {p}: {st}")
    picks = [int(i) for i in np.linspace(0, len(wl.problems) - 1, sample).round()]
    c0 = {p: wl.operands(p)[2].clone() for p in picks}
    items = [(gb.BATCH_GEMV_BF16, Q.data_ptr() + 2 * int(q_off[p]), xp, cp, al, mi, ni, int(ldq[p]))
             for p, (_, xp, cp, al, mi, ni, _) in enumerate(wl.problems)]
    batch = gb.Batch.from_items(items, table=table, device=device)
    for p in picks:  # errors after one launch from the original c
        wl.operands(p)[2].copy_(c0[p])
    batch.launch(stream.cuda_stream)
    torch.cuda.synchronize(device)
    err = 0.0
    for p in picks:
        a, x, c = wl.operands(p)
        n = int(wl.n[p])
        A = a[:, :n].double().cpu().numpy()
        xx = x.double().cpu().numpy()
        cc = c0[p].double().cpu().numpy()
        want = cc + A @ xx
        scale = np.abs(cc) + np.abs(A) @ np.abs(xx)
        err = max(err, float(np.max(np.abs(c.double().cpu().numpy() - want) / scale)))
    cap = torch.cuda.Stream(device)
    g = torch.cuda.CUDAGraph()
    cap.wait_stream(stream)
    with torch.cuda.graph(g, stream=cap):
        batch.launch(cap.cuda_stream)
    stream.wait_stream(cap)
    g.replay()
    torch.cuda.synchronize(device)
    t = _time_events(g.replay, stream, reps)
    nbytes = int((2 * wl.m * wl.n + 4 * wl.n + 8 * wl.m).sum())
    del g, batch, Q
    torch.cuda.empty_cache()
    return {"ms": round(t * 1e3, 3), "GB_s": round(nbytes / t / 1e9, 1), "bytes": nbytes,
            "frac_hbm": round(nbytes / t / 1e9 / hbm, 4), "solves_per_s": round(len(wl.problems) / t, 1),
            "speedup_vs_fp32_batched": round(fp32_ms / (t * 1e3), 3),
            "max_rel_err": float(f"{err:.3e}"), "bound": 2.0 ** -9, "sampled_problems": len(picks)}


# ------------------------------------------------------------------- arms --

def run_ours(args):
    import torch
    world, rank = init_dist("nccl")
    _, _, local = dist_info()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    wl = Workload(device)
    stream = torch.cuda.current_stream(device)
    sh = stream.cuda_stream
    ops = wl.ops

    # the operations moving the most bytes (the FP64 DOT and GERs) carry an
    # event pair inside the timed steps: the roofline kernel is timed live
    top = max(alg_bytes(k, dt, m, n) for (_, k, dt, _, m, n) in ops)
    live = [i for i, (_, k, dt, _, m, n) in enumerate(ops) if alg_bytes(k, dt, m, n) == top]

    def step(evs=None):
        for i, op in enumerate(ops):
            if evs is not None and i in evs:
                evs[i][0].record(stream)
            wl.launch(op, sh)
            if evs is not None and i in evs:
                evs[i][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(device)

    clocks = ClockSampler(local)
    clocks.start()
    for _ in range(2):  # keep the GPU busy while the sampler comes up
        step()
    live_ev = [{i: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for i in live}
               for _ in range(args.steps)]
    t_begin = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(device)
    barrier()
    wall0 = time.time()
    gpu_lead(stream)
    t_begin.record(stream)
    for k in range(args.steps):
        step(live_ev[k])
    t_end.record(stream)
    torch.cuda.synchronize(device)
    barrier()
    wall1 = time.time()
    elapsed = t_begin.elapsed_time(t_end) / 1e3
    elapsed_max = max_over_ranks(elapsed, device)

    # Per operation, after the timed steps: OP_CALLS calls back to back
    # between two events, OP_REPS times.  (An event pair around every call
    # would start each kernel from an idle stream and charge it a launch.)
    per_op = []
    for op in ops:
        wl.launch(op, sh)
        each = []
        for _ in range(OP_REPS):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            gpu_lead(stream)
            e0.record(stream)
            for _ in range(OP_CALLS):
                wl.launch(op, sh)
            e1.record(stream)
            e1.synchronize()
            each.append(e0.elapsed_time(e1) / 1e3 / OP_CALLS)
        per_op.append(sorted(each))
    # The same OP_CALLS calls replayed from one CUDA graph: no host launch
    # between the kernels, so the time per call is the device's alone
    per_op_graph = []
    cap = torch.cuda.Stream(device)
    for op in ops:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            for _ in range(OP_CALLS):
                wl.launch(op, cap.cuda_stream)
        g.replay()
        each = []
        for _ in range(OP_REPS):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            gpu_lead(stream)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            e1.synchronize()
            each.append(e0.elapsed_time(e1) / 1e3 / OP_CALLS)
        per_op_graph.append(statistics.mean(each))
        del g
    clocks.stop()

    bytes_step = sum(alg_bytes(k, dt, m, n) for (_, k, dt, _, m, n) in ops)
    value = whole_job_value(bytes_step, args.steps, world, elapsed_max)
    op_times = [statistics.mean(e) for e in per_op]
    live_times = {i: statistics.mean(live_ev[k][i][0].elapsed_time(live_ev[k][i][1]) / 1e3
                                     for k in range(args.steps)) for i in live}
    hbm, src = peaks()
    dom = max(live, key=lambda i: live_times[i])   # the largest time share of the step
    ops_report = []
    for i, (name, kind, dt, lay, m, n) in enumerate(ops):
        gbs = alg_bytes(kind, dt, m, n) / op_times[i] / 1e9
        each = per_op[i]
        ops_report.append({"op": name, "us": round(op_times[i] * 1e6, 2),
                           "us_median": round(each[len(each) // 2] * 1e6, 2), "us_min": round(each[0] * 1e6, 2),
                           "GB_s": round(gbs, 1), "frac_hbm": round(gbs / hbm, 4),
                           "frac_nominal": round(gbs / NOMINAL_HBM_GBS, 4),
                           "us_graph": round(per_op_graph[i] * 1e6, 2),
                           "frac_hbm_graph": round(alg_bytes(kind, dt, m, n) / per_op_graph[i] / 1e9 / hbm, 4)})

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(wl, stream, device, bytes_step, args, world)

    precision = batched = serving = None
    if not args.no_growth:
        precision = run_precision(device, stream)
        batched = run_batched(device, stream, hbm)
        serving = run_serving()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        work = oracle_sample(CPU_FRACTION)
        secs, sb = 0.0, 0
        while secs < 10.0:          # repeat the sample until ~10 s of oracle time
            t, b = time_sample(work)
            secs, sb = secs + t, sb + b
        extra = {}
        for name, frac, threads, acc in (("single_thread", CPU_FRACTION * 16, 1, False),
                                         ("acc", CPU_FRACTION * 4, oracle.threads(), True)):
            w2 = oracle_sample(frac, acc=acc)
            keep = oracle.threads()
            oracle.set_threads(threads)
            try:
                t2, b2 = 0.0, 0
                while t2 < 3.0:
                    t, b = time_sample(w2)
                    t2, b2 = t2 + t, b2 + b
            finally:
                oracle.set_threads(keep)
            extra[name] = {"value": round(b2 / t2 / 1e9, 3), "cores": threads,
                           "sample": f"1/{frac} of a step, {b2 / 1e9:.2f} GB in {t2:.1f} s"}
        cpu = {"value": round(sb / secs / 1e9, 3), "unit": "GB/s", "cores": oracle.threads(),
               "kind": "oracle", "single_thread": extra["single_thread"],
               "acc_oracle": extra["acc"],
               "sample": f"1/{CPU_FRACTION} of the rows (row-major) or columns (column-major) of "
                         f"every GEMV/GER and of the DOT vectors of one step (DOT single-threaded), "
                         f"plain FP64 oracle, repeated: {sb / 1e9:.2f} GB in {secs:.1f} s; "
                         f"{os.cpu_count()} host cores"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(elapsed_max / args.steps * 1e3, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (each large operand >= 268 MB, L2 129 MB)",
                       "bytes_per_step": bytes_step},
            "roofline": dict(roofline_of(ops[dom], live_times[dom], hbm, src),
                             timing="CUDA events around each launch inside the timed steps"),
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": len(ops) * args.steps,
            "clocks": clocks.summary(wall0, wall1),
            "precision": precision,
            "batched": batched,
            "serving": serving,
            # the per-operation table last, so that a reader of the end of
            # the output sees it whole
            "ops_timing": f"after the timed steps, each operation {OP_CALLS} times back to back between two "
                          f"CUDA events, {OP_REPS} such pairs; us = mean per call issued from the host, "
                          f"us_graph = the same calls replayed from one CUDA graph (no host launch between "
                          f"the kernels)",
            "ops": ops_report,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def measure_link(device, nbytes=1 << 30, reps=3):
    """GB/s of this machine's host link as the e2e leg uses it: a copy-engine
    upload from pinned memory, a gb_copy_to_host download, and both at once
    on two streams (best of `reps`)."""
    import torch
    import paper_2108_02025_gb300 as gb
    h_in = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    h_out = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    d_in = torch.empty(nbytes, dtype=torch.uint8, device=device)
    d_out = torch.zeros(nbytes, dtype=torch.uint8, device=device)
    s1, s2 = torch.cuda.Stream(device), torch.cuda.Stream(device)

    def up():
        with torch.cuda.stream(s1):
            d_in.copy_(h_in, non_blocking=True)

    def down():
        if gb.gb_copy_to_host(h_out, d_out, nbytes, s2) != gb.GB_OK:
            raise RuntimeError("gb_copy_to_host failed")

    def best(fns, moved):
        t = []
        for _ in range(reps + 1):
            torch.cuda.synchronize(device)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s1)
            s2.wait_event(e0)
            for f in fns:
                f()
            s1.wait_stream(s2)
            e1.record(s1)
            torch.cuda.synchronize(device)
            t.append(e0.elapsed_time(e1) / 1e3)
        return moved / min(t[1:]) / 1e9

    out = {"h2d_GB_s": round(best([up], nbytes), 1), "d2h_GB_s": round(best([down], nbytes), 1),
           "both_GB_s": round(best([up, down], 2 * nbytes), 1)}
    del h_in, h_out, d_in, d_out
    return out


def link_bound(bytes_step, h2d, d2h, link):
    """GB/s of algorithmic bytes that a step moving h2d bytes up and d2h
    bytes down cannot beat: its time is at least the upload alone, the
    download alone, and both at the rate the link reaches both ways."""
    t_min = max(h2d / (link["h2d_GB_s"] * 1e9), d2h / (link["d2h_GB_s"] * 1e9),
                (h2d + d2h) / (link["both_GB_s"] * 1e9))
    return bytes_step / t_min / 1e9


def run_e2e(wl, stream, device, bytes_step, args, world):
    """The same step through host buffers: every step copies all its inputs
    from pinned host memory to the device (copy engine), runs the 18 calls
    and copies the results (c, alpha, C) back with gb_copy_to_host (a kernel
    storing into the pinned buffers, so the download never waits behind an
    upload on a shared copy engine).  Two device sets of buffers let step
    k+1's upload overlap step k's calls and download; a set is reused only
    after its download is done."""
    import torch
    import paper_2108_02025_gb300 as gb
    wls = [wl, Workload(device)]
    host_in = [torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in wl.inputs()]
    for h, d in zip(host_in, wl.inputs()):
        h.copy_(d)
    host_out = [[torch.empty(t.shape, dtype=t.dtype, pin_memory=True) for t in w.results()] for w in wls]
    h2d = sum(t.numel() * t.element_size() for t in host_in)
    d2h = sum(t.numel() * t.element_size() for t in host_out[0])
    s_in, s_out = torch.cuda.Stream(device), torch.cuda.Stream(device)
    ev = [{k: torch.cuda.Event() for k in ("in", "comp", "out")} for _ in wls]
    for e in ev:
        e["out"].record(s_out)
    steps = max(1, min(args.steps, args.e2e_steps))

    def step(k):
        b = k % 2
        w, e = wls[b], ev[b]
        s_in.wait_event(e["out"])           # the set's previous download is done
        with torch.cuda.stream(s_in):
            for h, d in zip(host_in, w.inputs()):
                d.copy_(h, non_blocking=True)
        e["in"].record(s_in)
        stream.wait_event(e["in"])
        for op in w.ops:
            w.launch(op, stream.cuda_stream)
        e["comp"].record(stream)
        s_out.wait_event(e["comp"])
        for h, d in zip(host_out[b], w.results()):   # a kernel copy: no copy engine
            st = gb.gb_copy_to_host(h, d, d.numel() * d.element_size(), s_out)
            if st != gb.GB_OK:
                raise RuntimeError(f"gb_copy_to_host: {gb.gb_status_string(st)}")
        e["out"].record(s_out)

    step(0)
    step(1)
    torch.cuda.synchronize(device)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    for k in range(steps):
        step(k)
    s_out.wait_stream(stream)
    s_out.wait_stream(s_in)
    e1.record(s_out)
    torch.cuda.synchronize(device)
    barrier()
    secs = max_over_ranks(e0.elapsed_time(e1) / 1e3, device)
    del wls[1]
    torch.cuda.empty_cache()
    link = measure_link(device)
    value = whole_job_value(bytes_step, steps, world, secs)
    link["bound_GB_s"] = round(link_bound(bytes_step, h2d, d2h, link), 1)
    link["frac"] = round(value / world / link["bound_GB_s"], 3)
    return {"value": round(value, 1), "unit": "GB/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "ms_per_step": round(secs / steps * 1e3, 3), "link": link,
            "note": "two device buffer sets: uploads (copy engine), calls and downloads (gb_copy_to_host "
                    "kernel) of consecutive steps overlap"}


def run_reference(args):
    """The oracle (plain FP64 CPU definitions) on the host cores, timed on a
    bounded sample (1/REF_FRACTION) of the same step, on rank 0 only."""
    world, rank, _ = dist_info()
    if rank != 0:
        return
    import oracle
    work = oracle_sample(REF_FRACTION)
    for _ in range(args.warmup):
        time_sample(work)
    total_b, total_t = 0, 0.0
    for _ in range(args.steps):
        secs, sb = time_sample(work)
        total_b += sb
        total_t += secs
    threads = oracle.threads()
    value = total_b / total_t / 1e9
    sample = (f"each step: 1/{REF_FRACTION} of the rows (row-major) or columns (column-major) of every "
              f"GEMV/GER and of the DOT vectors of one GPU step (DOT single-threaded), plain FP64 oracle, "
              f"{total_b / args.steps / 1e9:.3f} GB per step")
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "impl": "reference",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_t / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": "host cores"},
        "cpu_baseline": {"value": round(value, 3), "unit": "GB/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------- one-case mode --

def fit_fixed_cost(points):
    """Least-squares fit of t = t0 + bytes / bw over (bytes, seconds) points:
    returns (t0 in seconds, bw in bytes per second)."""
    k = len(points)
    sx = sum(b for b, _ in points)
    sy = sum(t for _, t in points)
    sxx = sum(b * b for b, _ in points)
    sxy = sum(b * t for b, t in points)
    den = k * sxx - sx * sx
    if k < 2 or den == 0:
        return None, None
    slope = (k * sxy - sx * sy) / den
    t0 = (sy - slope * sx) / k
    return t0, (1.0 / slope if slope > 0 else None)


def case_bytes(op, dtype, m, n):
    """Compulsory bytes of one call of a --case operation."""
    if op in ("gemv", "dot", "ger"):
        return alg_bytes(op, dtype, m, n)
    return precision_bytes(dtype, m, n)


def run_case(args):
    """One operation of the library timed on its own (--case OP DTYPE LAYOUT
    M N): inputs uniform[-1,1] from the generator (gemvq: the precision
    workload's A, quantised before timing; quant: the quantiser of DTYPE on
    that A; batch: M GEMVs of the batched workload in one launch with the
    tuned table).  Each rep is --batch calls
    back to back between two CUDA events on the launching stream (the
    events' resolution is about 2 us), after an L2 flush by a read of 512
    MB; the calls take copies of the operands in turn (at least 600 MB
    together), so that none finds its operands in L2.  With
    --scale k1,k2,... the long dimension (the larger of M and N; n for DOT)
    is multiplied by each factor in turn and t = t0 + bytes/bw is fitted
    over the median times, which separates a fixed cost per call from the
    streaming bandwidth.  host_us_per_call is the host's time to issue one
    call; with --graph the rep's calls are replayed from one CUDA graph
    instead, so that no host time can show between the kernels."""
    import torch
    import paper_2108_02025_gb300 as gb
    import synth
    op, dtype, layout, m0, n0 = args.case
    m0, n0 = int(m0), int(n0)
    device = torch.device("cuda", torch.cuda.current_device())
    if args.graph:  # graphs are captured on a stream other than the default one
        torch.cuda.set_stream(torch.cuda.Stream(device))
    stream = torch.cuda.current_stream(device)
    # L2 flush by reading a buffer of 4x the L2: a write would leave dirty
    # lines whose write-back overlaps the timed call
    flush = torch.ones(128 << 20, dtype=torch.float32, device=device)
    lay = gb.COL_MAJOR if layout == "col" else gb.ROW_MAJOR
    hbm, src = peaks()
    scales = [int(s) for s in args.scale.split(",")] if args.scale else [1]
    rows = []
    for k in scales:
        m, n = (m0 * k, n0) if (m0 > n0 and op != "dot") or op == "batch" else (m0, n0 * k)
        tdt = torch.float64 if dtype == "f64" else torch.float32

        def filled(numel, s):
            t = torch.empty(max(numel, 1), dtype=tdt, device=device)
            synth.fill_uniform(t, 0, s)
            return t

        nb = case_bytes(op, dtype, m, n) if op not in ("batch", "quant") else quantize_bytes(dtype, m, n) \
            if op == "quant" else None
        # copies of the operands, used in turn, so that no call finds its
        # operands in L2 (together at least 4.5x the L2)
        copies = 1 if op == "batch" else max(1, min(8, -(-(600 << 20) // nb)))
        calls = []
        for r in range(copies):
            if op == "gemv":
                A, x, c = filled(m * n, 1 + 10 * r), filled(n, 2 + 10 * r), filled(m, 3 + 10 * r)
                ld = n if lay == gb.ROW_MAJOR else m
                calls.append(lambda A=A, x=x, c=c, ld=ld: gb.gemv(A, x, c, 1.0, lay, m, n, ld))
            elif op == "dot":
                x, y, a = filled(n, 4 + 10 * r), filled(n, 5 + 10 * r), filled(1, 6 + 10 * r)
                calls.append(lambda x=x, y=y, a=a: gb.dot(x, y, a, n))
            elif op == "ger":
                C, x, y = filled(m * n, 7 + 10 * r), filled(m, 8 + 10 * r), filled(n, 9 + 10 * r)
                ld = n if lay == gb.ROW_MAJOR else m
                calls.append(lambda C=C, x=x, y=y, ld=ld: gb.ger(x, y, C, 1.0, lay, m, n, ld))
            elif op == "quant":  # the quantiser of DTYPE (bf16 or e4m3) on the precision workload's A
                A = torch.empty((m, n), dtype=torch.float32, device=device)
                synth.fill_normal_rows(A, 0, 1 + 10 * r, -3.0, 3.0)
                Q, sc = gb.quantize(A, dtype)
                nb = quantize_bytes(dtype, m, n)
                if dtype == "bf16":
                    calls.append(lambda A=A, Q=Q: gb.lib().gb_quantize_bf16(m, n, A.data_ptr(), n, Q.data_ptr(),
                                                                            Q.stride(0), stream.cuda_stream))
                else:
                    calls.append(lambda A=A, Q=Q, sc=sc: gb.lib().gb_quantize_e4m3(
                        m, n, A.data_ptr(), n, Q.data_ptr(), Q.stride(0), sc.data_ptr(), stream.cuda_stream))
            elif op == "batch":  # M FP32 GEMVs of the batched workload in one launch; N unused
                bw_ = BatchWorkload(device, count=m)
                b = gb.Batch(bw_.problems, table=gb.load_tuning())
                nb = bw_.bytes
                calls.append(lambda b=b: b.launch())
            else:  # gemvq: dtype bf16 or e4m3
                A = torch.empty((m, n), dtype=torch.float32, device=device)
                synth.fill_normal_rows(A, 0, 1, -3.0, 3.0)
                x, c = filled(n, 2 + 10 * r), filled(m, 3 + 10 * r)
                Q, sc = gb.quantize(A, dtype)
                del A
                calls.append(lambda Q=Q, sc=sc, x=x, c=c: gb.gemv_q(Q, sc, x, c, 1.0, n=n))
        for i in range(3 * copies):
            calls[i % copies]()
        torch.cuda.synchronize(device)
        graph = None
        if args.graph:  # the rep's calls captured once, on this stream's workspace
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                for i in range(args.batch):
                    calls[i % copies]()
            graph.replay()
            torch.cuda.synchronize(device)
        times, host = [], []
        for _ in range(args.reps):
            flush.sum()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            gpu_lead(stream)
            e0.record(stream)
            h0 = time.perf_counter()
            if graph is not None:
                graph.replay()
            else:
                for i in range(args.batch):
                    calls[i % copies]()
            host.append((time.perf_counter() - h0) / args.batch)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1) / 1e3 / args.batch)
        times.sort()
        med = times[len(times) // 2]
        rows.append({"scale": k, "m": m, "n": n, "bytes": nb, "copies": copies,
                     "us_median": round(med * 1e6, 2), "us_min": round(times[0] * 1e6, 2),
                     "host_us_per_call": round(statistics.median(host) * 1e6, 2),
                     "GB_s": round(nb / med / 1e9, 1), "frac_hbm": round(nb / med / 1e9 / hbm, 4)})
        del graph
        del calls
        torch.cuda.empty_cache()
    out = {"case": [op, dtype, layout, m0, n0], "reps": args.reps, "calls_per_rep": args.batch,
           "issue": "one CUDA graph of the rep's calls" if args.graph else "calls issued from the host",
           "l2": "flushed (512 MB read) before each rep; the calls of a rep take the operand copies in turn",
           "peak_gbs": hbm, "peak_source": src, "points": rows}
    if len(rows) >= 2:
        t0, bw = fit_fixed_cost([(r["bytes"], r["us_median"] * 1e-6) for r in rows])
        out["fit"] = {"t0_us": round(t0 * 1e6, 2) if t0 is not None else None,
                      "bw_GB_s": round(bw / 1e9, 1) if bw else None,
                      "bw_frac_hbm": round(bw / 1e9 / hbm, 4) if bw else None}
    print(json.dumps(out), flush=True)


def run_serve_case(args):
    """One seeded Poisson stream through the serving engine alone (--serve):
    the serving workload (70% GEMV / 20% DOT / 10% GER, m and n log-uniform
    in [32, 16384], 4 streams) on resident operand pools of
    2^pool_log2 FP32 and BF16 values (or every operand drawn per request,
    --serve-drawn), under an HBM budget of --serve-budget-gb GB.  With the
    default rate every request arrives at once, which measures capacity; with
    --serve-loads the stream is served at saturation and then, the same
    requests, at 50%, 80% and 95% of the measured rate.  A small budget and
    pool keep the device footprint small enough for a profiler capture."""
    import paper_2108_02025_gb300 as gb
    form = gb.FORM_BF16 if args.serve_bf16 else gb.FORM_F32
    chunk = SERVE_CHUNK if args.serve_chunk_mb is None else int(args.serve_chunk_mb * (1 << 20))
    if args.serve_loads:
        r = serve_loads(args.serve, form, seed=args.serve_seed, chunk_bytes=chunk, pool=not args.serve_drawn)
        r = {"chunk_bytes": chunk, "saturated": r["saturated"]["solves_per_s"],
             "loads": {f: (v["solves_per_s"], v["p50_us"], v["p99_us"]) for f, v in r["loads"].items()}}
    else:
        r = serve_once(args.serve, args.serve_rate, form, seed=args.serve_seed, sample=0,
                       pool=not args.serve_drawn, budget=int(args.serve_budget_gb * (1 << 30)),
                       pool_elems=1 << args.serve_pool_log2, chunk_bytes=chunk)
    print(json.dumps(r), flush=True)


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--e2e-steps", type=int, default=16, help="steps of the host-buffer (e2e) leg")
    p.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline leg")
    p.add_argument("--no-growth", action="store_true",
                   help="skip the reduced-precision, batched and serving legs")
    p.add_argument("--case", nargs=5, metavar=("OP", "DTYPE", "LAYOUT", "M", "N"),
                   help="time one operation alone: OP gemv|dot|ger|gemvq|batch|quant, DTYPE f32|f64|bf16|e4m3, "
                        "LAYOUT row|col|-; for batch, M is the number of GEMVs")
    p.add_argument("--scale", default=None,
                   help="with --case: factors of the long dimension, e.g. 1,2,4,8, and a fit t = t0 + bytes/bw")
    p.add_argument("--reps", type=int, default=20, help="with --case: timed reps per size")
    p.add_argument("--batch", type=int, default=20, help="with --case: calls per rep, back to back")
    p.add_argument("--graph", action="store_true",
                   help="with --case: replay the rep's calls from one CUDA graph (no host issue time)")
    p.add_argument("--serve", type=int, default=None, metavar="REQUESTS",
                   help="serve one stream of this many requests through the engine alone")
    p.add_argument("--serve-rate", type=float, default=1e7, help="with --serve: arrivals per second")
    p.add_argument("--serve-bf16", action="store_true", help="with --serve: A stored as BF16")
    p.add_argument("--serve-seed", type=int, default=1)
    p.add_argument("--serve-drawn", action="store_true", help="with --serve: operands drawn per request, no pool")
    p.add_argument("--serve-budget-gb", type=float, default=64.0)
    p.add_argument("--serve-pool-log2", type=int, default=30)
    p.add_argument("--serve-chunk-mb", type=float, default=None,
                   help="with --serve: row chunk size in MB (default: the benchmark's; 0: whole requests)")
    p.add_argument("--serve-loads", action="store_true", help="with --serve: saturation, then 50/80/95%% of it")
    args = p.parse_args(argv)
    if args.serve is not None:
        run_serve_case(args)
        return
    if args.case:
        if args.case[0] not in ("gemv", "dot", "ger", "gemvq", "batch", "quant"):
            p.error("--case OP must be gemv, dot, ger, gemvq, batch or quant")
        run_case(args)
        return
    if args.warmup < 3 and args.impl == "ours":
        p.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
