"""Batched FP32 GEMV (gb_sgemv_batch: many row-major problems, one
persistent launch) on the GPU against the CPU oracle, problem by problem,
element by element (Def. GEMV per problem).

Tolerance as for the single FP32 GEMV, per row i of problem p:
    |c_i - c_oracle_i| / (|c0_i| + |alpha_p| sum_j |A_ij x_j|) <= 1e-5
Also: a problem's result is bit-identical alone and in any batch, a graph
replay equals a direct launch, every kernel variant a tuning table can
select passes, padding (NaN) and bytes around every c are never touched,
and the full-size workload (4096 problems, m, n log-uniform in [32, 8192])
matches the oracle on sampled problems."""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_02025_gb300 as gb
import synth
from gpu_util import Guarded, rel_err, to_dev

pytestmark = pytest.mark.gpu
TOL = 1e-5


def make(m, n, pad, seed):
    ld = max(n + pad, 1)
    size = (m - 1) * ld + n if m > 0 and n > 0 else 0
    A = synth.uniform(size, seed, 1, np.float32)
    for r in range(m - 1):
        A[r * ld + n:(r + 1) * ld] = np.nan  # any read of padding poisons c
    x = synth.uniform(n, seed, 2, np.float32)
    c0 = synth.uniform(m, seed, 3, np.float32)
    return A, x, c0, ld


class Problem:
    def __init__(self, m, n, pad=0, alpha=0.75, seed=0, misalign=0):
        self.m, self.n, self.alpha, self.misalign = m, n, alpha, misalign
        self.A, self.x, self.c0, self.ld = make(m, n, pad, seed)

    def device(self):
        self.dA = to_dev(self.A, self.misalign)
        self.dx = to_dev(self.x, self.misalign)
        self.dc = Guarded(self.c0, self.misalign)
        return (self.dA, self.dx, self.dc.view, self.alpha, self.m, self.n, self.ld)

    def want(self):
        return (oracle.gemv(0, self.m, self.n, self.alpha, self.A, self.ld, self.x, self.c0),
                oracle.gemv_scale(0, self.m, self.n, self.alpha, self.A, self.ld, self.x, self.c0))


def run(problems, table=None, graph=False, launches=1):
    b = gb.Batch([p.device() for p in problems], table=table)
    if graph:
        b.capture()
        for _ in range(launches):
            b.replay()
    else:
        for _ in range(launches):
            b.launch()
    torch.cuda.synchronize()
    return [p.dc.result() for p in problems], b


def mixed(seed=0, count=60):
    ms = synth.log_uniform_integers(count, seed, 11, 1, 3000)
    ns = synth.log_uniform_integers(count, seed, 12, 1, 3000)
    pads = synth.integers(count, seed, 13, 0, 5, np.int64)
    mis = synth.integers(count, seed, 14, 0, 3, np.int64)
    probs = [Problem(int(ms[i]), int(ns[i]), int(pads[i]), 0.75 if i % 3 else -1.25, seed * 1000 + i,
                     int(mis[i]) if i % 4 == 0 else 0) for i in range(count)]
    # edge cases: empty, zero alpha, single row / column, ragged tails
    probs += [Problem(0, 10), Problem(10, 0), Problem(7, 9, alpha=0.0), Problem(1, 1), Problem(1, 8193),
              Problem(8193, 1), Problem(5, 3, pad=1), Problem(33, 4099, pad=2, misalign=1),
              Problem(257, 4096), Problem(3, 8192, pad=4)]
    return probs


def check(probs, got):
    for p, g in zip(probs, got):
        want, scale = p.want()
        if p.alpha == 0.0 or p.m == 0 or p.n == 0:
            assert np.array_equal(g.view(np.uint32), p.c0.view(np.uint32)), (p.m, p.n)
            continue
        err = rel_err(g, want, scale)
        assert err <= TOL, (p.m, p.n, p.ld, p.misalign, err)


def test_mixed_batch_against_oracle():
    probs = mixed()
    got, b = run(probs)
    assert b.tiles > 0
    check(probs, got)


def test_alone_equals_mix_bit_exact():
    probs = mixed(seed=1)
    got, _ = run(probs)
    for i in (0, 5, 13, 41, len(probs) - 1, len(probs) - 3):
        alone, _ = run([probs[i]])
        assert np.array_equal(alone[0].view(np.uint32), got[i].view(np.uint32)), i


def test_graph_replay_equals_launch_and_repeats_bit_identical():
    probs = mixed(seed=2, count=30)
    direct, _ = run(probs, launches=2)
    graphed, _ = run(probs, graph=True, launches=2)
    again, _ = run(probs, launches=2)
    for a, b, c in zip(direct, graphed, again):
        assert np.array_equal(a.view(np.uint32), b.view(np.uint32))
        assert np.array_equal(a.view(np.uint32), c.view(np.uint32))


@pytest.mark.parametrize("lpr", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("u", [1, 2, 4])
def test_every_kernel_variant(lpr, u):
    table = gb.tuning_table({b: (lpr, u, 4096 if b % 2 else 65536) for b in range(gb.BATCH_BUCKETS)})
    # (m, n, pad, misalign): lda = n + pad; the 16-byte path needs lda % 4 == 0,
    # so the ragged columns of that path are covered by n % 4 = 1, 2, 3 with pad 3, 2, 1
    probs = [Problem(m, n, pad, 0.5, 100 + lpr * 10 + u, mis) for (m, n, pad, mis) in
             ((1, 1, 0, 0), (3, 5, 1, 0), (300, 257, 0, 0), (97, 1027, 3, 0), (40, 4096, 0, 0),
              (1000, 33, 0, 0), (17, 999, 0, 1), (2, 20000, 0, 0), (4097, 64, 0, 0),
              (374, 59, 1, 0), (70, 61, 3, 0), (9, 4098, 2, 0), (300, 3, 1, 0), (5, 2, 2, 0),
              (33, 1, 3, 0))]
    got, _ = run(probs, table=table)
    check(probs, got)


def test_empty_batch_is_a_no_op():
    b = gb.Batch([])
    assert b.tiles == 0
    b.launch()
    torch.cuda.synchronize()


def test_full_size_workload_sampled():
    """The 4096-problem workload of the batched benchmark, in its launch
    configuration, checked against the oracle on sampled problems (the
    largest, the smallest and seeded picks)."""
    import bench
    dev = torch.device("cuda", 0)
    wl = bench.BatchWorkload(dev)
    sizes = wl.m * wl.n
    picks = sorted({int(np.argmax(sizes)), int(np.argmin(sizes))} |
                   set(synth.integers(6, 0, 15, 0, len(wl.problems) - 1, np.int64).tolist()))
    before = {}
    for p in picks:
        a, x, c = wl.operands(p)
        before[p] = (a.cpu().numpy().ravel(), x.cpu().numpy(), c.cpu().numpy())
    b = gb.Batch(wl.problems, table=gb.load_tuning(), device=dev)
    b.launch()
    torch.cuda.synchronize()
    for p in picks:
        A, x, c0 = before[p]
        m, n, ld = int(wl.m[p]), int(wl.n[p]), int(wl.lda[p])
        got = wl.operands(p)[2].cpu().numpy()
        want = oracle.gemv(0, m, n, 1.0, A, ld, x, c0)
        scale = oracle.gemv_scale(0, m, n, 1.0, A, ld, x, c0)
        assert rel_err(got, want, scale) <= TOL, (p, m, n)
    del wl, b
    torch.cuda.empty_cache()


class Item:
    """One gb_batch_item on the device, with its oracle."""

    def __init__(self, kind, m, n, pad, alpha, seed, misalign=0):
        self.kind, self.m, self.n, self.alpha = kind, m, n, alpha
        self.ld = max(n + pad, 1)
        size = (m - 1) * self.ld + n if m > 0 and n > 0 else 0
        A = synth.uniform(size, seed, 1, np.float32)
        if kind == gb.BATCH_GEMV_BF16:
            self.codes = oracle.bf16_encode(A)
            for r in range(m - 1):  # padding codes: NaN
                self.codes[r * self.ld + n:(r + 1) * self.ld] = 0x7FC0
            self.A = oracle.bf16_decode(self.codes)
            self.dA = to_dev(self.codes.view(np.int16), misalign)
        else:
            for r in range(m - 1):
                A[r * self.ld + n:(r + 1) * self.ld] = np.nan
            self.A = A
            self.dA = to_dev(A, misalign)
        self.vec_n = synth.uniform(n, seed, 2, np.float32)
        self.vec_m = synth.uniform(m, seed, 3, np.float32)
        self.dx = to_dev(self.vec_n, misalign)
        if kind == gb.BATCH_GER_F32:
            self.dc = to_dev(self.vec_m, misalign)
            self.out = None
        else:
            self.out = Guarded(self.vec_m, misalign)
            self.dc = self.out.view

    def entry(self):
        return (self.kind, self.dA, self.dx, self.dc, self.alpha, self.m, self.n, self.ld)

    def check(self):
        if self.kind == gb.BATCH_GER_F32:
            got = self.dA.cpu().numpy()
            want = oracle.ger(0, self.m, self.n, self.alpha, self.vec_m, self.vec_n, self.A, self.ld)
            live = ~np.isnan(self.A)
            assert np.array_equal(got[live].view(np.uint32), want[live].view(np.uint32)), (self.m, self.n)
            assert np.all(np.isnan(got[~live])), "GER wrote padding"
            return
        got = self.out.result()
        if self.alpha == 0 or self.m == 0 or self.n == 0:
            assert np.array_equal(got.view(np.uint32), self.vec_m.view(np.uint32))
            return
        want = oracle.gemv(0, self.m, self.n, self.alpha, self.A, self.ld, self.vec_n, self.vec_m)
        scale = oracle.gemv_scale(0, self.m, self.n, self.alpha, self.A, self.ld, self.vec_n, self.vec_m)
        assert rel_err(got, want, scale) <= TOL, (self.kind, self.m, self.n, self.ld)


MIXED_SHAPES = ((1, 1, 0, 0), (3, 5, 1, 0), (300, 257, 0, 0), (97, 1027, 5, 0), (40, 4096, 0, 0),
                (1000, 33, 0, 0), (17, 999, 1, 1), (2, 20000, 0, 0), (4097, 64, 0, 0), (374, 59, 5, 0),
                (70, 61, 3, 0), (9, 4098, 6, 0), (300, 3, 5, 0), (5, 2, 6, 0), (33, 1, 7, 0), (50, 16, 0, 3))


@pytest.mark.parametrize("lpr", [1, 2, 4, 8, 16, 32])
@pytest.mark.parametrize("u", [1, 2, 4])
def test_mixed_kinds_every_variant(lpr, u):
    """FP32 GEMV, BF16 GEMV and GER items in one launch, 16-byte and scalar
    paths (pads make lda * element bytes a multiple of 16 or not)."""
    table = gb.tuning_table({b: (lpr, u, 4096 if b % 2 else 65536) for b in range(gb.BATCH_BUCKETS)})
    items = []
    for k, (m, n, pad, mis) in enumerate(MIXED_SHAPES):
        for kind in (gb.BATCH_GEMV_F32, gb.BATCH_GEMV_BF16, gb.BATCH_GER_F32):
            items.append(Item(kind, m, n, pad, (0.5, -1.25, 0.0)[k % 3] if k % 5 else 0.75,
                              1000 * lpr + 100 * u + 10 * k + kind, mis))
    b = gb.Batch.from_items([it.entry() for it in items], table=table)
    b.launch()
    torch.cuda.synchronize()
    for it in items:
        it.check()


DOT_BOUND = 2.0 ** -22   # two FP32 roundings of the condition-aware scale


@pytest.mark.parametrize("mis", [0, 1], ids=["aligned", "misaligned"])
def test_dot_items_fp64_final_sum(mis):
    """GB_BATCH_DOT_F32 tiles (Def. DOT; Algs. 3-4): per-thread Dot2 in FP32,
    the threads' parts and the initial accumulator summed in FP64, one
    rounding to FP32.  Each result within 2^-22 of |alpha0| + sum |x_p y_p|
    of the FP64 oracle, the bound gb_sdot meets on the same inputs; mixed
    with GEMV items in one launch."""
    ns = [1, 3, 4, 37, 1000, 1027, 4096, 16384, 100003]
    items, dots = [], []
    for k, n in enumerate(ns):
        x = synth.uniform(n, 500 + k, 1, np.float32)
        y = synth.uniform(n, 500 + k, 2, np.float32)
        a0 = synth.uniform(1, 500 + k, 3, np.float32)
        out = Guarded(a0, mis)
        dx, dy = to_dev(x, mis), to_dev(y, mis)
        items.append((gb.BATCH_DOT_F32, dx, dy, out.view, 1.0, 1, n, n))
        dots.append((n, x, y, a0, out, dx, dy))
    gemv = Item(gb.BATCH_GEMV_F32, 300, 257, 0, 0.5, 77)
    b = gb.Batch.from_items(items + [gemv.entry()])
    b.launch()
    torch.cuda.synchronize()
    gemv.check()
    for (n, x, y, a0, out, dx, dy) in dots:
        got = float(out.result()[0])
        want = oracle.dot(n, x, y, float(a0[0]))
        scale = oracle.dot_scale(n, x, y, float(a0[0]))
        assert abs(got - want) <= DOT_BOUND * scale, (n, abs(got - want) / scale)
        # gb_sdot on the same operands meets the same bound
        ref = Guarded(a0.copy())
        nb = gb.gb_workspace_bytes(gb.OP_DOT, gb.F32, 0, 0, n)
        ws = torch.zeros(max(nb, 1), dtype=torch.uint8, device="cuda")
        assert gb.gb_sdot(n, dx, dy, ref.view, ws, nb) == gb.GB_OK
        torch.cuda.synchronize()
        assert abs(float(ref.result()[0]) - want) <= DOT_BOUND * scale, n
