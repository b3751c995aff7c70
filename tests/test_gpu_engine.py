"""The serving engine on the GPU: a Poisson stream of GEMV (FP32 and
BF16-stored A), DOT and GER requests served with continuous batching, every
result against the CPU oracle on the same inputs (the engine draws operands
from the documented counter-based generator; synth.uniform_pairs reproduces
them here):

* GEMV FP32, DOT: condition-aware relative error <= 1e-5 (FP32 tolerance);
* GEMV BF16: <= 1e-5 against the oracle on the decoded BF16 matrix (the
  same FP32 accumulation as the FP32 form);
* GER: bit-exact (one fma per element).

Also: a request's result is bit-identical alone and in the mix, a small
HBM budget is respected while every request completes, and a result buffer
that is not page-locked is refused."""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_02025_gb300 as gb
import synth
from gpu_util import rel_err

pytestmark = pytest.mark.gpu


def round_up(v, a):
    return (v + a - 1) // a * a


def operands(op, form, m, n, seed):
    U = synth.uniform_pairs
    if op == gb.REQ_GEMV:
        ld = round_up(n, 8 if form == gb.FORM_BF16 else 4)
        A = U(m * ld, seed, 1).reshape(m, ld)[:, :n]
        if form == gb.FORM_BF16:
            A = oracle.bf16_decode(oracle.bf16_encode(A.ravel())).reshape(m, n)
        return np.ascontiguousarray(A), U(n, seed, 2), U(m, seed, 3)
    if op == gb.REQ_DOT:
        return U(n, seed, 1), U(n, seed, 2), U(1, seed, 3)
    ld = round_up(n, 4)
    C = np.ascontiguousarray(U(m * ld, seed, 1).reshape(m, ld)[:, :n])
    return C, U(m, seed, 2), U(n, seed, 3)


def out_elems(op, m, n):
    return m if op == gb.REQ_GEMV else 1 if op == gb.REQ_DOT else m * n


def check(req, got):
    op, form, m, n, alpha, seed = req
    if op == gb.REQ_GEMV:
        A, x, c0 = operands(op, form, m, n, seed)
        want = oracle.gemv(0, m, n, alpha, A.ravel(), n, x, c0)
        scale = oracle.gemv_scale(0, m, n, alpha, A.ravel(), n, x, c0)
        assert rel_err(got, want, scale) <= 1e-5, req
    elif op == gb.REQ_DOT:
        x, y, a0 = operands(op, form, m, n, seed)
        want = oracle.dot(n, x, y, float(a0[0]))
        scale = oracle.dot_scale(n, x, y, float(a0[0]))
        assert abs(float(got[0]) - want) <= 1e-5 * scale, req
    else:
        C, x, y = operands(op, form, m, n, seed)
        want = oracle.ger(0, m, n, alpha, x, y, C.ravel(), n)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), req


def stream(count, seed, lo=1, hi=1500, rate=20000.0, bf16_share=0.5):
    u = (synth.uniform(count, seed, 31) + 1.0) / 2.0
    t = np.cumsum(-np.log1p(-u) / rate * 1e9).astype(np.int64)
    pick = (synth.uniform(count, seed, 32) + 1.0) / 2.0
    ops = np.where(pick < 0.7, gb.REQ_GEMV, np.where(pick < 0.9, gb.REQ_DOT, gb.REQ_GER))
    form = np.where((synth.uniform(count, seed, 33) + 1.0) / 2.0 < bf16_share, gb.FORM_BF16, gb.FORM_F32)
    m = synth.log_uniform_integers(count, seed, 34, lo, hi)
    n = synth.log_uniform_integers(count, seed, 35, lo, hi)
    reqs = []
    for i in range(count):
        op = int(ops[i])
        reqs.append((op, int(form[i]) if op == gb.REQ_GEMV else gb.FORM_F32, int(m[i]), int(n[i]),
                     0.75 if i % 2 else -1.25, seed * 100000 + i))
    return reqs, t


def serve(reqs, offsets, budget=4 << 30, streams=4, max_step=256, start_delay_ns=50_000_000):
    outs = []
    with gb.Engine(budget, streams=streams, max_inflight=4096, max_step_requests=max_step) as e:
        t0 = e.now_ns() + start_delay_ns
        for i, (op, form, m, n, alpha, seed) in enumerate(reqs):
            out = torch.empty(out_elems(op, m, n), dtype=torch.float32, pin_memory=True)
            outs.append(out)
            assert e.submit(i, op, m, n, alpha, seed, out, arrival_ns=int(t0 + offsets[i]),
                            form=form) == gb.GB_OK
        assert e.drain(120000) == gb.GB_OK
        done = e.poll()
        stats = e.stats()
    assert len(done) == len(reqs) and all(c["status"] == gb.GB_OK for c in done)
    return [o.numpy().copy() for o in outs], done, stats


def test_poisson_mix_against_oracle():
    reqs, t = stream(120, 0)
    outs, done, stats = serve(reqs, t)
    assert stats["steps"] >= 2 and stats["completed"] == len(reqs)
    for r, o in zip(reqs, outs):
        check(r, o)


def test_alone_equals_mix_bit_exact():
    reqs, t = stream(60, 1, rate=200000.0)
    mixed, done, stats = serve(reqs, t)
    assert max(np.bincount([c["step"] for c in done])) > 1, "the mix shares steps"
    for i in (0, 3, 7, 12, 25, 40, 59):
        alone, _, _ = serve([reqs[i]], [0], streams=1)
        assert np.array_equal(alone[0].view(np.uint32), mixed[i].view(np.uint32)), reqs[i]


def test_small_budget_every_request_completes_within_it():
    reqs, t = stream(80, 2, lo=200, hi=1500, rate=1e6)
    budget = 32 << 20
    outs, done, stats = serve(reqs, t, budget=budget)
    assert stats["bytes_peak"] <= budget
    for r, o in list(zip(reqs, outs))[::8]:
        check(r, o)


def test_pageable_result_buffer_is_refused():
    with gb.Engine(1 << 30) as e:
        out = np.zeros(16, np.float32)
        assert e.submit(0, gb.REQ_GEMV, 16, 16, 1.0, 0, out.ctypes.data) == -2
        assert e.stats()["submitted"] == 0


def test_operands_are_the_documented_generator():
    """A GER with alpha 0 leaves C as generated: its bits must equal
    synth.uniform_pairs (stream 1, leading dimension rounded up to 4), for
    sizes that end on every residue of the four-element store."""
    reqs = [(gb.REQ_GER, gb.FORM_F32, m, n, 0.0, 77 + k) for k, (m, n) in
            enumerate(((1, 1), (3, 5), (7, 13), (64, 64), (33, 1023), (5, 4097)))]
    outs, _, _ = serve(reqs, [0] * len(reqs))
    for (op, form, m, n, alpha, seed), got in zip(reqs, outs):
        C, _, _ = operands(op, form, m, n, seed)
        assert np.array_equal(got.reshape(m, n).view(np.uint32), C.view(np.uint32)), (m, n)


def test_full_size_stream_sampled():
    """The benchmark's serving stream (sizes log-uniform in [32, 16384], 64
    GB budget, 4 streams, every request arriving at once), 300 requests, with
    the results of sampled requests of every kind checked against the
    oracle."""
    import bench
    t, ops, m, n = bench.serve_stream(300, 1e7, 3)
    reqs = [(int(ops[i]), gb.FORM_BF16 if (ops[i] == 0 and i % 2) else gb.FORM_F32, int(m[i]), int(n[i]), 1.0,
             3 * 1000003 + i) for i in range(300)]
    small = [i for i in range(300) if int(m[i]) * int(n[i]) <= 1 << 23]
    picks = set()
    for kind in (gb.REQ_GEMV, gb.REQ_DOT, gb.REQ_GER):
        picks |= set([i for i in small if reqs[i][0] == kind][:3])
    outs = {}
    with gb.Engine(64 << 30, streams=4, max_inflight=16384, max_step_requests=512) as e:
        t0 = e.now_ns() + 100_000_000
        for i, (op, form, mi, ni, alpha, seed) in enumerate(reqs):
            out = None
            if i in picks:
                out = torch.empty(out_elems(op, mi, ni), dtype=torch.float32, pin_memory=True)
                outs[i] = out
            assert e.submit(i, op, mi, ni, alpha, seed, out, arrival_ns=int(t0 + t[i]), form=form) == gb.GB_OK
        assert e.drain(300000) == gb.GB_OK
        done = e.poll()
        stats = e.stats()
    assert len(done) == 300 and all(c["status"] == gb.GB_OK for c in done)
    assert stats["bytes_peak"] <= 64 << 30
    assert len(outs) >= 7
    for i, out in outs.items():
        check(reqs[i], out.numpy())


# ------------------------------------------------- resident operand pool --

POOL = 1 << 22
POOL_SEED = 99


def pool_operands(op, form, m, n, seed, P=POOL, pool_seed=POOL_SEED):
    """The operands a GB_REQ_POOL request reads: windows of the FP32 pool
    (stream 1 of the pool seed) or, for the A of a BF16 GEMV, of the BF16
    pool (stream 2, rounded), at synth.pool_offset of each operand stream."""
    def window(s, L, bf16=False):
        o = synth.pool_offset(seed, s, L, P)
        v = synth.uniform_pairs(L, pool_seed, 2 if bf16 else 1, offset=o)
        return oracle.bf16_decode(oracle.bf16_encode(v)) if bf16 else v
    if op == gb.REQ_GEMV:
        ld = round_up(n, 8 if form == gb.FORM_BF16 else 4)
        A = window(1, m * ld, form == gb.FORM_BF16).reshape(m, ld)[:, :n]
        return np.ascontiguousarray(A), window(2, n), window(3, m)
    if op == gb.REQ_DOT:
        return window(1, n), window(2, n), window(3, 1)
    ld = round_up(n, 4)
    C = np.ascontiguousarray(window(1, m * ld).reshape(m, ld)[:, :n])
    return C, window(2, m), window(3, n)


def check_pool(req, got):
    op, form, m, n, alpha, seed = req
    if op == gb.REQ_GEMV:
        A, x, c0 = pool_operands(op, form, m, n, seed)
        want = oracle.gemv(0, m, n, alpha, A.ravel(), n, x, c0)
        scale = oracle.gemv_scale(0, m, n, alpha, A.ravel(), n, x, c0)
        assert rel_err(got, want, scale) <= 1e-5, req
    elif op == gb.REQ_DOT:
        x, y, a0 = pool_operands(op, form, m, n, seed)
        want = oracle.dot(n, x, y, float(a0[0]))
        assert abs(float(got[0]) - want) <= 1e-5 * oracle.dot_scale(n, x, y, float(a0[0])), req
    else:
        C, x, y = pool_operands(op, form, m, n, seed)
        want = oracle.ger(0, m, n, alpha, x, y, C.ravel(), n)
        assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), req


def serve_pool(reqs, offsets, budget=1 << 30, streams=4, max_step=256, chunk_bytes=0):
    outs = []
    with gb.Engine(budget, streams=streams, max_inflight=4096, max_step_requests=max_step,
                   pool_elems=POOL, pool_seed=POOL_SEED, chunk_bytes=chunk_bytes) as e:
        assert e.stats()["pool_bytes"] == POOL * 6
        t0 = e.now_ns() + 50_000_000
        for i, (op, form, m, n, alpha, seed) in enumerate(reqs):
            out = torch.empty(out_elems(op, m, n), dtype=torch.float32, pin_memory=True)
            outs.append(out)
            assert e.submit(i, op, m, n, alpha, seed, out, arrival_ns=int(t0 + offsets[i]), form=form,
                            pool=True) == gb.GB_OK
        assert e.drain(120000) == gb.GB_OK
        done = e.poll()
        stats = e.stats()
    assert len(done) == len(reqs) and all(c["status"] == gb.GB_OK for c in done)
    return [o.numpy().copy() for o in outs], done, stats


def test_pool_mix_against_oracle():
    reqs, t = stream(120, 4)
    outs, done, stats = serve_pool(reqs, t)
    assert stats["steps"] >= 2
    for r, o in zip(reqs, outs):
        check_pool(r, o)


def test_pool_alone_equals_mix_bit_exact():
    reqs, t = stream(60, 5, rate=200000.0)
    mixed, done, _ = serve_pool(reqs, t)
    assert max(np.bincount([c["step"] for c in done])) > 1, "the mix shares steps"
    for i in (0, 5, 11, 23, 42, 59):
        alone, _, _ = serve_pool([reqs[i]], [0], streams=1)
        assert np.array_equal(alone[0].view(np.uint32), mixed[i].view(np.uint32)), reqs[i]


def test_pool_contents_are_the_documented_generator():
    """GER with alpha 0 returns C0: the FP32 pool window at its documented
    offset, bit for bit (the BF16 pool is checked by the BF16 GEMVs against
    the oracle)."""
    reqs = [(gb.REQ_GER, gb.FORM_F32, m, n, 0.0, 300 + k) for k, (m, n) in
            enumerate(((1, 1), (3, 5), (7, 13), (33, 1023), (1024, 4096)))]
    outs, _, _ = serve_pool(reqs, [0] * len(reqs))
    for (op, form, m, n, alpha, seed), got in zip(reqs, outs):
        C, _, _ = pool_operands(op, form, m, n, seed)
        assert np.array_equal(got.reshape(m, n).view(np.uint32), C.view(np.uint32)), (m, n)


def test_pool_bf16_and_edges():
    """BF16 GEMVs, DOTs and GERs of ragged sizes, and operands as long as the
    pool allows (offset 0 is then the only start)."""
    side = 2048                               # 2048 x 2048 = POOL
    reqs = [(gb.REQ_GEMV, gb.FORM_BF16, m, n, 0.5, 400 + k) for k, (m, n) in
            enumerate(((1, 1), (5, 7), (64, 129), (333, 1000), (side, side)))]
    reqs += [(gb.REQ_DOT, gb.FORM_F32, 1, n, 1.0, 500 + k) for k, n in enumerate((1, 3, 4097, POOL))]
    reqs += [(gb.REQ_GER, gb.FORM_F32, m, n, -1.5, 600 + k) for k, (m, n) in
             enumerate(((1, 1), (9, 3), (100, 1001), (side, side)))]
    outs, _, _ = serve_pool(reqs, [0] * len(reqs))
    for r, o in zip(reqs, outs):
        check_pool(r, o)


def test_pool_refusals():
    with gb.Engine(1 << 30, pool_elems=POOL) as e:
        assert e.submit(0, gb.REQ_GER, 2048, 2049, pool=True) == -2       # ld 2052 x 2048 > POOL
        assert e.submit(1, gb.REQ_DOT, 1, POOL + 1, pool=True) == -2
        assert e.stats()["submitted"] == 0
    with gb.Engine(1 << 30) as e:
        assert e.submit(0, gb.REQ_GEMV, 8, 8, pool=True) == -2            # no pool


def test_pool_chunks_against_oracle_and_bit_identical_to_whole():
    """Row chunks of 64 KB (most GEMVs and GERs of the stream split into
    several steps, on several streams): every result against the oracle and
    bit-identical to the same request served whole and alone."""
    reqs, t = stream(80, 6, rate=100000.0)
    chunked, done, stats = serve_pool(reqs, t, chunk_bytes=64 << 10)
    assert stats["steps"] > 80
    for r, o in zip(reqs, chunked):
        check_pool(r, o)
    for i in (0, 3, 9, 17, 33, 51, 79):
        whole, _, _ = serve_pool([reqs[i]], [0], streams=1)
        assert np.array_equal(whole[0].view(np.uint32), chunked[i].view(np.uint32)), reqs[i]


def test_pool_chunks_of_one_row():
    """chunk_bytes below one row: every chunk is a single row."""
    reqs = [(gb.REQ_GEMV, gb.FORM_F32, 37, 300, 0.5, 700), (gb.REQ_GER, gb.FORM_F32, 29, 301, -2.0, 701),
            (gb.REQ_GEMV, gb.FORM_BF16, 41, 999, 1.0, 702), (gb.REQ_DOT, gb.FORM_F32, 1, 5000, 1.0, 703)]
    outs, done, stats = serve_pool(reqs, [0, 0, 0, 0], chunk_bytes=16)
    assert stats["steps"] >= 41
    for r, o in zip(reqs, outs):
        check_pool(r, o)


# ------------------------------------------------------------ served DOTs --

DOT_BOUND = 2.0 ** -22   # two FP32 roundings of |alpha0| + sum |x_p y_p|, as gb_sdot


def dot_stream(count, seed, rate):
    reqs, t = stream(count, seed, lo=32, hi=16384, rate=rate)
    return [(gb.REQ_DOT, gb.FORM_F32, 1, n, 1.0, s) for (_, _, _, n, _, s) in reqs], t


def test_served_dots_fp64_final_sum():
    """DOT requests (Def. DOT; Algs. 3-4) take per-thread Dot2 in FP32 and
    the final sum, with the initial alpha, in FP64 (the batched kernel's
    DOT tiles): every served result within 2^-22 of the condition-aware
    scale of the FP64 oracle, drawn and pool operands, and bit-identical
    alone and in the mix."""
    reqs, t = dot_stream(60, 5, rate=200000.0)
    outs, done, _ = serve(reqs, t)
    assert max(np.bincount([c["step"] for c in done])) > 1, "the DOTs share steps"
    for r, o in zip(reqs, outs):
        x, y, a0 = operands(gb.REQ_DOT, gb.FORM_F32, 1, r[3], r[5])
        want = oracle.dot(r[3], x, y, float(a0[0]))
        scale = oracle.dot_scale(r[3], x, y, float(a0[0]))
        assert abs(float(o[0]) - want) <= DOT_BOUND * scale, (r, abs(float(o[0]) - want) / scale)
    for i in (0, 9, 33):
        alone, _, _ = serve([reqs[i]], [0], streams=1)
        assert np.array_equal(alone[0].view(np.uint32), outs[i].view(np.uint32)), reqs[i]
    pouts, _, _ = serve_pool(reqs, t)
    for r, o in zip(reqs, pouts):
        x, y, a0 = pool_operands(gb.REQ_DOT, gb.FORM_F32, 1, r[3], r[5])
        want = oracle.dot(r[3], x, y, float(a0[0]))
        scale = oracle.dot_scale(r[3], x, y, float(a0[0]))
        assert abs(float(o[0]) - want) <= DOT_BOUND * scale, (r, abs(float(o[0]) - want) / scale)
