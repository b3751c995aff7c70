"""The serving engine's host logic, without a GPU (GB_ENGINE_HOST_ONLY: the
arena is bookkeeping only and a step completes after its operand bytes /
simulated bandwidth).  Checked: requests are admitted in arrival order and
never before they arrive, the HBM budget, the in-flight cap and the step
size are never exceeded, requests that arrive while steps run are batched
into later steps that overlap, the timestamps of every completion are
ordered, oversize and invalid requests are refused, and a failed step
(host-side fault injection) completes its requests with an error while the
engine goes on."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

import paper_2108_02025_gb300 as gb
import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MB = 1 << 20


def poisson_stream(count, rate_per_s, seed, lo=32, hi=4096, mix=(0.7, 0.2, 0.1)):
    """(arrival offset ns, op, m, n) of a Poisson stream with the op mix."""
    u = (synth.uniform(count, seed, 21) + 1.0) / 2.0
    gaps = -np.log1p(-u) / rate_per_s * 1e9
    t = np.cumsum(gaps).astype(np.int64)
    pick = (synth.uniform(count, seed, 22) + 1.0) / 2.0
    ops = np.where(pick < mix[0], gb.REQ_GEMV, np.where(pick < mix[0] + mix[1], gb.REQ_DOT, gb.REQ_GER))
    m = synth.log_uniform_integers(count, seed, 23, lo, hi)
    n = synth.log_uniform_integers(count, seed, 24, lo, hi)
    return t, ops, m, n


def run_stream(engine, count, rate, seed=0, start_delay_ns=20_000_000, **kw):
    t, ops, m, n = poisson_stream(count, rate, seed, **kw)
    t0 = engine.now_ns() + start_delay_ns
    for i in range(count):
        assert engine.submit(i, int(ops[i]), int(m[i]), int(n[i]), 1.0, seed * 100000 + i,
                             arrival_ns=int(t0 + t[i])) == gb.GB_OK
    assert engine.drain(60000) == gb.GB_OK
    done = engine.poll()
    assert len(done) == count
    return sorted(done, key=lambda c: c["id"]), (t0 + t), ops, m, n


def test_admission_order_budget_and_caps():
    budget = 256 * MB
    with gb.Engine(budget, streams=3, max_inflight=40, max_step_requests=16, host_only=True,
                   sim_bytes_per_ns=200.0) as e:
        done, arrivals, ops, m, n = run_stream(e, 400, 20000.0, seed=1)
        st = e.stats()
    assert st["completed"] == 400 and st["failed"] == 0
    assert st["bytes_peak"] <= budget and st["bytes_in_use"] == 0
    assert st["inflight_peak"] <= 40
    assert 1 < st["steps_inflight_peak"] <= 3, "steps overlap, at most one per stream"
    adm = np.array([c["admitted_ns"] for c in done])
    arr = np.array([c["arrival_ns"] for c in done])
    assert np.array_equal(arr, arrivals)
    assert np.all(adm >= arr), "no request is admitted before it arrives"
    assert np.all(np.diff(adm) >= 0), "admission in arrival order"
    for c in done:
        assert c["arrival_ns"] <= c["admitted_ns"] <= c["launched_ns"] <= c["done_ns"]
        assert c["status"] == gb.GB_OK
        assert c["bytes"] == gb.request_bytes(c["op"], int(m[c["id"]]), int(n[c["id"]]))
    steps = np.array([c["step"] for c in done])
    assert np.bincount(steps).max() <= 16
    assert np.all(np.diff(steps) >= 0), "steps take admitted requests in order"


def test_continuous_batching_under_load():
    """At an arrival rate above the simulated capacity, requests that arrive
    while steps are running are launched together in later steps."""
    with gb.Engine(1 << 34, streams=2, max_inflight=4096, max_step_requests=256, host_only=True,
                   sim_bytes_per_ns=20.0) as e:
        done, _, _, _, _ = run_stream(e, 600, 200000.0, seed=2)
        st = e.stats()
    steps = np.bincount([c["step"] for c in done])
    assert st["steps"] < 600 / 4, "requests share steps"
    assert steps.max() > 10
    assert st["steps_inflight_peak"] == 2


def test_memory_returns_and_big_requests_wait_for_it():
    """Requests of half the budget each run at most two at a time."""
    r_bytes = gb.request_bytes(gb.REQ_GER, 2048, 2048)
    budget = 2 * r_bytes + MB
    with gb.Engine(budget, streams=4, max_inflight=100, max_step_requests=100, host_only=True,
                   sim_bytes_per_ns=50.0) as e:
        t0 = e.now_ns()
        for i in range(10):
            assert e.submit(i, gb.REQ_GER, 2048, 2048, 1.0, i, arrival_ns=t0) == gb.GB_OK
        assert e.drain(60000) == gb.GB_OK
        done = e.poll()
        st = e.stats()
    assert st["bytes_peak"] <= budget and st["inflight_peak"] == 2
    assert len(done) == 10 and all(c["status"] == gb.GB_OK for c in done)


def test_refusals():
    with gb.Engine(64 * MB, host_only=True) as e:
        assert e.submit(0, gb.REQ_GEMV, 8192, 8192) == gb.GB_ERR_BUDGET      # 256 MB alone
        assert e.submit(1, gb.REQ_GEMV, 0, 10) == -2
        assert e.submit(2, gb.REQ_GEMV, 10, 0) == -2
        assert e.submit(3, 7, 10, 10) == -2
        assert e.submit(4, gb.REQ_DOT, 1, 10, form=gb.FORM_BF16) == -2
        assert e.submit(5, gb.REQ_GER, 10, 2 ** 31) == -2
        assert e.submit(6, gb.REQ_DOT, 0, 10) == gb.GB_OK                     # DOT ignores m
        assert e.drain(10000) == gb.GB_OK
        assert len(e.poll()) == 1
        assert e.stats()["submitted"] == 1
    cfg = gb.EngineConfig(1 << 10, 1, 1, 1, gb.ENGINE_HOST_ONLY, 1.0, None)   # budget < 1 MiB
    h = gb.ctypes.c_void_p()
    assert gb.gb_engine_create(cfg, gb.ctypes.addressof(h)) == -1
    cfg = gb.EngineConfig(1 << 30, 17, 1, 1, gb.ENGINE_HOST_ONLY, 1.0, None)  # streams
    assert gb.gb_engine_create(cfg, gb.ctypes.addressof(h)) == -1
    cfg = gb.EngineConfig(1 << 30, 1, 1, 1, gb.ENGINE_HOST_ONLY, 0.0, None)   # bandwidth
    assert gb.gb_engine_create(cfg, gb.ctypes.addressof(h)) == -1
    bad = gb.tuning_table({3: (3, 1, 65536)})
    cfg = gb.EngineConfig(1 << 30, 1, 1, 1, gb.ENGINE_HOST_ONLY, 1.0, gb._addr(bad))
    assert gb.gb_engine_create(cfg, gb.ctypes.addressof(h)) == -1
    assert gb.gb_engine_create(None, gb.ctypes.addressof(h)) == -1
    assert gb.gb_engine_create(cfg, None) == -2
    assert gb.gb_engine_submit(None, None) == -1
    assert gb.gb_engine_poll(None, None, 1) == -1
    assert gb.gb_engine_drain(None, 1) == -1


def test_request_bytes():
    # GEMV FP32 10 x 10: A 10 x 12 floats, x, c: 256-byte pieces
    assert gb.request_bytes(gb.REQ_GEMV, 10, 10) == 512 + 256 + 256
    assert gb.request_bytes(gb.REQ_GEMV, 1000, 1000) == 4000000 + 4096 + 4096
    assert gb.request_bytes(gb.REQ_GEMV, 1000, 1000, gb.FORM_BF16) >= 2000000 + 2 * 4096
    assert gb.request_bytes(gb.REQ_DOT, 5, 1000) == 4096 + 4096 + 256
    assert gb.request_bytes(gb.REQ_GER, 1000, 1000) == 4000000 + 4096 + 4096
    assert gb.request_bytes(gb.REQ_GEMV, 0, 10) == 0


def test_injected_step_failure_completes_with_error_and_the_engine_goes_on():
    code = textwrap.dedent("""
        import sys
        sys.path.insert(0, %r)
        import paper_2108_02025_gb300 as gb
        with gb.Engine(1 << 30, streams=1, max_step_requests=1, host_only=True,
                       sim_bytes_per_ns=100.0) as e:
            t0 = e.now_ns()
            for i in range(4):
                assert e.submit(i, gb.REQ_GEMV, 64, 64, 1.0, i, arrival_ns=t0 + i * 1000000) == 0
            assert e.drain(20000) == 0
            done = sorted(e.poll(), key=lambda c: c["id"])
            print([c["status"] for c in done], [c["step"] for c in done], e.stats()["failed"])
    """ % ROOT)
    env = dict(os.environ, GB_FAULT_INJECT="step:2")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                         timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "[0, -103, 0, 0] [0, 1, 2, 3] 1"


def test_engine_header_symbols_exported():
    import re
    text = open(os.path.join(ROOT, "include", "gbserve.h")).read()
    names = sorted(set(re.findall(r"^\s*(?:int|int64_t|size_t|void)\s*(gb_\w+)\s*\(", text, re.M)))
    assert names == sorted(gb.ENGINE_EXPORTS)
    for name in names:
        assert hasattr(gb.lib(), name)


def test_pool_requests_hold_only_their_output():
    """With resident operands (GB_REQ_POOL) a request holds its output alone
    in the arena; operands longer than the pool, pool requests without a pool
    and unknown flags are refused; pool sizes must be multiples of 8."""
    assert gb.request_bytes(gb.REQ_GEMV, 10, 10, pool=True) == 256
    assert gb.request_bytes(gb.REQ_GEMV, 1000, 1000, gb.FORM_BF16, pool=True) == 4096
    assert gb.request_bytes(gb.REQ_DOT, 1, 1000, pool=True) == 256
    assert gb.request_bytes(gb.REQ_GER, 1000, 1001, pool=True) == 1000 * 1004 * 4 // 256 * 256 + 256
    P = 1 << 20
    with gb.Engine(64 * MB, host_only=True, pool_elems=P, sim_bytes_per_ns=100.0) as e:
        assert e.submit(0, gb.REQ_GEMV, 1024, 1024, pool=True) == gb.GB_OK        # A = 2^20 elements
        assert e.submit(1, gb.REQ_GEMV, 1024, 1025, pool=True) == -2              # ld 1028: too long
        assert e.submit(2, gb.REQ_GEMV, 1024, 1024, form=gb.FORM_BF16, pool=True) == gb.GB_OK
        assert e.submit(3, gb.REQ_DOT, 1, P, pool=True) == gb.GB_OK
        assert e.submit(4, gb.REQ_DOT, 1, P + 1, pool=True) == -2
        assert e.submit(5, gb.REQ_GER, 2048, 512, pool=True) == gb.GB_OK
        assert e.submit(6, gb.REQ_GER, 2048, 513, pool=True) == -2
        r = gb.Request(7, gb.REQ_GEMV, 0, 8, 8, 1.0, 2, 0, None, 0)               # unknown flag
        assert gb.gb_engine_submit(e.h, gb.ctypes.addressof(r)) == -2
        assert e.drain(10000) == gb.GB_OK
        done = sorted(e.poll(), key=lambda c: c["id"])
        assert [c["id"] for c in done] == [0, 2, 3, 5]
        assert [c["bytes"] for c in done] == [4096, 4096, 256, 2048 * 512 * 4]
        assert e.stats()["pool_bytes"] == 0                                       # host-only: none allocated
    with gb.Engine(64 * MB, host_only=True) as e:
        assert e.submit(0, gb.REQ_GEMV, 8, 8, pool=True) == -2
    h = gb.ctypes.c_void_p()
    for bad in (-8, 12):
        cfg = gb.EngineConfig(1 << 30, 1, 1, 1, gb.ENGINE_HOST_ONLY, 1.0, None, bad, 0)
        assert gb.gb_engine_create(cfg, gb.ctypes.addressof(h)) == -1


def test_pool_offsets_stay_inside_the_pool_and_are_aligned():
    import synth
    P = 1 << 16
    for seed in range(200):
        for s, L in ((1, 1), (2, 4093), (3, P), (1, P - 8), (2, 777)):
            o = synth.pool_offset(seed, s, L, P)
            assert o % 8 == 0 and 0 <= o and o + L <= P
    offs = {synth.pool_offset(seed, 1, 1000, P) for seed in range(200)}
    assert len(offs) > 150, "operands of different requests start at different places"


def test_chunks_let_small_requests_pass_large_ones():
    """With chunk_bytes set, a large pool GEMV or GER is launched a chunk of
    rows at a time; small requests that arrive after it run between its
    chunks and complete long before it, and it completes once, with every
    row launched."""
    P = 1 << 26
    chunk = 4 * MB
    with gb.Engine(1 << 30, streams=2, max_inflight=1000, max_step_requests=64, host_only=True,
                   sim_bytes_per_ns=4.0, pool_elems=P, chunk_bytes=chunk) as e:
        t0 = e.now_ns() + 5_000_000
        assert e.submit(0, gb.REQ_GEMV, 4096, 4096, pool=True, arrival_ns=t0) == gb.GB_OK      # 64 MB
        assert e.submit(1, gb.REQ_GER, 2048, 4096, pool=True, arrival_ns=t0 + 1) == gb.GB_OK   # 64 MB
        for i in range(2, 40):
            assert e.submit(i, gb.REQ_GEMV, 64, 64, pool=True, arrival_ns=t0 + 200_000 * i) == gb.GB_OK
        assert e.drain(60000) == gb.GB_OK
        done = {c["id"]: c for c in e.poll()}
        st = e.stats()
    assert len(done) == 40 and all(c["status"] == gb.GB_OK for c in done.values())
    assert st["steps"] >= 2 * (64 * MB // chunk), "the large requests went in chunks"
    assert st["bytes_in_use"] == 0 and st["inflight_peak"] <= 40
    big_done = min(done[0]["done_ns"], done[1]["done_ns"])
    small = [done[i] for i in range(2, 40) if done[i]["arrival_ns"] < big_done - 4_000_000]
    assert len(small) > 5
    assert all(c["done_ns"] <= big_done for c in small), "small requests overtake the chunked ones"
    for c in done.values():
        assert c["arrival_ns"] <= c["admitted_ns"] <= c["launched_ns"] <= c["done_ns"]


def test_chunked_request_with_a_failed_chunk_completes_with_the_error():
    code = textwrap.dedent("""
        import sys
        sys.path.insert(0, %r)
        import paper_2108_02025_gb300 as gb
        with gb.Engine(1 << 30, streams=2, host_only=True, sim_bytes_per_ns=100.0, pool_elems=1 << 24,
                       chunk_bytes=1 << 20) as e:
            assert e.submit(0, gb.REQ_GER, 1024, 1024, pool=True) == 0        # 8 MB: 8 chunks
            assert e.drain(20000) == 0
            assert e.submit(1, gb.REQ_GEMV, 32, 32, pool=True) == 0
            assert e.drain(20000) == 0
            done = sorted(e.poll(), key=lambda c: c["id"])
            st = e.stats()
            print([c["status"] for c in done], st["failed"], st["steps"], st["bytes_in_use"])
    """ % ROOT)
    env = dict(os.environ, GB_FAULT_INJECT="step:3")
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert out.stdout.strip() == "[-103, 0] 1 9 0"
