"""Property tests of the host-side logic (no GPU): randomized batches for
the batched-GEMV planner, randomized streams for the serving engine in
host-only mode, and the workspace function.  Uses hypothesis when it is
installed."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import paper_2108_02025_gb300 as gb  # noqa: E402
from test_batch_plan import aligned_buffer, decode_raw  # noqa: E402

KINDS = (gb.BATCH_GEMV_F32, gb.BATCH_GEMV_BF16, gb.BATCH_GER_F32)


def item_arrays(specs, base=1 << 42):
    arr = (gb.BatchItem * max(1, len(specs)))()
    addr = base
    for i, (kind, m, n, pad, alpha) in enumerate(specs):
        eb = 2 if kind == gb.BATCH_GEMV_BF16 else 4
        lda = max(n + pad, 1)
        a = addr
        addr += (max(m, 1) * lda * eb + 255) // 256 * 256 + 256
        xx = addr
        addr += (max(n, 1) * 4 + 255) // 256 * 256 + 256
        cc = addr
        addr += (max(m, 1) * 4 + 255) // 256 * 256 + 256
        arr[i] = gb.BatchItem(kind, 0, m, n, lda, alpha, 0, a, xx, cc)
    return arr


spec = st.tuples(st.sampled_from(KINDS), st.integers(0, 3000), st.integers(0, 9000), st.integers(0, 9),
                 st.sampled_from([1.0, -0.5, 0.0, 2.0]))


@settings(max_examples=60, deadline=None)
@given(st.lists(spec, min_size=0, max_size=25), st.integers(0, 3))
def test_planner_covers_every_row_once(specs, tune):
    table = [None, gb.tuning_table(), gb.tuning_table({b: (1 << (b % 6), 1 << (b % 3), 4096 << (b % 5))
                                                      for b in range(gb.BATCH_BUCKETS)}),
             gb.tuning_table({b: (32, 4, 1 << 21) for b in range(gb.BATCH_BUCKETS)})][tune]
    arr = item_arrays(specs)
    nb = gb.gb_batch_plan_bytes(len(specs), arr, table)
    assert nb > 0
    buf = aligned_buffer(nb)
    assert gb.gb_batch_plan(len(specs), arr, table, buf, nb) == gb.GB_OK
    h, probs, raw, prefix = decode_raw(buf)
    assert h["tiles"] == raw.size and prefix[0] == 0 and prefix[-1] == h["total"]
    assert np.all(np.diff(prefix) > 0)
    seen = 0
    for p, (kind, m, n, pad, alpha) in enumerate(specs):
        c0 = arr[p].c
        mine = raw[(raw["c"] >= np.uint64(c0)) & (raw["c"] < np.uint64(c0 + 4 * max(m, 1)))]
        if m == 0 or n == 0 or alpha == 0.0:
            assert mine.size == 0
            continue
        rows0 = (mine["c"] - np.uint64(c0)) // np.uint64(4)
        assert np.array_equal(rows0, np.concatenate([[0], np.cumsum(mine["rows"])[:-1]]).astype(np.uint64))
        assert int(mine["rows"].sum()) == m and np.all(mine["kind"] == kind)
        assert np.all(mine["n"] == n) and np.all(mine["alpha"] == np.float32(alpha))
        seen += mine.size
    assert seen == raw.size


@settings(max_examples=40, deadline=None)
@given(st.lists(st.tuples(st.sampled_from([gb.REQ_GEMV, gb.REQ_DOT, gb.REQ_GER]), st.integers(1, 3000),
                          st.integers(1, 3000), st.integers(0, 200000), st.booleans()), min_size=1, max_size=60),
       st.integers(8, 64), st.integers(1, 4), st.integers(1, 50), st.integers(1, 20),
       st.sampled_from([0, 1, 4096, 1 << 20]))
def test_engine_host_only_invariants(reqs, budget_mb, streams, max_inflight, max_step, chunk):
    """Random streams of drawn and pool requests, with and without row
    chunks: every accepted request completes once, the budget and the caps
    hold, admission follows arrival order."""
    budget = budget_mb << 20
    # a pool holds every operand drawn here (m, n <= 3000, rows padded to
    # 16 bytes): a longer operand is refused by design (gbserve.h)
    P = 1 << 24
    with gb.Engine(budget, streams=streams, max_inflight=max_inflight, max_step_requests=max_step,
                   host_only=True, sim_bytes_per_ns=500.0, pool_elems=P, chunk_bytes=chunk) as e:
        t0 = e.now_ns() + 2_000_000
        ok = []
        for i, (op, m, n, dt, pool) in enumerate(reqs):
            st_ = e.submit(i, op, m, n, 1.0, i, arrival_ns=t0 + dt, pool=pool)
            size = gb.request_bytes(op, m, n, pool=pool)
            assert st_ == (gb.GB_OK if size <= budget else gb.GB_ERR_BUDGET)
            if st_ == gb.GB_OK:
                ok.append(i)
        assert e.drain(60000) == gb.GB_OK
        done = e.poll()
        stats = e.stats()
    assert sorted(c["id"] for c in done) == ok
    assert stats["bytes_peak"] <= budget and stats["bytes_in_use"] == 0
    assert stats["inflight_peak"] <= max_inflight and stats["steps_inflight_peak"] <= streams
    per_step = {}
    for c in done:
        assert c["arrival_ns"] <= c["admitted_ns"] <= c["launched_ns"] <= c["done_ns"]
        per_step[c["step"]] = per_step.get(c["step"], 0) + 1
    if chunk == 0:
        assert max(per_step.values(), default=0) <= max_step
    # admission follows arrival order (ties by submission)
    by_arrival = sorted(done, key=lambda c: (c["arrival_ns"], c["id"]))
    adm = [c["admitted_ns"] for c in by_arrival]
    assert adm == sorted(adm)


@settings(max_examples=200, deadline=None)
@given(st.sampled_from([gb.F32, gb.F64]), st.sampled_from([gb.ROW_MAJOR, gb.COL_MAJOR]),
       st.integers(-3, 1 << 40), st.integers(-3, 1 << 40))
def test_workspace_follows_its_contract(dt, layout, m, n):
    """gb_workspace_bytes is a pure function of its arguments, 0 for invalid
    ones, and DOT ignores m and the layout."""
    a = gb.gb_workspace_bytes(gb.OP_GEMV, dt, layout, m, n)
    assert a == gb.gb_workspace_bytes(gb.OP_GEMV, dt, layout, m, n)
    if m < 0 or n < 0:
        assert a == 0
    d = gb.gb_workspace_bytes(gb.OP_DOT, dt, layout, m, n)
    assert d == gb.gb_workspace_bytes(gb.OP_DOT, dt, 1 - layout, 7, n)
    if n < 0:
        assert d == 0
    assert gb.gb_workspace_bytes(gb.OP_GEMV, 9, layout, m, n) == 0
    assert gb.gb_workspace_bytes(gb.OP_GEMV, dt, 9, abs(m), abs(n)) == 0
