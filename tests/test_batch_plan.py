"""Host planner of the batched FP32 GEMV (gb_sgemv_batch_plan): a pure host
function of the C ABI, so it is tested here without a GPU.  Device pointers
are fake addresses: the planner stores them and checks overlaps, it never
dereferences them.

Checked: every row of every active problem lies in exactly one tile, the
tiles of a problem are consecutive and ordered, a tile holds a multiple of
the block's row groups (except a problem's last), the cost prefix is
increasing and ends at the total, the tuning entry is the one of the
problem's bucket ceil(log2 n), the plan of a problem is the same alone and
in a mix, and the argument checks."""
import numpy as np
import pytest

import paper_2108_02025_gb300 as gb
import synth

HEADER = np.dtype([("magic", "<u4"), ("version", "<u4"), ("count", "<i8"), ("tiles", "<i8"),
                   ("total", "<i8"), ("off_problems", "<i8"), ("off_tiles", "<i8"),
                   ("off_prefix", "<i8"), ("reserved", "<i8")])
PROBLEM = np.dtype([("A", "<u8"), ("x", "<u8"), ("c", "<u8"), ("lda", "<i8"), ("m", "<i4"),
                    ("n", "<i4"), ("alpha", "<f4"), ("vec", "u1"), ("kind", "u1"), ("pad", "<u2")])
TILE = np.dtype([("A", "<u8"), ("x", "<u8"), ("c", "<u8"), ("lda", "<i8"), ("rows", "<i4"),
                 ("n", "<i4"), ("alpha", "<f4"), ("lpr_log2", "u1"), ("u_log2", "u1"), ("vec", "u1"),
                 ("kind", "u1")])


def log_uniform(count, seed, stream, lo, hi):
    u = (synth.uniform(count, seed, stream) + 1.0) / 2.0
    return np.round(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))).astype(np.int64)


class FakeBatch:
    """Problems laid out at fake, disjoint, 256-byte aligned addresses."""

    def __init__(self, m, n, alpha=None, pad=3, base=1 << 40):
        self.count = len(m)
        self.m = np.asarray(m, np.int64)
        self.n = np.asarray(n, np.int64)
        self.lda = np.maximum(self.n + pad, 1).astype(np.int64)
        self.alpha = np.ones(self.count, np.float32) if alpha is None else np.asarray(alpha, np.float32)
        self.A = np.zeros(self.count, np.uint64)
        self.x = np.zeros(self.count, np.uint64)
        self.c = np.zeros(self.count, np.uint64)
        addr = base
        for p in range(self.count):
            for name, nbytes in (("A", 4 * int(self.m[p]) * int(self.lda[p])), ("x", 4 * int(self.n[p])),
                                 ("c", 4 * int(self.m[p]))):
                getattr(self, name)[p] = addr
                addr += (nbytes + 255) // 256 * 256 + 256

    def plan(self, table=None):
        nb = gb.gb_sgemv_batch_plan_bytes(self.count, self.m, self.n, self.alpha, table)
        assert nb > 0
        buf = aligned_buffer(nb)
        st = gb.gb_sgemv_batch_plan(self.count, self.m, self.n, self.lda, self.alpha, self.A, self.x,
                                    self.c, table, buf, nb)
        return st, buf

    def call(self, table=None, plan=None, nbytes=None, **override):
        args = {k: getattr(self, k) for k in ("m", "n", "lda", "alpha", "A", "x", "c")}
        args.update(override)
        if plan is None:
            nbytes = 1 << 20
            plan = aligned_buffer(nbytes)
        return gb.gb_sgemv_batch_plan(self.count, args["m"], args["n"], args["lda"], args["alpha"],
                                      args["A"], args["x"], args["c"], table, plan, nbytes)


def aligned_buffer(nbytes):
    raw = np.zeros(nbytes + 16, np.uint8)
    off = (-raw.ctypes.data) % 16
    return raw[off:off + nbytes]


def decode(buf):
    """Header, problems, tiles and cost prefix of a plan; each tile gets the
    problem p it belongs to (the one whose c holds its output) and its first
    row row0."""
    h = np.frombuffer(buf[:HEADER.itemsize].tobytes(), HEADER)[0]
    probs = np.frombuffer(buf[h["off_problems"]:h["off_problems"] + h["count"] * PROBLEM.itemsize].tobytes(),
                          PROBLEM)
    raw = np.frombuffer(buf[h["off_tiles"]:h["off_tiles"] + h["tiles"] * TILE.itemsize].tobytes(), TILE)
    prefix = np.frombuffer(buf[h["off_prefix"]:h["off_prefix"] + (h["tiles"] + 1) * 8].tobytes(), "<i8")
    tiles = np.zeros(raw.size, dtype=TILE.descr + [("p", "<i8"), ("row0", "<i8")])
    for f in TILE.names:
        tiles[f] = raw[f]
    if raw.size:
        order = np.argsort(probs["c"])
        k = np.searchsorted(probs["c"][order], raw["c"], side="right") - 1
        tiles["p"] = order[k]
        tiles["row0"] = (raw["c"] - probs["c"][tiles["p"]]) // 4
    return h, probs, tiles, prefix


def bucket(n):
    b = 0
    while b < gb.BATCH_BUCKETS - 1 and (1 << b) < n:
        b += 1
    return b


def check_plan(fb, buf, table):
    h, probs, tiles, prefix = decode(buf)
    assert h["magic"] == 0x47425042 and h["count"] == fb.count
    assert h["tiles"] == gb.gb_sgemv_batch_tiles(buf)
    assert prefix[0] == 0 and prefix[-1] == h["total"]
    assert np.all(np.diff(prefix) > 0)
    for p in range(fb.count):
        pr = probs[p]
        assert (pr["m"], pr["n"], pr["lda"]) == (fb.m[p], fb.n[p], fb.lda[p])
        assert (pr["A"], pr["x"], pr["c"]) == (fb.A[p], fb.x[p], fb.c[p])
        mine = tiles[tiles["p"] == p]
        idx = np.nonzero(tiles["p"] == p)[0]
        active = fb.m[p] > 0 and fb.n[p] > 0 and fb.alpha[p] != 0
        if not active:
            assert mine.size == 0
            continue
        assert np.all(np.diff(idx) == 1), "tiles of a problem are consecutive"
        starts = np.concatenate([[0], np.cumsum(mine["rows"])[:-1]])
        assert np.array_equal(mine["row0"], starts) and mine["rows"].sum() == fb.m[p]
        a_row0 = fb.A[p] + np.uint64(4) * mine["row0"].astype(np.uint64) * np.uint64(fb.lda[p])
        assert np.array_equal(mine["A"], a_row0)
        assert np.all(mine["x"] == fb.x[p]) and np.all(mine["lda"] == fb.lda[p])
        assert np.all(mine["n"] == fb.n[p]) and np.all(mine["alpha"] == fb.alpha[p])
        assert np.all(mine["vec"] == pr["vec"]) and np.all(mine["kind"] == 0) and pr["kind"] == 0
        e = table[bucket(int(fb.n[p]))]
        assert np.all(mine["lpr_log2"] == int(np.log2(e.lanes_per_row)))
        assert np.all(mine["u_log2"] == int(np.log2(e.packs_per_iter)))
        groups = 256 // e.lanes_per_row
        assert np.all(mine["rows"][:-1] % groups == 0) and np.all(mine["rows"] > 0)
        assert np.all(mine["rows"][:-1] == mine["rows"][0])
    return h, probs, tiles, prefix


def test_default_table():
    t = gb.tuning_table()
    for b in range(gb.BATCH_BUCKETS):
        e = t[b]
        assert e.lanes_per_row in (1, 2, 4, 8, 16, 32)
        assert e.packs_per_iter in (1, 2, 4)
        assert e.tile_bytes >= 4096 and e.reserved == 0
    assert t[13].lanes_per_row == 32  # n up to 8192: 2048 packs per row


def test_buckets():
    assert [bucket(n) for n in (1, 2, 3, 32, 33, 64, 8192, 8193)] == [0, 1, 2, 5, 6, 6, 13, 14]


def test_random_batch_covers_every_row():
    count = 300
    m = log_uniform(count, 0, 1, 32, 8192)
    n = log_uniform(count, 0, 2, 32, 8192)
    fb = FakeBatch(m, n)
    table = gb.tuning_table()
    st, buf = fb.plan(table)
    assert st == gb.GB_OK
    h, probs, tiles, prefix = check_plan(fb, buf, table)
    # cost per tile: rows * (4n + 8) + 4n + 256
    pn = tiles["n"].astype(np.int64)
    cost = tiles["rows"].astype(np.int64) * (4 * pn + 8) + 4 * pn + 256
    assert np.array_equal(np.diff(prefix), cost)
    # aligned fake addresses and lda = n + 3: only n = 1 (mod 4) rows are 16-byte multiples
    assert np.array_equal(probs["vec"].astype(bool), (fb.lda % 4) == 0)


def test_null_table_is_default_and_custom_table_is_used():
    fb = FakeBatch([100, 5000, 7], [40, 3000, 9000])
    st, buf = fb.plan(None)
    assert st == gb.GB_OK
    check_plan(fb, buf, gb.tuning_table())
    custom = gb.tuning_table({b: (4, 1, 8192) for b in range(gb.BATCH_BUCKETS)})
    st, buf = fb.plan(custom)
    assert st == gb.GB_OK
    h, probs, tiles, prefix = check_plan(fb, buf, custom)
    assert np.all(tiles["lpr_log2"] == 2) and np.all(tiles["u_log2"] == 0)


def test_inactive_problems_have_no_tiles_and_may_be_null():
    fb = FakeBatch([0, 50, 60, 70], [10, 0, 20, 30], alpha=[1, 1, 0, 2])
    for name in ("A", "x", "c"):
        getattr(fb, name)[:3] = 0
    st, buf = fb.plan(gb.tuning_table())
    assert st == gb.GB_OK
    h, probs, tiles, prefix = check_plan(fb, buf, gb.tuning_table())
    assert set(tiles["p"].tolist()) == {3}


def test_empty_batch():
    fb = FakeBatch([], [])
    st, buf = fb.plan(None)
    assert st == gb.GB_OK
    h, _, tiles, prefix = decode(buf)
    assert h["tiles"] == 0 and prefix.tolist() == [0]


def test_same_problem_same_tiles_alone_and_in_a_mix():
    m = log_uniform(50, 3, 1, 32, 8192)
    n = log_uniform(50, 3, 2, 32, 8192)
    mix = FakeBatch(m, n)
    _, buf = mix.plan(None)
    _, _, tiles_mix, _ = decode(buf)
    for p in (0, 17, 49):
        alone = FakeBatch(m[p:p + 1], n[p:p + 1])
        _, b1 = alone.plan(None)
        _, _, t1, _ = decode(b1)
        tm = tiles_mix[tiles_mix["p"] == p]
        for f in ("row0", "rows", "lpr_log2", "u_log2"):
            assert np.array_equal(t1[f], tm[f])


def test_argument_checks():
    fb = FakeBatch([10, 20], [30, 40])
    assert fb.call(m=np.array([10, -1], np.int64)) == -2
    assert fb.call(n=np.array([-5, 40], np.int64)) == -3
    assert fb.call(m=np.array([10, 2 ** 31], np.int64)) == -2
    assert fb.call(lda=np.array([29, 43], np.int64)) == -4
    assert fb.call(A=np.array([0, fb.A[1]], np.uint64)) == -6
    assert fb.call(x=np.array([fb.x[0], 0], np.uint64)) == -7
    assert fb.call(c=np.array([0, fb.c[1]], np.uint64)) == -8
    # c of problem 1 overlapping c of problem 0, then A of problem 0
    assert fb.call(c=np.array([fb.c[0], fb.c[0] + 8], np.uint64)) == -8
    assert fb.call(c=np.array([fb.c[0], fb.A[0] + 4 * 50], np.uint64)) == -8
    # c of problem 0 overlapping its own x
    assert fb.call(c=np.array([fb.x[0], fb.c[1]], np.uint64)) == -8
    bad = gb.tuning_table({7: (3, 1, 65536)})
    assert fb.call(table=bad) == -9
    assert gb.gb_sgemv_batch_plan_bytes(2, fb.m, fb.n, fb.alpha, bad) == 0
    assert fb.call(table=gb.tuning_table({7: (4, 8, 65536)})) == -9
    assert fb.call(table=gb.tuning_table({7: (4, 1, 100)})) == -9
    nb = gb.gb_sgemv_batch_plan_bytes(2, fb.m, fb.n, fb.alpha, None)
    buf = aligned_buffer(nb + 16)
    assert fb.call(plan=buf[1:], nbytes=nb) == -10
    assert fb.call(plan=buf, nbytes=nb - 16) == -11
    assert fb.call(plan=buf, nbytes=nb) == gb.GB_OK
    assert gb.gb_sgemv_batch_plan(-1, None, None, None, None, None, None, None, None, buf, nb) == -1
    assert gb.gb_sgemv_batch_plan_bytes(-1, None, None, None, None) == 0


def test_launch_rejects_a_non_plan_without_touching_the_device():
    junk = aligned_buffer(64)
    assert gb.gb_sgemv_batch(junk, 1 << 40, 0) == -1
    assert gb.gb_sgemv_batch_tiles(junk) == -1
    fb = FakeBatch([10], [30])
    st, buf = fb.plan(None)
    assert st == gb.GB_OK
    assert gb.gb_sgemv_batch(buf, None, 0) == -2
    assert gb.gb_sgemv_batch(buf, (1 << 40) + 4, 0) == -2


def items_of(specs, base=1 << 41):
    """gb_batch_item array from (kind, m, n, lda, alpha) at fake disjoint addresses."""
    arr = (gb.BatchItem * max(1, len(specs)))()
    addr = base
    for i, (kind, m, n, lda, alpha) in enumerate(specs):
        eb = 2 if kind == gb.BATCH_GEMV_BF16 else 4
        a = addr
        addr += (m * lda * eb + 255) // 256 * 256 + 256
        xx = addr
        addr += (n * 4 + 255) // 256 * 256 + 256
        cc = addr
        addr += (m * 4 + 255) // 256 * 256 + 256
        arr[i] = gb.BatchItem(kind, 0, m, n, lda, alpha, 0, a, xx, cc)
    return arr


def test_mixed_items_plan():
    specs = [(gb.BATCH_GEMV_F32, 100, 40, 40, 1.0), (gb.BATCH_GEMV_BF16, 300, 1000, 1000, 0.5),
             (gb.BATCH_GEMV_BF16, 7, 30, 30, 1.0), (gb.BATCH_GER_F32, 50, 64, 64, -1.0),
             (gb.BATCH_GER_F32, 9, 10, 11, 2.0), (gb.BATCH_GEMV_F32, 5, 5, 5, 0.0)]
    arr = items_of(specs)
    table = gb.tuning_table()
    nb = gb.gb_batch_plan_bytes(len(specs), arr, table)
    buf = aligned_buffer(nb)
    assert gb.gb_batch_plan(len(specs), arr, table, buf, nb) == gb.GB_OK
    h, probs, raw, prefix = decode_raw(buf)
    assert list(probs["kind"]) == [s[0] for s in specs]
    # 16-byte path: lda * element bytes a multiple of 16 (aligned fake addresses)
    assert list(probs["vec"]) == [1, 1, 0, 1, 0, 0]
    kinds = []
    for p, (kind, m, n, lda, alpha) in enumerate(specs):
        inside = (raw["c"] >= np.uint64(arr[p].c)) & (raw["c"] < np.uint64(arr[p].c + 4 * m))
        mine = raw[inside]
        if alpha == 0:
            assert mine.size == 0
            continue
        eb = 2 if kind == gb.BATCH_GEMV_BF16 else 4
        row0 = (mine["c"] - arr[p].c) // 4
        assert np.array_equal(mine["A"], arr[p].A + row0.astype(np.uint64) * np.uint64(lda * eb))
        assert mine["rows"].sum() == m and np.all(mine["kind"] == kind)
        kinds += [kind] * mine.size
        # cost: rows * (row bytes moved + 8) + 4n + 256; GER moves its rows twice
        row = (8 if kind == gb.BATCH_GER_F32 else eb) * n
        idx = np.nonzero(inside)[0]
        assert np.array_equal(np.diff(prefix)[idx], mine["rows"].astype(np.int64) * (row + 8) + 4 * n + 256)
    assert len(kinds) == h["tiles"]


def decode_raw(buf):
    h = np.frombuffer(buf[:HEADER.itemsize].tobytes(), HEADER)[0]
    probs = np.frombuffer(buf[h["off_problems"]:h["off_problems"] + h["count"] * PROBLEM.itemsize].tobytes(),
                          PROBLEM)
    raw = np.frombuffer(buf[h["off_tiles"]:h["off_tiles"] + h["tiles"] * TILE.itemsize].tobytes(), TILE)
    prefix = np.frombuffer(buf[h["off_prefix"]:h["off_prefix"] + (h["tiles"] + 1) * 8].tobytes(), "<i8")
    return h, probs, raw, prefix


def test_mixed_items_argument_checks():
    ok = [(gb.BATCH_GEMV_F32, 10, 10, 12, 1.0), (gb.BATCH_GER_F32, 10, 10, 12, 1.0)]
    arr = items_of(ok)
    nb = gb.gb_batch_plan_bytes(2, arr, None)
    buf = aligned_buffer(nb + 16)
    assert gb.gb_batch_plan(2, arr, None, buf, nb) == gb.GB_OK
    assert gb.gb_batch_plan(-1, arr, None, buf, nb) == -1
    assert gb.gb_batch_plan(2, None, None, buf, nb) == -2
    for field, value in (("kind", 4), ("reserved", 1), ("reserved2", 1), ("m", -1), ("n", -2), ("lda", 9),
                         ("A", 0), ("x", 0), ("c", 0)):
        bad = items_of(ok)
        setattr(bad[1], field, value)
        assert gb.gb_batch_plan(2, bad, None, buf, nb) == -2, field
    # GER: C written, x and y read; GEMV: c written, A and x read
    bad = items_of(ok)
    bad[1].c = bad[0].c          # GER's x is GEMV's output
    assert gb.gb_batch_plan(2, bad, None, buf, nb) == -2
    bad = items_of(ok)
    bad[1].x = bad[1].A + 64     # GER's y inside its own C
    assert gb.gb_batch_plan(2, bad, None, buf, nb) == -2
    bad = items_of(ok)
    bad[0].x = bad[1].x          # two readers of one vector are fine
    assert gb.gb_batch_plan(2, bad, None, buf, nb) == gb.GB_OK
    # GEMVs reading overlapping windows of one resident operand pool (the
    # serving engine's pool requests): shared A and x, distinct outputs
    pool = items_of([(gb.BATCH_GEMV_F32, 10, 10, 12, 1.0)] * 3)
    for k in (1, 2):
        pool[k].A = pool[0].A + 16 * k
        pool[k].x = pool[0].x + 32 * k
    nb3 = gb.gb_batch_plan_bytes(3, pool, None)
    buf3 = aligned_buffer(nb3)
    assert gb.gb_batch_plan(3, pool, None, buf3, nb3) == gb.GB_OK
    pool[2].c = pool[1].c + 4    # two outputs overlapping: refused
    assert gb.gb_batch_plan(3, pool, None, buf3, nb3) == -2
    assert gb.gb_batch_plan(2, arr, gb.tuning_table({4: (4, 3, 65536)}), buf, nb) == -3
    assert gb.gb_batch_plan(2, arr, None, buf[1:], nb) == -4
    assert gb.gb_batch_plan(2, arr, None, buf, nb - 16) == -5
    assert gb.gb_batch_plan_bytes(2, items_of([(7, 1, 1, 1, 1.0)] * 2), None) == 0


def test_dot_items_plan_and_checks():
    """GB_BATCH_DOT_F32: one tile per DOT (m = 1, alpha = 1; alpha 0 skips
    it), its accumulator written, both vectors read; the 16-byte path needs
    only aligned vectors (lda does not matter for one row)."""
    specs = [(gb.BATCH_DOT_F32, 1, 16384, 16384, 1.0), (gb.BATCH_DOT_F32, 1, 37, 37, 1.0),
             (gb.BATCH_DOT_F32, 1, 5, 5, 0.0), (gb.BATCH_GEMV_F32, 100, 40, 40, 1.0)]
    arr = items_of(specs)
    nb = gb.gb_batch_plan_bytes(len(specs), arr, None)
    assert nb > 0
    buf = aligned_buffer(nb)
    assert gb.gb_batch_plan(len(specs), arr, None, buf, nb) == gb.GB_OK
    h, probs, raw, prefix = decode_raw(buf)
    assert list(probs["vec"][:2]) == [1, 1]
    dots = raw[raw["kind"] == gb.BATCH_DOT_F32]
    assert dots.size == 2 and np.all(dots["rows"] == 1)
    assert sorted(dots["n"]) == [37, 16384]
    for field, value in (("m", 2), ("alpha", 0.5), ("alpha", -1.0)):
        bad = items_of(specs)
        setattr(bad[0], field, value)
        assert gb.gb_batch_plan(len(specs), bad, None, buf, nb) == -2, (field, value)
        assert gb.gb_batch_plan_bytes(len(specs), bad, None) == 0, (field, value)
    bad = items_of(specs)
    bad[0].c = bad[0].A + 8      # the accumulator inside the first vector
    assert gb.gb_batch_plan(len(specs), bad, None, buf, nb) == -2
