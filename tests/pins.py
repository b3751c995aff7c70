"""Pins for the CPU oracle: facts fixed by the paper's definitions and by
mathematics, not by the oracle itself.

Each ``pin_*`` function takes an ``oracle.Oracle`` and raises AssertionError
when the oracle disagrees with the pinned fact.  ``tests/test_oracle_pins.py``
runs them against the oracle; ``tests/test_oracle_mutants.py`` runs them
against deliberately broken copies of the oracle, to show that a plausible
mistake (a dropped term, a wrong sign, a transposed index) fails at least
one of them.

What pins what (Singh & Bassoy, Sec. 3.1 Defs. DOT / GEM / GEMV):
  * closed forms: all-ones A and x give c0 + alpha*n; the identity gives
    c0 + x; dot(1, 1) = n; dot(1, (-1)^p) = n mod 2; GER with y = e_k touches
    column k only;
  * integer-valued inputs, where every summation order is exact, against
    numpy's int64 matrix product (an independent library routine);
  * brute force on tiny shapes against exact rational arithmetic
    (``fractions``), including the rounding of GER to the nearest f32/f64;
  * invariants: row-major storage of A equals column-major storage of A^T,
    results do not depend on the thread count, alpha = 0 reads nothing.
"""
from __future__ import annotations

from fractions import Fraction as _Fraction

import numpy as np

import synth

ROW, COL = 0, 1


def Fraction(v, d=None):
    """Exact rational of a number (numpy scalars included)."""
    if d is not None:
        return _Fraction(v, d)
    if isinstance(v, (_Fraction, int)):
        return _Fraction(v)
    return _Fraction(float(v))
U64 = 2.0 ** -53
U32 = 2.0 ** -24


def store(M: np.ndarray, layout: int, ld: int, fill=np.nan) -> np.ndarray:
    """Flat storage of logical matrix M (m x n) with leading dimension ld;
    padding elements are set to ``fill`` (NaN by default: a read of padding
    poisons the result)."""
    m, n = M.shape
    if layout == ROW:
        buf = np.full(max((m - 1) * ld + n, 0) if m and n else 0, fill, dtype=M.dtype)
        for i in range(m):
            buf[i * ld:i * ld + n] = M[i]
    else:
        buf = np.full(max((n - 1) * ld + m, 0) if m and n else 0, fill, dtype=M.dtype)
        for j in range(n):
            buf[j * ld:j * ld + m] = M[:, j]
    return buf


def load(buf: np.ndarray, layout: int, m: int, n: int, ld: int) -> np.ndarray:
    out = np.empty((m, n), dtype=buf.dtype)
    for i in range(m):
        for j in range(n):
            out[i, j] = buf[i * ld + j] if layout == ROW else buf[i + j * ld]
    return out


def round_f32(q: Fraction) -> float:
    """Round an exact rational to the nearest float32 (ties to even)."""
    if q == 0:
        return 0.0
    sign = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    quantum_exp = max(e - 23, -149)
    scaled = a / Fraction(2) ** quantum_exp
    k = scaled.numerator // scaled.denominator
    rem = scaled - k
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and k % 2 == 1):
        k += 1
    return sign * float(Fraction(k) * Fraction(2) ** quantum_exp)


def _ld(layout, m, n, pad):
    return (n if layout == ROW else m) + pad


# --------------------------------------------------------------- GEMV ----

def pin_gemv_all_ones(O):
    for layout in (ROW, COL):
        for (m, n, pad) in ((37, 53, 3), (1, 1, 0), (64, 1, 1), (5, 300, 0)):
            ld = _ld(layout, m, n, pad)
            A = store(np.ones((m, n)), layout, ld)
            x = np.ones(n)
            c0 = synth.uniform(m, 11, 1)
            alpha = 0.75
            want = np.array([float(Fraction(c) + Fraction(alpha) * n) for c in c0])
            for acc in (False, True):
                got = O.gemv(layout, m, n, alpha, A, ld, x, c0, acc=acc)
                assert np.array_equal(got, want), (layout, m, n, acc)


def pin_gemv_identity(O):
    for layout in (ROW, COL):
        n = 29
        ld = _ld(layout, n, n, 2)
        A = store(np.eye(n), layout, ld)
        x = synth.uniform(n, 12, 1)
        c0 = synth.uniform(n, 12, 2)
        want = np.array([float(Fraction(c) + Fraction(v)) for c, v in zip(c0, x)])
        for acc in (False, True):
            got = O.gemv(layout, n, n, 1.0, A, ld, x, c0, acc=acc)
            assert np.array_equal(got, want), (layout, acc)


def pin_gemv_integer_exact(O):
    for layout in (ROW, COL):
        for (m, n, pad, alpha) in ((48, 77, 5, 2.0), (130, 9, 0, -3.0), (3, 1000, 1, 1.0)):
            ld = _ld(layout, m, n, pad)
            Ai = synth.integers(m * n, 21, 1, -8, 8, np.int64).reshape(m, n)
            xi = synth.integers(n, 21, 2, -8, 8, np.int64)
            ci = synth.integers(m, 21, 3, -8, 8, np.int64)
            want = (ci + int(alpha) * (Ai @ xi)).astype(np.float64)
            A = store(Ai.astype(np.float64), layout, ld)
            for acc in (False, True):
                got = O.gemv(layout, m, n, alpha, A, ld, xi.astype(np.float64),
                             ci.astype(np.float64), acc=acc)
                assert np.array_equal(got, want), (layout, m, n, acc)


def pin_gemv_bruteforce_exact(O):
    for layout in (ROW, COL):
        for m in (0, 1, 2, 3, 5):
            for n in (0, 1, 2, 4, 7):
                for pad in (0, 1, 3):
                    ld = max(_ld(layout, m, n, pad), 1)
                    seed = 1000 + 100 * m + 10 * n + pad
                    M = synth.uniform(m * n, seed, 1).reshape(m, n)
                    x = synth.uniform(n, seed, 2)
                    c0 = synth.uniform(m, seed, 3)
                    alpha = float(synth.uniform(1, seed, 4)[0]) * 3.0
                    A = store(M, layout, ld)
                    exact = [Fraction(c0[i]) + Fraction(alpha) * sum(
                        (Fraction(M[i, j]) * Fraction(x[j]) for j in range(n)), Fraction(0))
                        for i in range(m)]
                    scale = [abs(Fraction(c0[i])) + abs(Fraction(alpha)) * sum(
                        (abs(Fraction(M[i, j]) * Fraction(x[j])) for j in range(n)), Fraction(0))
                        for i in range(m)]
                    acc = O.gemv(layout, m, n, alpha, A, ld, x, c0, acc=True)
                    plain = O.gemv(layout, m, n, alpha, A, ld, x, c0, acc=False)
                    sc = O.gemv_scale(layout, m, n, alpha, A, ld, x, c0)
                    g = (n + 3) * U64 / (1 - (n + 3) * U64)
                    for i in range(m):
                        e = abs(Fraction(acc[i]) - exact[i])
                        assert e <= 2 * U64 * abs(exact[i]) + 1e-30 * scale[i], (layout, m, n, i)
                        e = abs(Fraction(plain[i]) - exact[i])
                        assert e <= g * scale[i], (layout, m, n, i)
                        assert abs(Fraction(sc[i]) - scale[i]) <= g * scale[i]


def pin_gemv_layout_equivalence(O):
    m, n = 23, 41
    M = synth.uniform(m * n, 31, 1).reshape(m, n)
    x = synth.uniform(n, 31, 2)
    c0 = synth.uniform(m, 31, 3)
    row = store(M, ROW, n)
    col_as_transpose = np.ascontiguousarray(M.T).ravel()  # A^T row-major == A col-major
    for acc in (False, True):
        a = O.gemv(ROW, m, n, 0.5, row, n, x, c0, acc=acc)
        b = O.gemv(COL, m, n, 0.5, col_as_transpose, m, x, c0, acc=acc)
        assert np.array_equal(a, b)


def pin_gemv_alpha_zero(O):
    m, n = 4, 6
    A = np.full(m * n, np.nan)
    c0 = synth.uniform(m, 41, 1)
    for acc in (False, True):
        got = O.gemv(ROW, m, n, 0.0, A, n, np.full(n, np.nan), c0, acc=acc)
        assert np.array_equal(got, c0)


def pin_gemv_plain_vs_acc(O):
    m, n = 16, 20000
    M = synth.uniform(m * n, 51, 1)
    x = synth.uniform(n, 51, 2)
    c0 = synth.uniform(m, 51, 3)
    a = O.gemv(ROW, m, n, 1.0, M, n, x, c0, acc=True)
    p = O.gemv(ROW, m, n, 1.0, M, n, x, c0, acc=False)
    sc = O.gemv_scale(ROW, m, n, 1.0, M, n, x, c0)
    g = (n + 2) * U64 / (1 - (n + 2) * U64)
    assert np.all(np.abs(a - p) <= g * sc)
    # the two really are different sums (plain is not secretly compensated)
    assert np.any(a != p)


# ---------------------------------------------------------------- DOT ----

def pin_dot_closed_forms(O):
    for n in (0, 1, 2, 7, 1000, 65536 + 3):
        ones = np.ones(n)
        alt = np.array([(-1.0) ** p for p in range(n)])
        for acc in (False, True):
            assert O.dot(n, ones, ones, 0.25, acc=acc) == 0.25 + n
            assert O.dot(n, ones, alt, 0.25, acc=acc) == 0.25 + (n % 2)


def pin_dot_bruteforce_exact(O):
    for n in (1, 2, 3, 10, 33):
        x = synth.uniform(n, 61 + n, 1)
        y = synth.uniform(n, 61 + n, 2)
        a0 = float(synth.uniform(1, 61 + n, 3)[0])
        exact = Fraction(a0) + sum((Fraction(x[p]) * Fraction(y[p]) for p in range(n)), Fraction(0))
        scale = abs(Fraction(a0)) + sum((abs(Fraction(x[p]) * Fraction(y[p])) for p in range(n)),
                                        Fraction(0))
        acc = O.dot(n, x, y, a0, acc=True)
        plain = O.dot(n, x, y, a0, acc=False)
        assert abs(Fraction(acc) - exact) <= 2 * U64 * abs(exact) + 1e-30 * scale
        g = (n + 1) * U64 / (1 - (n + 1) * U64)
        assert abs(Fraction(plain) - exact) <= g * scale
        assert abs(Fraction(O.dot_scale(n, x, y, a0)) - scale) <= g * scale


def pin_dot_multichunk_exact(O):
    # several of the oracle's 2^16-element chunks plus a ragged tail; the exact
    # value comes from integer arithmetic on the 52-bit fixed-point inputs
    n = 3 * 65536 + 7
    x = synth.uniform(n, 71, 1)
    y = synth.uniform(n, 71, 2)
    xi = [int(v) for v in np.rint(x * 2.0 ** 52)]
    yi = [int(v) for v in np.rint(y * 2.0 ** 52)]
    assert all(float(a) * 2.0 ** -52 == b for a, b in zip(xi[:100], x[:100]))
    s = sum(a * b for a, b in zip(xi, yi))
    exact = Fraction(s, 2 ** 104) + Fraction(0.5)
    acc = O.dot(n, x, y, 0.5, acc=True)
    assert abs(Fraction(acc) - exact) <= U64 * abs(exact) * 1.0000001 + Fraction(1, 2 ** 90)


def pin_dot_integer_exact(O):
    n = 200003
    xi = synth.integers(n, 81, 1, -1, 1, np.int64)
    yi = synth.integers(n, 81, 2, -1, 1, np.int64)
    want = float(int(xi @ yi) + 3)
    for acc in (False, True):
        assert O.dot(n, xi.astype(float), yi.astype(float), 3.0, acc=acc) == want


# ---------------------------------------------------------------- GER ----

def pin_ger_unit_vector(O):
    for layout in (ROW, COL):
        for dt in (np.float64, np.float32):
            m, n, k = 13, 9, 4
            ld = _ld(layout, m, n, 2)
            C0 = synth.uniform(m * n, 91, 1, dt).reshape(m, n)
            Cbuf = store(C0, layout, ld)
            x = synth.uniform(m, 91, 2, dt)
            y = np.zeros(n, dtype=dt)
            y[k] = 1
            alpha = dt(1.5)
            out = O.ger(layout, m, n, alpha, x, y, Cbuf, ld)
            got = load(out, layout, m, n, ld)
            rnd = float if dt == np.float64 else round_f32
            for i in range(m):
                for j in range(n):
                    if j == k:
                        assert got[i, j] == rnd(Fraction(C0[i, j]) + Fraction(x[i]) * Fraction(alpha))
                    else:
                        assert got[i, j] == C0[i, j]
            # padding untouched (still NaN)
            mask = np.ones(out.size, bool)
            for i in range(m):
                for j in range(n):
                    mask[i * ld + j if layout == ROW else i + j * ld] = False
            assert np.all(np.isnan(out[mask]))


def pin_ger_bruteforce_rounding(O):
    for layout in (ROW, COL):
        for dt in (np.float64, np.float32):
            for (m, n) in ((1, 1), (3, 5), (6, 2), (0, 4), (4, 0)):
                ld = max(_ld(layout, m, n, 1), 1)
                C0 = synth.uniform(m * n, 101, 1, dt).reshape(m, n)
                x = synth.uniform(m, 101, 2, dt)
                y = synth.uniform(n, 101, 3, dt)
                alpha = dt(-0.7)
                Cbuf = store(C0, layout, ld)
                got = load(O.ger(layout, m, n, alpha, x, y, Cbuf, ld), layout, m, n, ld)
                rnd = float if dt == np.float64 else round_f32
                for i in range(m):
                    for j in range(n):
                        t = rnd(Fraction(alpha) * Fraction(y[j]))
                        want = rnd(Fraction(C0[i, j]) + Fraction(x[i]) * Fraction(t))
                        assert got[i, j] == want, (layout, dt, m, n, i, j)


def pin_ger_alpha_zero(O):
    C = synth.uniform(12, 111, 1)
    out = O.ger(ROW, 3, 4, 0.0, np.full(3, np.nan), np.full(4, np.nan), C, 4)
    assert np.array_equal(out, C)


# ----------------------------------------------------------- threading ---

def pin_thread_count_independent(O):
    t0 = O.threads()
    m, n = 97, 3001
    M = synth.uniform(m * n, 121, 1)
    x = synth.uniform(n, 121, 2)
    c0 = synth.uniform(m, 121, 3)
    nd = 5 * 65536 + 11
    dx = synth.uniform(nd, 121, 4)
    dy = synth.uniform(nd, 121, 5)
    res = []
    for t in (1, max(t0, 2)):
        O.set_threads(t)
        res.append((O.gemv(COL, m, n, 1.25, M, m, x, c0), O.dot(nd, dx, dy, 0.0),
                    O.ger(ROW, m, n, 0.5, c0, x, M, n)))
    O.set_threads(t0)
    assert np.array_equal(res[0][0], res[1][0])
    assert res[0][1] == res[1][1]
    assert np.array_equal(res[0][2], res[1][2])




# ----------------------------------------------- reduced-precision A ----
# Facts of the formats: BF16 is the top half of a binary32 with
# round-to-nearest-even on the dropped half; E4M3 (OCP FP8) has bias 7, 3
# mantissa bits, largest finite 448 = 0x7E, smallest normal 2^-6 = 0x08,
# smallest subnormal 2^-9 = 0x01, NaN 0x7F, and saturating encoding.

def pin_bf16_roundtrip_and_ties(O):
    codes = np.arange(65536, dtype=np.uint32)
    vals = (codes << np.uint32(16)).view(np.float32)
    finite = np.isfinite(vals)
    assert np.array_equal(O.bf16_encode(vals[finite]), codes[finite].astype(np.uint16))
    # halfway between code k and k+1 (same sign, k not the largest finite):
    # ties go to the even code; one unit above or below goes to the nearer
    k = codes[finite & (codes % 0x8000 != 0x7F7F) & (codes % 0x8000 < 0x7F7F)]
    half = ((k << np.uint32(16)) | np.uint32(0x8000)).view(np.float32)
    want = np.where(k % 2 == 0, k, k + 1).astype(np.uint16)
    assert np.array_equal(O.bf16_encode(half), want)
    above = ((k << np.uint32(16)) | np.uint32(0x8001)).view(np.float32)
    below = ((k << np.uint32(16)) | np.uint32(0x7FFF)).view(np.float32)
    assert np.array_equal(O.bf16_encode(above), (k + 1).astype(np.uint16))
    assert np.array_equal(O.bf16_encode(below), k.astype(np.uint16))
    assert O.bf16_encode([1.0, -2.0, np.pi, np.float32(3.4028235e38)]).tolist() == [0x3F80, 0xC000, 0x4049, 0x7F80]


def pin_e4m3_known_values(O):
    enc = O.e4m3_encode([448.0, 2.0 ** -6, 2.0 ** -9, 1.0, -0.0, 0.0, 0.0625, 240.0, -1.75])
    assert enc.tolist() == [0x7E, 0x08, 0x01, 0x38, 0x80, 0x00, 0x18, 0x77, 0xBE]
    dec = O.e4m3_decode(np.arange(256, dtype=np.uint8))
    assert np.isnan(dec[0x7F]) and np.isnan(dec[0xFF])
    pos = dec[:0x7F]
    assert np.all(np.diff(pos) > 0)                 # strictly increasing codes 0..0x7E
    assert pos[-1] == 448.0 and pos[1] == 2.0 ** -9 and pos[8] == 2.0 ** -6
    assert np.array_equal(dec[0x80:0xFF], -pos)     # sign-magnitude
    # spacing is constant inside a binade: 2^(e-3) for e >= -6, 2^-9 below
    for e in range(-6, 9):
        lo, hi = 2.0 ** e, min(2.0 ** (e + 1), 448.0)
        inside = pos[(pos >= lo) & (pos <= hi)]
        assert np.allclose(np.diff(inside), 2.0 ** (e - 3))


def pin_e4m3_roundtrip_ties_saturation(O):
    codes = np.array([c for c in range(256) if c not in (0x7F, 0xFF)], dtype=np.uint8)
    assert np.array_equal(O.e4m3_encode(O.e4m3_decode(codes)), codes)
    pos = O.e4m3_decode(np.arange(0x7F, dtype=np.uint8))
    mid = (pos[:-1] + pos[1:]) / 2                   # exact in binary64
    k = np.arange(0x7E)
    assert np.array_equal(O.e4m3_encode(mid), np.where(k % 2 == 0, k, k + 1).astype(np.uint8))
    assert np.array_equal(O.e4m3_encode(np.nextafter(mid, 0)), k.astype(np.uint8))
    assert np.array_equal(O.e4m3_encode(np.nextafter(mid, 1e9)), (k + 1).astype(np.uint8))
    assert O.e4m3_encode([448.0001, 464.0, 470.0, 1e30, np.inf, -1e30]).tolist() == [0x7E, 0x7E, 0x7E, 0x7E, 0x7E, 0xFE]
    assert O.e4m3_encode([2.0 ** -10, 2.0 ** -10 * 1.0001, 3 * 2.0 ** -10]).tolist() == [0, 1, 2]


def pin_quantize_e4m3_rows(O):
    m, n = 6, 40
    A = synth.uniform(m * n, 131, 1, np.float32).reshape(m, n)
    A[0] *= 448.0 / np.abs(A[0]).max()              # amax 448: scale exactly 1
    A[1] = 0.0                                      # all-zero row: scale 0, codes 0
    A[2] *= 1e-3
    A[3] *= 1e3
    Q, s = O.quantize_e4m3_rows(m, n, A.ravel(), n)
    Q = Q.reshape(m, n)
    assert s[0] == 1.0 and np.array_equal(Q[0], O.e4m3_encode(A[0].astype(np.float64)))
    assert s[1] == 0.0 and not Q[1].any()
    for i in (2, 3, 4, 5):
        amax = np.abs(A[i]).max()
        assert s[i] == np.float32(amax) / np.float32(448.0)
        assert np.abs(O.e4m3_decode(Q[i])).max() == 448.0      # the largest element maps to 448
        deq = O.e4m3_decode(Q[i]) * np.float64(s[i])
        # half a unit of the 3-bit mantissa, or the subnormal floor
        assert np.all(np.abs(deq - A[i]) <= np.maximum(2.0 ** -4 * np.abs(A[i]), s[i] * 2.0 ** -10) * 1.0000001)


ALL_PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
