"""The worst-case bound of the FP64 kernels' FP32-emulated products, checked
in exact rational arithmetic on the CPU (no GPU, no kernel code).

The FP64 GEMV and DOT kernels form part of their products a*x with FP32
instructions: each operand is cut into a 24-bit head and the next 23 bits,
the head product is split exactly by TwoProduct (p + e), the cross terms
are added in FP32 (t), and K products accumulate in an unevaluated FP32 pair
(H, L) updated with TwoSum.  The written bound (Defs. GEMV and DOT of
Sec. 3.1, FP64 gate 1e-12 of the condition-aware denominator) is

    |H + L - sum a_k x_k| <= (u^2 (K(K+1)/2 + 6K + 5) + 2.5 * 2^-45) * sum |a_k x_k|

with u = 2^-24.  Here every FP32 operation is a correctly rounded rational
(round to nearest, ties to even), the sums are exact Fractions, and chains
built to make the pair's errors large must stay inside the bound: for
K = 16 it is 9.2e-13, below the gate (for 32 products per pair it would be
2.6e-12, above it).  A pair that drops the cross terms, a plausible slip,
breaks the bound on the same chains, so the check can fail.
"""
import random
from fractions import Fraction

import pytest

U = Fraction(1, 1 << 24)


def rn32(q):
    """q rounded to the nearest binary32 value (ties to even), as a Fraction;
    normal range only (every value here is far from underflow and overflow)."""
    if q == 0:
        return Fraction(0)
    s = -1 if q < 0 else 1
    a = abs(q)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    ulp = Fraction(2) ** (e - 23)
    n = a / ulp
    f = n.numerator // n.denominator
    r = n - f
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and f % 2 == 1):
        f += 1
    return s * f * ulp


def cut(v):
    """v = hi + lo + r: hi the top 24 significant bits, lo the next 23 (both
    truncated toward zero), as the kernels cut an FP64 operand."""
    a = abs(Fraction(v))
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    s = -1 if v < 0 else 1
    q1 = Fraction(2) ** (e - 23)
    hi = (a / q1).__floor__() * q1
    q2 = Fraction(2) ** (e - 46)
    lo = ((a - hi) / q2).__floor__() * q2
    return s * hi, s * lo


def pair_sum(avals, xvals, cross=True):
    """H + L after the emulated products of a and x enter one pair (without
    the cross terms t when cross is False)."""
    H = L = Fraction(0)
    for a, x in zip(avals, xvals):
        ah, al = cut(a)
        xh, xl = cut(x)
        p = rn32(ah * xh)
        e = ah * xh - p                         # exact (TwoProduct)
        t = rn32(ah * xl + rn32(al * xh + e)) if cross else e
        s = rn32(H + p)                         # TwoSum(H, p)
        z = rn32(s - H)
        err = rn32(rn32(H - rn32(s - z)) + rn32(p - z))
        assert s + err == H + p
        H = s
        L = rn32(L + rn32(err + t))
    return H + L


def bound(K):
    return U * U * (Fraction(K * (K + 1), 2) + 6 * K + 5) + Fraction(5, 2) * Fraction(2) ** -45


def rel_error(avals, xvals, cross=True):
    exact = sum(Fraction(a) * Fraction(x) for a, x in zip(avals, xvals))
    scale = sum(abs(Fraction(a) * Fraction(x)) for a, x in zip(avals, xvals))
    return abs(pair_sum(avals, xvals, cross) - exact) / scale


def near_top(rng):
    """Positive FP64 value just below a power of two (all mantissa bits set
    in the head and in the cut-off tail: the largest cut and TwoSum errors)."""
    return (2.0 - rng.random() * 2.0 ** -20) * 2.0 ** rng.randint(-4, 4)


def chains(kind, K, rng):
    if kind == "same_sign_top":
        return [near_top(rng) for _ in range(K)], [near_top(rng) for _ in range(K)]
    if kind == "one_large_then_ulps":
        # the first product sets H; the rest are each about one FP32 ulp of
        # it, so every TwoSum error is as large as it can be relative to S
        a = [1.9999999 * 2.0 ** 10] + [(1.0 + rng.random()) * 2.0 ** -14 for _ in range(K - 1)]
        x = [1.9999999] + [1.0 + rng.random() for _ in range(K - 1)]
        return a, x
    if kind == "growing":
        a = [(1.0 + rng.random()) * 2.0 ** (k // 2) for k in range(K)]
        x = [(1.0 + rng.random()) * 2.0 ** (k // 2) for k in range(K)]
        return a, x
    assert kind == "random_sign"
    a = [rng.choice((-1, 1)) * near_top(rng) for _ in range(K)]
    x = [rng.choice((-1, 1)) * near_top(rng) for _ in range(K)]
    return a, x


def test_rounding_helpers():
    assert rn32(Fraction(1) + U) == 1                # halfway: to the even neighbour
    assert rn32(Fraction(1) + 3 * U) == 1 + 4 * U
    assert rn32(Fraction(1) + U + U / 4) == 1 + 2 * U
    assert rn32(Fraction(3, 2) - U / 4) == Fraction(3, 2)
    v = 1.0 + 2.0 ** -30 + 2.0 ** -50
    hi, lo = cut(v)
    assert hi == 1 and lo == Fraction(2) ** -30 and abs(Fraction(v) - hi - lo) < Fraction(2) ** -46


def test_bound_values():
    assert float(bound(16)) == pytest.approx(9.13e-13, rel=1e-2)
    assert float(bound(16)) < 1e-12 < float(bound(32))


@pytest.mark.parametrize("kind", ["same_sign_top", "one_large_then_ulps", "growing", "random_sign"])
def test_pair_within_bound(kind):
    rng = random.Random(20210804)
    worst = Fraction(0)
    for _ in range(12):
        a, x = chains(kind, 16, rng)
        worst = max(worst, rel_error(a, x))
        assert rel_error(a, x, cross=False) > bound(16)
    assert worst <= bound(16), float(worst)


def test_search_stays_inside_bound():
    """A small random search for the chain of 16 with the largest relative
    error (mutating one operand at a time, keeping improvements) still ends
    inside the bound."""
    rng = random.Random(7)
    a, x = chains("one_large_then_ulps", 16, rng)
    best = rel_error(a, x)
    for _ in range(80):
        k = rng.randrange(16)
        a2, x2 = list(a), list(x)
        a2[k] = a2[k] * (1.0 + (rng.random() - 0.5) * 2.0 ** -rng.randint(1, 20))
        e = rel_error(a2, x2)
        if e > best:
            a, x, best = a2, x2, e
    assert best <= bound(16), float(best)
