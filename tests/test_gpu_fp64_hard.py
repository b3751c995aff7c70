"""FP64 GEMV and DOT on inputs that are hard for the FP32 emulation of part
of the products, against the oracle, element by element, at the FP64 gate
of Def. GEMV / Def. DOT (Sec. 3.1):

    |c_gpu_i - c_oracle_i| / (|c0_i| + |alpha| * sum_j |A_ij x_j|) <= 1e-12

The FP64 kernels form part of their products with FP32 instructions: each
operand cut into two FP32 parts, the head product by TwoProduct, the
running sum an FP32 pair updated by TwoSum and folded into FP64 after at
most 16 products.  Three input classes aim at the weak points of that:

* chains: every operand positive and just below a power of two, so every
  row is a long same-sign chain whose running sum grows fastest and whose
  TwoSum errors are largest;
* logu: magnitudes log-uniform over [2^-60, 2^60] with random signs, so the
  floor of each emulated product's error shows beside the small terms;
* mixed: uniform[-1,1] with zeros, subnormals, values below 2^-30 and values
  of magnitude 2^31 to 2^39 (across the top of the emulated range, 2^34)
  mixed in, so the warp vote moves groups of products between the emulated
  path and the FP64 fallback in the middle of a row.

Each shape selects one kernel: one-row long rows (fewer than 16 rows), the
row-group kernel (with and without column splits), short rows, realigned
rows (odd leading dimension), column tiles (tall, wide, square) and DOT
(one block and the grid)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_02025_gb300 as gb
import synth
from gpu_util import Guarded, rel_err, to_dev, workspace

ROW, COL = gb.ROW_MAJOR, gb.COL_MAJOR
TOL = 1e-12


def unit(size, seed, stream):
    """Seeded values in [0, 1)."""
    return (synth.uniform(size, seed, stream, np.float64) + 1.0) * 0.5


def hard(kind, size, seed, stream):
    if size == 0:
        return np.zeros(0)
    if kind == "chains":
        e = np.floor(unit(size, seed, stream) * 7.0) - 3.0          # binades 2^-3 .. 2^3
        frac = 2.0 - unit(size, seed, stream + 100) * 2.0 ** -10     # just below the next power of two
        return np.ldexp(frac, e.astype(np.int64))
    if kind == "logu":
        mag = np.exp2(unit(size, seed, stream) * 120.0 - 60.0)
        sign = np.where(unit(size, seed, stream + 100) < 0.5, -1.0, 1.0)
        return sign * mag
    assert kind == "mixed"
    v = synth.uniform(size, seed, stream, np.float64)
    pick = unit(size, seed, stream + 100)
    v[pick < 0.08] = 0.0
    sub = (pick >= 0.08) & (pick < 0.11)
    v[sub] = np.ldexp(1.0 + unit(int(sub.sum()), seed, stream + 200), -1040)   # subnormal
    big = (pick >= 0.11) & (pick < 0.14)
    v[big] = np.ldexp(1.0 + unit(int(big.sum()), seed, stream + 300), 31 + (np.arange(int(big.sum())) % 9))
    tiny = (pick >= 0.14) & (pick < 0.16)
    v[tiny] = np.ldexp(1.0 + unit(int(tiny.sum()), seed, stream + 400), -40)    # normal, below 2^-30
    return v


GEMV_SHAPES = [  # (layout, m, n, pad, kernel it selects)
    (ROW, 8, 200000, 0, "row-long"),
    (ROW, 300, 5000, 0, "row-group"),
    (ROW, 40, 200000, 0, "row-group-split"),
    (ROW, 5000, 64, 0, "short"),
    (ROW, 3000, 200, 0, "short-200"),
    (ROW, 300, 5001, 0, "realigned"),
    (COL, 5000, 64, 0, "col-tall"),
    (COL, 5001, 32, 0, "col-tall-32"),
    (COL, 64, 100000, 0, "col-wide"),
    (COL, 1000, 1000, 0, "col-square"),
]
KINDS = ["chains", "logu", "mixed"]


@pytest.mark.gpu
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("layout,m,n,pad,name", GEMV_SHAPES, ids=[s[-1] for s in GEMV_SHAPES])
def test_gemv_hard_inputs(kind, layout, m, n, pad, name):
    ld = (n if layout == ROW else m) + pad
    size = (m - 1) * ld + n if layout == ROW else (n - 1) * ld + m
    seed = 11 + KINDS.index(kind)
    A, x, c0 = hard(kind, size, seed, 1), hard(kind, n, seed, 2), hard(kind, m, seed, 3)
    alpha = 0.75
    nb = gb.gb_workspace_bytes(gb.OP_GEMV, gb.F64, layout, m, n)
    dc = Guarded(c0)
    st = gb.gb_dgemv(layout, m, n, alpha, to_dev(A), ld, to_dev(x), dc.view, workspace(nb), nb)
    assert st == gb.GB_OK, gb.gb_status_string(st)
    torch.cuda.synchronize()
    got = dc.result()
    want = oracle.gemv(layout, m, n, alpha, A, ld, x, c0)
    scale = oracle.gemv_scale(layout, m, n, alpha, A, ld, x, c0)
    err = rel_err(got, want, scale)
    assert err <= TOL, (name, kind, err)


@pytest.mark.gpu
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("n", [6000, 1 << 20], ids=["one-block", "grid"])
def test_dot_hard_inputs(kind, n):
    seed = 21 + KINDS.index(kind)
    x, y = hard(kind, n, seed, 4), hard(kind, n, seed, 5)
    a0 = 0.375
    nb = gb.gb_workspace_bytes(gb.OP_DOT, gb.F64, 0, 0, n)
    da = Guarded(np.array([a0]))
    st = gb.gb_ddot(n, to_dev(x), to_dev(y), da.view, workspace(nb), nb)
    assert st == gb.GB_OK, gb.gb_status_string(st)
    torch.cuda.synchronize()
    got = float(da.result()[0])
    want = oracle.dot(n, x, y, a0)
    scale = oracle.dot_scale(n, x, y, a0)
    assert abs(got - want) / scale <= TOL, (kind, n, abs(got - want) / scale)


def test_hard_classes_reach_the_emulation_limits():
    """The classes are what they claim: chains are positive and within
    2^-10 below a power of two; logu spans both ends of the emulated
    range; mixed holds zeros, subnormals and values on both sides of
    2^34, the top of the emulated range."""
    c = hard("chains", 10000, 1, 1)
    assert np.all(c > 0)
    top = np.exp2(np.ceil(np.log2(c)))
    assert np.all((top - c) / top <= 2.0 ** -11 + 1e-15)
    lg = np.abs(hard("logu", 10000, 1, 1))
    assert lg.min() < 2.0 ** -55 and lg.max() > 2.0 ** 55
    mx = hard("mixed", 10000, 1, 1)
    assert np.any(mx == 0.0)
    assert np.any((mx != 0) & (np.abs(mx) < np.finfo(np.float64).tiny))
    assert np.any(np.abs(mx) >= 2.0 ** 34)
    assert np.any((np.abs(mx) >= 2.0 ** 31) & (np.abs(mx) < 2.0 ** 34))
    assert np.any((np.abs(mx) > 0) & (np.abs(mx) < 2.0 ** -30) & (np.abs(mx) >= np.finfo(np.float64).tiny))
