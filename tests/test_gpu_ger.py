"""GER on the GPU (Def. GEM; Alg. 2) against the CPU oracle through the C
ABI: C_ij <- fma(x_i, fl(alpha*y_j), C_ij), one rounding per element, so the
results must be bit-identical, and padding between rows (or columns) must
stay untouched."""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_02025_gb300 as gb
import synth
from gpu_util import Guarded, to_dev

pytestmark = pytest.mark.gpu

ROW, COL = gb.ROW_MAJOR, gb.COL_MAJOR
DTYPES = [np.float64, np.float32]
DT_IDS = ["f64", "f32"]


def storage(layout, m, n, ld):
    if m == 0 or n == 0:
        return 0
    return (m - 1) * ld + n if layout == ROW else (n - 1) * ld + m


def check(dt, layout, m, n, pad=0, alpha=-0.7, seed=0, misalign=0):
    ld = max((n if layout == ROW else m) + pad, 1)
    size = storage(layout, m, n, ld)
    C = synth.uniform(size, seed, 1, dt)
    lines, length = (m, n) if layout == ROW else (n, m)
    for L in range(max(lines - 1, 0)):
        C[L * ld + length:(L + 1) * ld] = np.nan  # padding: must stay NaN
    x = synth.uniform(m, seed, 2, dt)
    y = synth.uniform(n, seed, 3, dt)
    dC = Guarded(C, misalign)
    f = gb.gb_dger if dt == np.float64 else gb.gb_sger
    st = f(layout, m, n, alpha, to_dev(x, misalign) if m else None,
           to_dev(y, misalign) if n else None, dC.view if size else None, ld)
    assert st == gb.GB_OK, gb.gb_status_string(st)
    torch.cuda.synchronize()
    got = dC.result()
    want = oracle.ger(layout, m, n, alpha, x, y, C, ld)
    assert np.array_equal(got.view(np.uint8), want.view(np.uint8)), (dt, layout, m, n, pad, misalign)


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
def test_tiny_exhaustive(dt, layout):
    for m in (0, 1, 2, 3, 5, 33):
        for n in (0, 1, 2, 3, 7, 33, 129):
            for pad in (0, 3):
                check(dt, layout, m, n, pad, seed=m * 100 + n)


SHAPES = [(1000, 777), (777, 1000), (100003, 64), (64, 100003), (3, 300001), (300001, 3),
          (2049, 2051)]


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{m}x{n}" for m, n in SHAPES])
def test_shapes(dt, layout, shape):
    check(dt, layout, *shape, pad=0, seed=4)
    check(dt, layout, *shape, pad=5, alpha=1.0, seed=5)


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
@pytest.mark.parametrize("misalign", [1, 3])
def test_misaligned(dt, layout, misalign):
    check(dt, layout, 1000, 777, pad=1, seed=6, misalign=misalign)


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
def test_alpha_zero_reads_nothing(dt):
    C = synth.uniform(12, 7, 1, dt)
    dC = Guarded(C)
    f = gb.gb_dger if dt == np.float64 else gb.gb_sger
    nan = to_dev(np.full(4, np.nan, dt))
    assert f(ROW, 3, 4, 0.0, nan, nan, dC.view, 4) == gb.GB_OK
    torch.cuda.synchronize()
    assert np.array_equal(dC.result(), C)
