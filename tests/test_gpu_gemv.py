"""GEMV on the GPU (Def. GEMV; Alg. 1 column-major, Alg. 2 row-major)
against the CPU oracle, element by element, through the C ABI.

Tolerance (condition-aware, per row i):
    |c_gpu_i - c_oracle_i| / (|c0_i| + |alpha| * sum_j |A_ij x_j|)
    <= 1e-12 (FP64), <= 1e-5 (FP32)
Integer-valued inputs make every summation order exact, so there the
results must be bit-identical."""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_02025_gb300 as gb
import synth
from gpu_util import Guarded, rel_err, to_dev, workspace

pytestmark = pytest.mark.gpu

ROW, COL = gb.ROW_MAJOR, gb.COL_MAJOR
TOL = {np.float64: 1e-12, np.float32: 1e-5}


def storage(layout, m, n, ld):
    if m == 0 or n == 0:
        return 0
    return (m - 1) * ld + n if layout == ROW else (n - 1) * ld + m


def padding_mask(layout, m, n, ld, size):
    mask = np.zeros(size, bool)
    if size == 0:
        return mask
    lines, length = (m, n) if layout == ROW else (n, m)
    for L in range(lines - 1):
        mask[L * ld + length:(L + 1) * ld] = True
    return mask


def make(dt, layout, m, n, pad, seed, ints=False):
    ld = max((n if layout == ROW else m) + pad, 1)
    size = storage(layout, m, n, ld)
    if ints:
        A = synth.integers(size, seed, 1, -8, 8, dt)
        x = synth.integers(n, seed, 2, -8, 8, dt)
        c0 = synth.integers(m, seed, 3, -8, 8, dt)
    else:
        A = synth.uniform(size, seed, 1, dt)
        x = synth.uniform(n, seed, 2, dt)
        c0 = synth.uniform(m, seed, 3, dt)
    A[padding_mask(layout, m, n, ld, size)] = np.nan  # any read of padding poisons c
    return A, x, c0, ld


def gpu_gemv(dt, layout, m, n, alpha, A, ld, x, c0, misalign=0, ws=None):
    dA, dx = to_dev(A, misalign), to_dev(x, misalign)
    dc = Guarded(c0, misalign)
    code = gb.F64 if dt == np.float64 else gb.F32
    nb = gb.gb_workspace_bytes(gb.OP_GEMV, code, layout, m, n)
    if ws is None:
        ws = workspace(nb)
    f = gb.gb_dgemv if dt == np.float64 else gb.gb_sgemv
    st = f(layout, m, n, alpha, dA if A.size else None, ld, dx if n else None, dc.view, ws, nb)
    assert st == gb.GB_OK, gb.gb_status_string(st)
    torch.cuda.synchronize()
    return dc.result()


def check(dt, layout, m, n, pad=0, alpha=0.75, seed=0, misalign=0):
    A, x, c0, ld = make(dt, layout, m, n, pad, seed)
    got = gpu_gemv(dt, layout, m, n, alpha, A, ld, x, c0, misalign)
    want = oracle.gemv(layout, m, n, alpha, A, ld, x, c0)
    scale = oracle.gemv_scale(layout, m, n, alpha, A, ld, x, c0)
    err = rel_err(got, want, scale)
    assert err <= TOL[dt], (dt, layout, m, n, pad, misalign, err)
    return err


DTYPES = [np.float64, np.float32]
DT_IDS = ["f64", "f32"]


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
def test_tiny_exhaustive(dt, layout):
    for m in (0, 1, 2, 3, 5, 17, 33):
        for n in (0, 1, 2, 3, 7, 33, 65, 130):
            for pad in (0, 3):
                check(dt, layout, m, n, pad, seed=m * 1000 + n * 10 + pad)


SHAPES = [(1000, 777), (777, 1000), (64, 100003), (100003, 64), (100001, 5), (5, 100001),
          (33, 250001), (250001, 33), (1, 70000), (70000, 1), (4097, 129), (20003, 32)]


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{m}x{n}" for m, n in SHAPES])
def test_shapes(dt, layout, shape):
    m, n = shape
    check(dt, layout, m, n, pad=0, seed=7)
    check(dt, layout, m, n, pad=5, alpha=-1.25, seed=8)


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
@pytest.mark.parametrize("misalign", [1, 2, 3])
def test_misaligned_pointers(dt, layout, misalign):
    for (m, n) in ((1000, 777), (64, 20000), (20000, 64)):
        check(dt, layout, m, n, pad=1, seed=9, misalign=misalign)


def test_config1_fp64_rowmajor_4096():
    """FP64 row-major 4096 x 4096, A, x, c uniform[-1,1] from seed 0, one
    call against the oracle."""
    check(np.float64, ROW, 4096, 4096, pad=0, alpha=1.0, seed=0)


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
def test_integer_inputs_bit_exact(dt, layout):
    for (m, n) in ((513, 2050), (64, 60001), (30001, 64), (7, 9)):
        A, x, c0, ld = make(dt, layout, m, n, 2, seed=11, ints=True)
        got = gpu_gemv(dt, layout, m, n, 2.0, A, ld, x, c0)
        want = oracle.gemv(layout, m, n, 2.0, A, ld, x, c0)
        assert np.array_equal(got.astype(np.float64), want), (dt, layout, m, n)


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
def test_alpha_zero_reads_nothing(dt, layout):
    m, n = 100, 300
    A = np.full(m * n, np.nan, dt)
    x = np.full(n, np.nan, dt)
    c0 = synth.uniform(m, 12, 3, dt)
    got = gpu_gemv(dt, layout, m, n, 0.0, A, n if layout == ROW else m, x, c0)
    assert np.array_equal(got, c0)


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
def test_nan_inf_propagate_to_their_row_only(dt, layout):
    m, n = 70, 5000
    A, x, c0, ld = make(dt, layout, m, n, 0, seed=13)
    A[(5 * ld + 17) if layout == ROW else (5 + 17 * ld)] = np.nan
    A[(9 * ld + 4000) if layout == ROW else (9 + 4000 * ld)] = np.inf
    got = gpu_gemv(dt, layout, m, n, 1.0, A, ld, x, c0)
    assert np.isnan(got[5])
    assert np.isinf(got[9]) and np.sign(got[9]) == np.sign(x[4000])
    others = np.ones(m, bool)
    others[[5, 9]] = False
    assert np.all(np.isfinite(got[others]))


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
def test_deterministic_and_workspace_reusable(dt, layout):
    """Split sums reset their counters: the same workspace serves repeated
    calls, and repeated calls are bit-identical."""
    for (m, n) in ((64, 200003), (3000, 3000)):
        A, x, c0, ld = make(dt, layout, m, n, 0, seed=14)
        code = gb.F64 if dt == np.float64 else gb.F32
        ws = workspace(gb.gb_workspace_bytes(gb.OP_GEMV, code, layout, m, n))
        r1 = gpu_gemv(dt, layout, m, n, 1.5, A, ld, x, c0, ws=ws)
        r2 = gpu_gemv(dt, layout, m, n, 1.5, A, ld, x, c0, ws=ws)
        r3 = gpu_gemv(dt, layout, m, n, 1.5, A, ld, x, c0, ws=ws)
        assert np.array_equal(r1, r2) and np.array_equal(r2, r3)
        want = oracle.gemv(layout, m, n, 1.5, A, ld, x, c0)
        scale = oracle.gemv_scale(layout, m, n, 1.5, A, ld, x, c0)
        assert rel_err(r3, want, scale) <= TOL[dt]


def test_row_major_equals_col_major_of_transpose():
    """The same logical matrix stored both ways gives the same c within
    tolerance (different kernels, different summation orders)."""
    m, n = 900, 1100
    M = synth.uniform(m * n, 15, 1).reshape(m, n)
    x = synth.uniform(n, 15, 2)
    c0 = synth.uniform(m, 15, 3)
    r = gpu_gemv(np.float64, ROW, m, n, 1.0, M.ravel(), n, x, c0)
    c = gpu_gemv(np.float64, COL, m, n, 1.0, np.ascontiguousarray(M.T).ravel(), m, x, c0)
    scale = oracle.gemv_scale(ROW, m, n, 1.0, M.ravel(), n, x, c0)
    assert rel_err(r, c, scale) <= 2e-12


def gpu_gemv_offsets(dt, m, n, alpha, A, ld, x, c0, a_off):
    """A starts a_off elements after a 256-byte boundary, x 16-byte aligned."""
    dA = to_dev(A, a_off)
    dx = to_dev(x, 0)
    dc = Guarded(c0, 0)
    code = gb.F64 if dt == np.float64 else gb.F32
    nb = gb.gb_workspace_bytes(gb.OP_GEMV, code, ROW, m, n)
    ws = workspace(nb)
    f = gb.gb_dgemv if dt == np.float64 else gb.gb_sgemv
    assert f(ROW, m, n, alpha, dA, ld, dx, dc.view, ws, nb) == gb.GB_OK
    torch.cuda.synchronize()
    return dc.result()


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
@pytest.mark.parametrize("shape", [(37, 5000), (3, 200001), (600, 2049), (1, 4099), (5000, 1030),
                                   (1000, 63), (3000, 130), (257, 1021), (77, 5), (4, 1)],
                         ids=lambda s: f"{s[0]}x{s[1]}")
def test_rows_off_16_bytes_with_aligned_x(dt, shape):
    """Row-major A whose rows do not start on 16 bytes (lda not a multiple of
    the pack, or A offset by whole elements) with x 16-byte aligned: the
    realigned long-row and short-row paths, every row offset, ragged ends,
    split rows."""
    m, n = shape
    V = 16 // np.dtype(dt).itemsize
    for pad, a_off in ((1, 0), (2, 1), (3, 0), (0, 1), (V - 1, V - 1), (5, 2)):
        A, x, c0, ld = make(dt, ROW, m, n, pad, seed=m + n + pad)
        got = gpu_gemv_offsets(dt, m, n, -0.75, A, ld, x, c0, a_off % V)
        want = oracle.gemv(ROW, m, n, -0.75, A, ld, x, c0)
        scale = oracle.gemv_scale(ROW, m, n, -0.75, A, ld, x, c0)
        err = rel_err(got, want, scale)
        assert err <= TOL[dt], (dt, m, n, pad, a_off, err)


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
def test_rows_off_16_bytes_integer_exact(dt):
    m, n = 64, 30001
    A = synth.integers((m - 1) * (n + 1) + n, 31, 1, -8, 8, dt)
    x = synth.integers(n, 31, 2, -8, 8, dt)
    c0 = synth.integers(m, 31, 3, -8, 8, dt)
    got = gpu_gemv_offsets(dt, m, n, 1.0, A, n + 1, x, c0, 0)
    want = oracle.gemv(ROW, m, n, 1.0, A, n + 1, x, c0)
    assert np.array_equal(got.astype(np.float64), want)


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
def test_short_rows_padded_ld_ragged_end(dt):
    """Aligned short rows (lda a multiple of the pack, n not): the ragged
    columns past the last pack when a row has fewer lanes than ragged
    columns (1 or 2 lanes per row, FP32)."""
    V = 16 // np.dtype(dt).itemsize
    for n in (1, 2, 3, 5, 6, 7, 9, 14, 15, 31, 63, 127):
        m = 700
        ld = (n + V - 1) // V * V
        check(dt, ROW, m, n, pad=ld - n, alpha=0.5, seed=n)
