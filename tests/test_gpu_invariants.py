"""Invariants of the definitions (Def. GEMV, Def. DOT, Def. GEM) checked on
the GPU path alone, with shapes that take the split sums:

* scaling alpha or x by a power of two scales c exactly (every rounding in
  the sum commutes with it while nothing overflows or underflows; operands
  are kept above 2^-20 in magnitude so that the choice between the FP64
  and the emulated FP64 products does not change with the scaling);
* GEMV is linear in x, within the tolerance of the three sums;
* DOT equals a one-row row-major GEMV with c0 = alpha0;
* (C + alpha x y^T) z = C z + alpha x (y . z), GER then GEMV against GEMV
  and DOT, within the tolerance of the sums plus the rounding of C."""
import numpy as np
import pytest
import torch

import paper_2108_02025_gb300 as gb
import synth
from gpu_util import rel_err, to_dev, workspace

pytestmark = pytest.mark.gpu

ROW, COL = gb.ROW_MAJOR, gb.COL_MAJOR
TOL = {np.float64: 1e-12, np.float32: 1e-5}
SHAPES = [(3000, 3001), (64, 200003), (100000, 33), (7, 70001), (1, 1 << 18)]


def away_from_zero(v):
    tiny = np.float64(2.0 ** -20)
    return np.where(np.abs(v) < tiny, np.copysign(tiny, v), v).astype(v.dtype)


def gemv(dt, layout, m, n, alpha, A, ld, x, c0):
    dc = to_dev(c0)
    code = gb.F64 if dt == np.float64 else gb.F32
    nb = gb.gb_workspace_bytes(gb.OP_GEMV, code, layout, m, n)
    f = gb.gb_dgemv if dt == np.float64 else gb.gb_sgemv
    st = f(layout, m, n, alpha, A, ld, to_dev(x), dc, workspace(nb), nb)
    assert st == gb.GB_OK, gb.gb_status_string(st)
    torch.cuda.synchronize()
    return dc.cpu().numpy()


def dot(dt, n, x, y, a0):
    da = to_dev(np.array([a0], dt))
    code = gb.F64 if dt == np.float64 else gb.F32
    nb = gb.gb_workspace_bytes(gb.OP_DOT, code, 0, 0, n)
    f = gb.gb_ddot if dt == np.float64 else gb.gb_sdot
    st = f(n, to_dev(x), to_dev(y), da, workspace(nb), nb)
    assert st == gb.GB_OK, gb.gb_status_string(st)
    torch.cuda.synchronize()
    return float(da.cpu().numpy()[0])


def operands(dt, layout, m, n, seed):
    ld = n if layout == ROW else m
    A = away_from_zero(synth.uniform(m * n, seed, 1, dt))
    x = away_from_zero(synth.uniform(n, seed, 2, dt))
    return A, ld, x


def abs_scale(layout, m, n, A, x):
    A2 = np.abs(A.astype(np.float64)).reshape((m, n) if layout == ROW else (n, m))
    A2 = A2 if layout == ROW else A2.T
    return A2 @ np.abs(x.astype(np.float64))


@pytest.mark.parametrize("dt", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{m}x{n}" for m, n in SHAPES])
def test_power_of_two_scaling_is_exact(dt, layout, shape):
    m, n = shape
    A, ld, x = operands(dt, layout, m, n, 11)
    dA = to_dev(A)
    zero = np.zeros(m, dt)
    base = gemv(dt, layout, m, n, 0.75, dA, ld, x, zero)
    a2 = gemv(dt, layout, m, n, 1.5, dA, ld, x, zero)
    x4 = gemv(dt, layout, m, n, 0.75, dA, ld, (x * dt(4)).astype(dt), zero)
    assert np.array_equal(a2.view(np.uint8), (base * dt(2)).view(np.uint8))
    assert np.array_equal(x4.view(np.uint8), (base * dt(4)).view(np.uint8))


@pytest.mark.parametrize("dt", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
@pytest.mark.parametrize("shape", SHAPES[:4], ids=[f"{m}x{n}" for m, n in SHAPES[:4]])
def test_linear_in_x(dt, layout, shape):
    m, n = shape
    A, ld, x1 = operands(dt, layout, m, n, 12)
    x2 = away_from_zero(synth.uniform(n, 12, 3, dt))
    xs = (x1.astype(np.float64) + x2).astype(dt)      # rounded sum: the reference uses xs itself
    dA = to_dev(A)
    zero = np.zeros(m, dt)
    r1 = gemv(dt, layout, m, n, 1.0, dA, ld, x1, zero).astype(np.float64)
    r2 = gemv(dt, layout, m, n, 1.0, dA, ld, x2, zero).astype(np.float64)
    rs = gemv(dt, layout, m, n, 1.0, dA, ld, xs, zero).astype(np.float64)
    # xs_j = x1_j + x2_j + d_j with |d_j| <= u |xs_j|: A d is within u * |A||xs|
    u = float(np.finfo(dt).eps) / 2
    s1, s2, ss = (abs_scale(layout, m, n, A, v) for v in (x1, x2, xs))
    scale = s1 + s2 + ss
    assert rel_err(rs, r1 + r2, scale) <= TOL[dt] + u * 2


@pytest.mark.parametrize("dt", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("n", [1, 31, 4096, 65537, 1 << 20, 3 << 20])
def test_dot_equals_one_row_gemv(dt, n):
    x = synth.uniform(n, 13, 1, dt)
    y = synth.uniform(n, 13, 2, dt)
    a0 = dt(0.3125)
    d = dot(dt, n, x, y, a0)
    g = gemv(dt, ROW, 1, n, 1.0, to_dev(x), n, y, np.array([a0], dt))[0]
    scale = abs(float(a0)) + float(np.abs(x.astype(np.float64)) @ np.abs(y.astype(np.float64)))
    assert abs(d - float(g)) <= 2 * TOL[dt] * scale


@pytest.mark.parametrize("dt", [np.float64, np.float32], ids=["f64", "f32"])
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
@pytest.mark.parametrize("shape", [(1000, 1001), (64, 100003), (50000, 17)], ids=["sq", "wide", "tall"])
def test_ger_then_gemv(dt, layout, shape):
    m, n = shape
    alpha = -0.625
    ld = n if layout == ROW else m
    C = synth.uniform(m * n, 14, 1, dt)
    x = synth.uniform(m, 14, 2, dt)
    y = synth.uniform(n, 14, 3, dt)
    z = synth.uniform(n, 14, 4, dt)
    dC = to_dev(C)
    zero = np.zeros(m, dt)
    cz = gemv(dt, layout, m, n, 1.0, dC, ld, z, zero).astype(np.float64)
    f = gb.gb_dger if dt == np.float64 else gb.gb_sger
    assert f(layout, m, n, alpha, to_dev(x), to_dev(y), dC, ld) == gb.GB_OK
    torch.cuda.synchronize()
    c2z = gemv(dt, layout, m, n, 1.0, dC, ld, z, zero).astype(np.float64)
    yz = dot(dt, n, y, z, dt(0))
    want = cz + alpha * x.astype(np.float64) * yz
    ay = abs(alpha) * np.abs(x.astype(np.float64)) * float(np.abs(y.astype(np.float64)) @ np.abs(z))
    scale = abs_scale(layout, m, n, C, z) + ay
    # three sums within TOL each, the rounding of alpha*y and of each C + x t (u each)
    u = float(np.finfo(dt).eps) / 2
    assert rel_err(c2z, want, scale) <= 3 * TOL[dt] + 4 * u
