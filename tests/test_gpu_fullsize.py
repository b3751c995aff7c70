"""The plain-method sweep at full size (GEMV 16384^2, 1048576x64 and
64x1048576 in both layouts; DOT n = 2^28; GER 16384^2 in both layouts; FP32
and FP64; inputs uniform[-1,1]), called exactly as the benchmark calls it,
checked on sampled outputs that the oracle computes one by one (GEMV rows,
GER lines) or in full (the DOT scalar)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_02025_gb300 as gb
import synth

pytestmark = pytest.mark.gpu

ROW, COL = gb.ROW_MAJOR, gb.COL_MAJOR
TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
TDT = [torch.float64, torch.float32]
IDS = ["f64", "f32"]


def filled(numel, dtype, seed, stream):
    t = torch.empty(numel, dtype=dtype, device="cuda")
    synth.fill_uniform(t, seed, stream)
    return t


def sample(count, k, seed):
    rng = np.random.default_rng(seed)
    s = {0, 1, count // 2, count - 2, count - 1}
    s.update(rng.choice(count, size=min(k, count), replace=False).tolist())
    return np.array(sorted(i for i in s if 0 <= i < count))


GEMV_SHAPES = [(16384, 16384), (1048576, 64), (64, 1048576)]


@pytest.mark.parametrize("dtype", TDT, ids=IDS)
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
@pytest.mark.parametrize("shape", GEMV_SHAPES, ids=[f"{m}x{n}" for m, n in GEMV_SHAPES])
def test_gemv_full_size_sampled_rows(dtype, layout, shape):
    m, n = shape
    A = filled(m * n, dtype, 0, 1)
    x = filled(n, dtype, 0, 2)
    c = filled(m, dtype, 0, 3)
    c0 = c.cpu().numpy().astype(np.float64)
    gb.gemv(A, x, c, alpha=1.0, layout=layout, m=m, n=n, lda=n if layout == ROW else m)
    torch.cuda.synchronize()
    rows = sample(m, 60, 1)
    if layout == ROW:
        Ar = A.view(m, n)[torch.from_numpy(rows).cuda()].cpu().numpy()
    else:
        Ar = A.view(n, m)[:, torch.from_numpy(rows).cuda()].t().contiguous().cpu().numpy()
    xs = x.cpu().numpy()
    k = len(rows)
    want = oracle.gemv(ROW, k, n, 1.0, Ar.ravel(), n, xs, c0[rows])
    scale = oracle.gemv_scale(ROW, k, n, 1.0, Ar.ravel(), n, xs, c0[rows])
    got = c.cpu().numpy()[rows].astype(np.float64)
    err = np.max(np.abs(got - want) / scale)
    assert err <= TOL[dtype], (dtype, layout, shape, err)
    del A


@pytest.mark.parametrize("dtype", TDT, ids=IDS)
def test_dot_full_size(dtype):
    n = 1 << 28
    x = filled(n, dtype, 0, 4)
    y = filled(n, dtype, 0, 5)
    a = torch.tensor([0.5], dtype=dtype, device="cuda")
    gb.dot(x, y, a)
    torch.cuda.synchronize()
    xs, ys = x.cpu().numpy(), y.cpu().numpy()
    want = oracle.dot(n, xs, ys, 0.5)
    scale = oracle.dot_scale(n, xs, ys, 0.5)
    err = abs(float(a.item()) - want) / scale
    assert err <= TOL[dtype], (dtype, err)


@pytest.mark.parametrize("dtype", TDT, ids=IDS)
@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
def test_ger_full_size_sampled_lines(dtype, layout):
    m = n = 16384
    C = filled(m * n, dtype, 0, 6)
    x = filled(m, dtype, 0, 7)
    y = filled(n, dtype, 0, 8)
    lines = sample(m, 40, 2)
    idx = torch.from_numpy(lines).cuda()
    before = C.view(m, n)[idx].cpu().numpy()  # lines are rows (row-major) or columns (col-major)
    gb.ger(x, y, C, alpha=-0.7, layout=layout, m=m, n=n, ldc=n)
    torch.cuda.synchronize()
    after = C.view(m, n)[idx].cpu().numpy()
    xs, ys = x.cpu().numpy(), y.cpu().numpy()
    k = len(lines)
    if layout == ROW:
        want = oracle.ger(ROW, k, n, -0.7, xs[lines], ys, before.ravel(), n).reshape(k, n)
    else:
        want = oracle.ger(COL, m, k, -0.7, xs, ys[lines], before.ravel(), m).reshape(k, m)
    assert np.array_equal(after.view(np.uint8), want.view(np.uint8))
