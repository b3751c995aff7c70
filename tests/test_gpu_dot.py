"""DOT on the GPU (Def. DOT; Alg. 3 single block, Alg. 4 blocked) against
the CPU oracle through the C ABI.  Tolerance relative to
|alpha0| + sum_p |x_p y_p|: 1e-12 (FP64), 1e-5 (FP32)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_02025_gb300 as gb
import synth
from gpu_util import Guarded, to_dev, workspace

pytestmark = pytest.mark.gpu

TOL = {np.float64: 1e-12, np.float32: 1e-5}
DTYPES = [np.float64, np.float32]
DT_IDS = ["f64", "f32"]


def gpu_dot(dt, n, x, y, a0, misalign=0, ws=None):
    dx, dy = to_dev(x, misalign), to_dev(y, (2 * misalign) % 3)
    da = Guarded(np.array([a0], dtype=dt))
    code = gb.F64 if dt == np.float64 else gb.F32
    nb = gb.gb_workspace_bytes(gb.OP_DOT, code, 0, 0, n)
    if ws is None:
        ws = workspace(nb)
    f = gb.gb_ddot if dt == np.float64 else gb.gb_sdot
    st = f(n, dx if n else None, dy if n else None, da.view, ws, nb)
    assert st == gb.GB_OK, gb.gb_status_string(st)
    torch.cuda.synchronize()
    return float(da.result()[0])


def check(dt, n, seed=0, a0=0.375, misalign=0):
    x = synth.uniform(n, seed, 1, dt)
    y = synth.uniform(n, seed, 2, dt)
    got = gpu_dot(dt, n, x, y, dt(a0), misalign)
    want = oracle.dot(n, x, y, float(dt(a0)))
    scale = oracle.dot_scale(n, x, y, float(dt(a0)))
    err = abs(got - want) / scale
    assert err <= TOL[dt], (dt, n, misalign, err)


SIZES = [0, 1, 2, 3, 7, 255, 1024, 16383, 16384, 16385, 100003, 1 << 20, (1 << 22) + 5,
         3 * (1 << 21) + 1]


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
@pytest.mark.parametrize("n", SIZES)
def test_sizes(dt, n):
    check(dt, n, seed=n % 97)


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
@pytest.mark.parametrize("misalign", [1, 2])
def test_misaligned(dt, misalign):
    for n in (5, 20000, 1000003):
        check(dt, n, seed=3, misalign=misalign)


def single_block_limit(dt):
    """Largest n that DOT runs as one block: the workspace (partials of the
    blocks) is empty exactly there."""
    code = gb.F64 if dt == np.float64 else gb.F32
    lo, hi = 1, 1 << 30
    while lo < hi:
        mid = (lo + hi + 1) // 2
        if gb.gb_workspace_bytes(gb.OP_DOT, code, 0, 0, mid) == 0:
            lo = mid
        else:
            hi = mid - 1
    return lo


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
def test_small_and_large_regimes_agree(dt):
    """At the single-block / multi-block boundary both forms match the
    oracle (the paper's small/large cutoff, Sec. 4.3.1)."""
    b = single_block_limit(dt)
    assert 1024 <= b < 1 << 24
    for n in (b - 1, b, b + 1, b + 7):
        check(dt, n, seed=5)


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
def test_integer_inputs_exact_and_deterministic(dt):
    n = (1 << 21) + 17
    x = synth.integers(n, 6, 1, -1, 1, dt)
    y = synth.integers(n, 6, 2, -1, 1, dt)
    want = float(int(x.astype(np.int64) @ y.astype(np.int64)) + 3)
    nb = gb.gb_workspace_bytes(gb.OP_DOT, gb.F64 if dt == np.float64 else gb.F32, 0, 0, n)
    ws = workspace(nb)
    r = [gpu_dot(dt, n, x, y, dt(3), ws=ws) for _ in range(3)]
    assert r[0] == want and r[1] == want and r[2] == want


@pytest.mark.parametrize("dt", DTYPES, ids=DT_IDS)
def test_alpha_is_accumulator(dt):
    n = 1000
    x = np.ones(n, dt)
    y = np.ones(n, dt)
    assert gpu_dot(dt, n, x, y, dt(0.5)) == 1000.5
    assert gpu_dot(dt, 0, x[:0], y[:0], dt(0.5)) == 0.5
