"""Operands past 2^31 elements: 64-bit index arithmetic in every path.

A_ij = (i mod 7) - 3 and x_j, y_j small integers make every sum exact in any
order, so each output has a closed form that a wrong row or column index
would break: GEMV c_i = ((i mod 7) - 3) * sum_j x_j; DOT = sum_p x_p y_p
with period-21 patterns (4.3e9 in total, past FP32's integers: one
rounding of the exact FP64 sum);
GER C_ij = (i mod 7) - 3 + alpha x_i y_j.  Built on the device (8.6 GB per
FP32 matrix), checked in full on the device."""
import numpy as np
import pytest
import torch

import paper_2108_02025_gb300 as gb

pytestmark = pytest.mark.gpu

M, N = (1 << 16) + 3, (1 << 15) + 1  # m*n > 2^31


def row_pattern(m, dev):
    return (torch.arange(m, device=dev) % 7 - 3).to(torch.float32)


@pytest.mark.parametrize("layout,ld_pad", [(gb.ROW_MAJOR, 3), (gb.ROW_MAJOR, 0), (gb.COL_MAJOR, 1)],
                         ids=["row-aligned", "row-odd-ld", "col"])
def test_gemv_past_2_31(layout, ld_pad):
    dev = torch.device("cuda", 0)
    m, n = M, N
    ld = (n if layout == gb.ROW_MAJOR else m) + ld_pad
    pat = row_pattern(m, dev)
    if layout == gb.ROW_MAJOR:
        A = torch.empty((m, ld), dtype=torch.float32, device=dev)
        A[:] = pat[:, None]
    else:
        A = torch.empty((n, ld), dtype=torch.float32, device=dev)
        A[:, :m] = pat[None, :]
        A[:, m:] = float("nan")
    x = (torch.arange(n, device=dev) % 5 - 2).to(torch.float32)
    c = torch.zeros(m, dtype=torch.float32, device=dev)
    gb.gemv(A, x, c, 1.0, layout, m, n, ld)
    want = pat * float(x.double().sum())
    assert torch.equal(c, want)
    del A
    torch.cuda.empty_cache()


def test_dot_past_2_31():
    dev = torch.device("cuda", 0)
    n = (1 << 31) + 5
    x = (torch.arange(n, device=dev, dtype=torch.int64) % 3).to(torch.float32)
    y = (torch.arange(n, device=dev, dtype=torch.int64) % 7 - 1).to(torch.float32)
    a = torch.zeros(1, dtype=torch.float32, device=dev)
    gb.dot(x, y, a, n)
    k = np.arange(21)
    period = float(((k % 3) * (k % 7 - 1)).sum())  # the pattern repeats every 21 (sum 42)
    q, r = divmod(n, 21)
    want = q * period + float(((k[:r] % 3) * (k[:r] % 7 - 1)).sum())
    assert a.item() == float(np.float32(want))  # the FP64 total rounded once to FP32
    del x, y
    torch.cuda.empty_cache()


def test_ger_past_2_31():
    dev = torch.device("cuda", 0)
    m, n = M, N
    C = torch.empty((m, n), dtype=torch.float32, device=dev)
    C[:] = row_pattern(m, dev)[:, None]
    x = (torch.arange(m, device=dev) % 3 - 1).to(torch.float32)
    y = (torch.arange(n, device=dev) % 4 - 2).to(torch.float32)
    gb.ger(x, y, C, 0.5, gb.ROW_MAJOR, m, n, n)
    # check every 97th row in full, and the last row
    rows = torch.cat([torch.arange(0, m, 97, device=dev), torch.tensor([m - 1], device=dev)])
    want = row_pattern(m, dev)[rows, None] + 0.5 * x[rows, None] * y[None, :]
    assert torch.equal(C[rows], want)
    del C
    torch.cuda.empty_cache()
