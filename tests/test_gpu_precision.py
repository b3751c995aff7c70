"""Reduced-precision storage of A (BF16; FP8 E4M3 with per-row FP32 scales)
on the GPU, against the CPU oracle's encoders (written from the format
definitions and pinned in tests/pins.py):

* quantisers: bit-exact codes and scales;
* decoding inside the GEMV: exact for every code;
* GEMV: against the FP64 oracle on the dequantised matrix, within 5e-6 of
  |c0| + |alpha| * s_i * sum_j |q_ij x_j| (FP32 products in chains of at most
  32, compensated FP32 sum); and, for the workload with rows scaled
  log-uniformly in [1e-3, 1e3], the total error against the FP64 oracle on
  the FP32 master matrix within the quantisation bound (BF16: 2^-9, E4M3:
  2^-4 of sum_j |A_ij x_j|, plus the E4M3 subnormal floor s_i 2^-10 sum |x_j|)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2108_02025_gb300 as gb
import synth

pytestmark = pytest.mark.gpu
TOL = 5e-6


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def specials_f32(n, seed):
    v = synth.uniform(n, seed, 1, np.float32) * np.float32(1e3)
    bits = synth.integers(n, seed, 2, 0, 2 ** 31 - 1, np.int64).astype(np.uint32)
    v[::7] = bits[::7].view(np.float32)                          # random bit patterns
    v[1::11] = ((bits[1::11] & np.uint32(0xFFFF0000)) | np.uint32(0x8000)).view(np.float32)  # ties
    v[2::13] = np.float32(1e-40)                                  # subnormal
    v[3::17] = -np.float32(3.4e38)
    v[:4] = [0.0, -0.0, np.inf, -np.inf]
    return v[np.isfinite(v) | np.isinf(v)]


def test_bf16_quantiser_bit_exact():
    v = specials_f32(100003, 3)
    v = v[~np.isnan(v)]
    m = 7
    n = v.size // m
    A = v[:m * n].reshape(m, n)
    Q = torch.empty((m, n), dtype=torch.int16, device="cuda")
    assert gb.gb_quantize_bf16(m, n, dev(A), n, Q, n) == gb.GB_OK
    torch.cuda.synchronize()
    assert np.array_equal(Q.cpu().numpy().view(np.uint16).ravel(), oracle.bf16_encode(A.ravel()))


@pytest.mark.parametrize("n", [1, 17, 1000, 40000])
def test_e4m3_quantiser_bit_exact(n):
    m = 9
    A = synth.uniform(m * n, 5, 1, np.float32).reshape(m, n)
    A[1] = 0.0
    A[2] *= np.float32(1e-30)
    A[3] *= np.float32(1e30)
    A[4, ::3] = 0.0
    A[5] = np.round(A[5] * 8) / 8                                  # many exact ties
    ldq = n + 3
    Q = torch.zeros((m, ldq), dtype=torch.uint8, device="cuda")
    s = torch.empty(m, dtype=torch.float32, device="cuda")
    assert gb.gb_quantize_e4m3(m, n, dev(A), n, Q, ldq, s) == gb.GB_OK
    torch.cuda.synchronize()
    Qo, so = oracle.quantize_e4m3_rows(m, n, A.ravel(), n)
    assert np.array_equal(s.cpu().numpy(), so)
    assert np.array_equal(Q.cpu().numpy()[:, :n], Qo.reshape(m, n))


def test_e4m3_decoding_in_gemv_is_exact():
    """Row r holds code r in column 0 (all finite codes), x = e_0, scales 1:
    c_r = decode(code r) exactly."""
    codes = np.array([c for c in range(256) if c not in (0x7F, 0xFF)], dtype=np.uint8)
    m, n = codes.size, 16
    Q = np.zeros((m, n), dtype=np.uint8)
    Q[:, 0] = codes
    x = np.zeros(n, np.float32)
    x[0] = 1.0
    c = torch.zeros(m, dtype=torch.float32, device="cuda")
    nb = gb.gb_workspace_bytes(gb.OP_GEMV_E4M3, 0, gb.ROW_MAJOR, m, n)
    ws = torch.zeros(max(nb, 1), dtype=torch.uint8, device="cuda")
    st = gb.gb_gemv_e4m3(m, n, 1.0, dev(Q), n, dev(np.ones(m, np.float32)), dev(x), c, ws, nb)
    assert st == gb.GB_OK
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy().astype(np.float64), oracle.e4m3_decode(codes))


def test_bf16_decoding_in_gemv_is_exact():
    codes = np.arange(65536, dtype=np.uint32)
    vals = (codes << np.uint32(16)).view(np.float32)
    keep = np.isfinite(vals)
    codes = codes[keep].astype(np.uint16)
    m, n = codes.size, 8
    Q = np.zeros((m, n), dtype=np.uint16)
    Q[:, 0] = codes
    x = np.zeros(n, np.float32)
    x[0] = 1.0
    c = torch.zeros(m, dtype=torch.float32, device="cuda")
    nb = gb.gb_workspace_bytes(gb.OP_GEMV_BF16, 0, gb.ROW_MAJOR, m, n)
    ws = torch.zeros(max(nb, 1), dtype=torch.uint8, device="cuda")
    assert gb.gb_gemv_bf16(m, n, 1.0, dev(Q.view(np.int16)), n, dev(x), c, ws, nb) == gb.GB_OK
    torch.cuda.synchronize()
    assert np.array_equal(c.cpu().numpy(), oracle.bf16_decode(codes))


def run_q(fmt, A, x, c0, alpha):
    m, n = A.shape
    dA = dev(A)
    Q, s = gb.quantize(dA, fmt)
    c = dev(c0)
    gb.gemv_q(Q, s, dev(x), c, alpha, n=n)
    torch.cuda.synchronize()
    Qh = Q.cpu().numpy()
    if fmt == "bf16":
        deq = oracle.bf16_decode(Qh.view(np.uint16)[:, :n].ravel()).astype(np.float64).reshape(m, n)
    else:
        sh = s.cpu().numpy().astype(np.float64)
        deq = oracle.e4m3_decode(Qh[:, :n].ravel()).reshape(m, n) * sh[:, None]
    return c.cpu().numpy().astype(np.float64), deq


SHAPES = [(1, 1), (5, 17), (1000, 777), (64, 200003), (3000, 4096), (33, 50000)]


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
@pytest.mark.parametrize("shape", SHAPES, ids=[f"{m}x{n}" for m, n in SHAPES])
def test_gemv_against_dequantised_oracle(fmt, shape):
    m, n = shape
    A = synth.uniform(m * n, 7, 1, np.float32).reshape(m, n) * np.float32(3.0)
    x = synth.uniform(n, 7, 2, np.float32)
    c0 = synth.uniform(m, 7, 3, np.float32)
    got, deq = run_q(fmt, A, x, c0, 0.75)
    want = oracle.gemv(0, m, n, 0.75, deq.ravel(), n, x, c0)
    scale = oracle.gemv_scale(0, m, n, 0.75, deq.ravel(), n, x, c0)
    err = np.max(np.abs(got - want) / scale)
    assert err <= TOL, (fmt, shape, err)


@pytest.mark.parametrize("fmt", ["bf16", "e4m3"])
def test_gemv_twice_bit_identical(fmt):
    m, n = 64, 200003
    A = dev(synth.uniform(m * n, 8, 1, np.float32).reshape(m, n))
    x = dev(synth.uniform(n, 8, 2, np.float32))
    Q, s = gb.quantize(A, fmt)
    r = []
    for _ in range(2):
        c = torch.zeros(m, dtype=torch.float32, device="cuda")
        gb.gemv_q(Q, s, x, c, 1.0, n=n)
        r.append(c.cpu().numpy())
    assert np.array_equal(r[0], r[1])


@pytest.mark.parametrize("fmt,bound", [("bf16", 2.0 ** -9), ("e4m3", 2.0 ** -4)])
def test_rows_scaled_log_uniform_error_budget(fmt, bound):
    """A = N(0,1) with row i scaled by 10^U[-3,3] (the reduced-precision
    workload's recipe), 4096 x 4096: kernel vs dequantised oracle within TOL,
    and total vs the FP64 oracle on the FP32 master within the format's
    quantisation bound."""
    m = n = 4096
    A = torch.empty((m, n), dtype=torch.float32, device="cuda")
    synth.fill_normal_rows(A, 9, 1, -3.0, 3.0)
    xh = synth.uniform(n, 9, 3, np.float32)
    c0 = np.zeros(m, np.float32)
    Ah = A.cpu().numpy()
    got, deq = run_q(fmt, Ah, xh, c0, 1.0)
    want_q = oracle.gemv(0, m, n, 1.0, deq.ravel(), n, xh, c0)
    scale_q = oracle.gemv_scale(0, m, n, 1.0, deq.ravel(), n, xh, c0)
    assert np.max(np.abs(got - want_q) / scale_q) <= TOL
    want = oracle.gemv(0, m, n, 1.0, Ah.ravel(), n, xh, c0)
    scale = oracle.gemv_scale(0, m, n, 1.0, Ah.ravel(), n, xh, c0)
    floor = 0.0
    if fmt == "e4m3":
        floor = (np.abs(Ah).max(axis=1) / 448.0) * 2.0 ** -10 * np.abs(xh.astype(np.float64)).sum()
    assert np.all(np.abs(got - want) <= bound * scale + floor + TOL * scale)


@pytest.mark.parametrize("fmt,bound", [("bf16", 2.0 ** -9), ("e4m3", 2.0 ** -4)])
def test_full_size_32768_sampled_rows(fmt, bound):
    """The benchmark's reduced-precision workload and launch: A 32768 x 32768
    (N(0,1), rows scaled by 10^U[-3,3]) quantised on the GPU, one GEMV; 48
    seeded rows against the FP64 oracle on their decoded codes (kernel
    arithmetic, TOL) and on the FP32 master (quantisation bound)."""
    m = n = 32768
    A = torch.empty((m, n), dtype=torch.float32, device="cuda")
    synth.fill_normal_rows(A, 10, 1, -3.0, 3.0)
    xh = synth.uniform(n, 10, 3, np.float32)
    c0 = synth.uniform(m, 10, 4, np.float32)
    rows = np.unique(synth.integers(48, 10, 5, 0, m - 1, np.int64))
    idx = torch.from_numpy(rows).cuda()
    Ar = A[idx].cpu().numpy()
    Q, s = gb.quantize(A, fmt)
    del A
    c = dev(c0)
    gb.gemv_q(Q, s, dev(xh), c, 0.5, n=n)
    got = c[idx].cpu().numpy().astype(np.float64)
    Qr = Q[idx].cpu().numpy()
    if fmt == "bf16":
        deq = oracle.bf16_decode(Qr.view(np.uint16)[:, :n].ravel()).astype(np.float64).reshape(-1, n)
    else:
        deq = oracle.e4m3_decode(Qr[:, :n].ravel()).reshape(-1, n) * s[idx].cpu().numpy().astype(np.float64)[:, None]
    k = rows.size
    c0r = c0[rows]
    want_q = oracle.gemv(0, k, n, 0.5, deq.ravel(), n, xh, c0r)
    scale_q = oracle.gemv_scale(0, k, n, 0.5, deq.ravel(), n, xh, c0r)
    assert np.max(np.abs(got - want_q) / scale_q) <= TOL
    want = oracle.gemv(0, k, n, 0.5, Ar.ravel(), n, xh, c0r)
    scale = oracle.gemv_scale(0, k, n, 0.5, Ar.ravel(), n, xh, c0r)
    floor = 0.0
    if fmt == "e4m3":
        floor = 0.5 * (np.abs(Ar).max(axis=1) / 448.0) * 2.0 ** -10 * np.abs(xh.astype(np.float64)).sum()
    assert np.all(np.abs(got - want) <= bound * scale + floor + TOL * scale)
    del Q, s
    torch.cuda.empty_cache()
