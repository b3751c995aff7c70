"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module holds no arithmetic of GEMV, DOT or GER.  It only turns
(seed, stream, index) into numbers, with one counter-based generator that
has two implementations which must agree bit for bit:

* ``numpy`` (host), used for small cases and for the oracle's inputs;
* ``libsynth.so`` (``synth.cu``, a CUDA kernel), used to fill large device
  buffers quickly.

Generator (SplitMix64 of Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014, used here as a hash of a
counter):

    mix(z)  = z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
              z ^= z >> 27; z *= 0x94D049BB133111EB; z ^ (z >> 31)
    key     = mix(mix(seed + G) ^ (stream * 0xD1B54A32D192ED03))
    u_k     = mix(key + (k + 1) * G)          G = 0x9E3779B97F4A7C15

all arithmetic modulo 2^64.  ``k`` is the linear element index (offset
included), so a sub-range of a large buffer can be regenerated on its own.

Value maps (all exact in the target type):

* uniform f64 in [-1, 1):  (u >> 11) * 2^-52 - 1
* uniform f32 in [-1, 1):  (u >> 40) * 2^-23 - 1
* integers in [lo, hi]:    lo + (((u >> 32) * (hi - lo + 1)) >> 32)
* normal rows (device only): Box-Muller on words 2k+1, 2k+2 of element k,
  times 10^(lo + (hi - lo) * u_i) per row, u_i from stream + 1
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

G = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)
S = np.uint64(0xD1B54A32D192ED03)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsynth.so")


def _mix(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * M1
    z = z ^ (z >> np.uint64(27))
    z = z * M2
    return z ^ (z >> np.uint64(31))


def key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        a = _mix(np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + G], dtype=np.uint64))
        b = np.array([np.uint64(stream & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64) * S
        return _mix(a ^ b)[0]


def raw(n: int, seed: int, stream: int, offset: int = 0) -> np.ndarray:
    """The uint64 words u_k for k in [offset, offset + n)."""
    k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key(seed, stream) + k * G)


def uniform(n: int, seed: int, stream: int, dtype=np.float64, offset: int = 0) -> np.ndarray:
    u = raw(n, seed, stream, offset)
    if np.dtype(dtype) == np.float64:
        return (u >> np.uint64(11)).astype(np.float64) * 2.0 ** -52 - 1.0
    if np.dtype(dtype) == np.float32:
        v = (u >> np.uint64(40)).astype(np.float32) * np.float32(2.0 ** -23)
        return (v - np.float32(1.0)).astype(np.float32)
    raise TypeError(dtype)


def integers(n: int, seed: int, stream: int, lo: int, hi: int, dtype=np.float64,
             offset: int = 0) -> np.ndarray:
    """Integer-valued numbers in [lo, hi] (inclusive), stored as ``dtype``."""
    u = raw(n, seed, stream, offset) >> np.uint64(32)
    span = np.uint64(hi - lo + 1)
    with np.errstate(over="ignore"):
        r = ((u * span) >> np.uint64(32)).astype(np.int64) + lo
    return r.astype(dtype)


# ----------------------------------------------------------------------------
# device fill (same numbers, written by a CUDA kernel)
# ----------------------------------------------------------------------------
_lib = None


def uniform_pairs(n: int, seed: int, stream: int, offset: int = 0) -> np.ndarray:
    """FP32 uniform in [-1, 1) with two elements per word (the serving
    engine's operands): element 2k takes bits 63..40 of u_k, element 2k+1
    bits 39..16, each b mapped to b * 2^-23 - 1 (exact)."""
    if n == 0:
        return np.zeros(0, np.float32)
    k = np.arange(offset, offset + n, dtype=np.int64)
    w0 = offset // 2
    u = raw((offset + n - 1) // 2 - w0 + 1, seed, stream, w0)[k // 2 - w0]
    b = np.where(k % 2 == 0, u >> np.uint64(40), (u >> np.uint64(16)) & np.uint64(0xFFFFFF))
    return (b.astype(np.float32) * np.float32(2.0 ** -23) - np.float32(1.0)).astype(np.float32)


def pool_offset(seed: int, stream: int, extent: int, pool_elems: int) -> int:
    """Start (elements) of a serving request's operand in a resident pool of
    pool_elems elements: 8 * (mix(key(seed, stream)) mod (floor((pool_elems
    - extent) / 8) + 1)), extent <= pool_elems."""
    with np.errstate(over="ignore"):
        h = int(_mix(np.array([key(seed, stream)], np.uint64))[0])
    return 8 * (h % ((pool_elems - extent) // 8 + 1))


def log_uniform_integers(n: int, seed: int, stream: int, lo: int, hi: int) -> np.ndarray:
    """round(exp(ln lo + u (ln hi - ln lo))) with u uniform in [0, 1): sizes
    spread evenly over the decades between lo and hi (int64)."""
    u = (uniform(n, seed, stream) + 1.0) * 0.5
    v = np.round(np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo))))
    return np.clip(v, lo, hi).astype(np.int64)


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build()")
        lib = ctypes.CDLL(LIB_PATH)
        for name in ("synth_uniform_f64", "synth_uniform_f32"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                          ctypes.c_int64, ctypes.c_void_p]
            f.restype = ctypes.c_int
        for name in ("synth_integers_f64", "synth_integers_f32"):
            f = getattr(lib, name)
            f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64,
                          ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
            f.restype = ctypes.c_int
        f = lib.synth_normal_rows_f32
        f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint64,
                      ctypes.c_uint64, ctypes.c_float, ctypes.c_float, ctypes.c_void_p]
        f.restype = ctypes.c_int
        _lib = lib
    return _lib


def fill_uniform(t, seed: int, stream: int, offset: int = 0) -> None:
    """Fill a contiguous CUDA tensor (float32/float64) with ``uniform`` values."""
    import torch
    assert t.is_cuda and t.is_contiguous()
    lib = _load()
    s = torch.cuda.current_stream(t.device).cuda_stream
    if t.dtype == torch.float64:
        rc = lib.synth_uniform_f64(t.data_ptr(), t.numel(), seed, stream, offset, s)
    elif t.dtype == torch.float32:
        rc = lib.synth_uniform_f32(t.data_ptr(), t.numel(), seed, stream, offset, s)
    else:
        raise TypeError(t.dtype)
    if rc != 0:
        raise RuntimeError(f"synth fill failed: cuda error {rc}")


def fill_integers(t, seed: int, stream: int, lo: int, hi: int, offset: int = 0) -> None:
    import torch
    assert t.is_cuda and t.is_contiguous()
    lib = _load()
    s = torch.cuda.current_stream(t.device).cuda_stream
    if t.dtype == torch.float64:
        rc = lib.synth_integers_f64(t.data_ptr(), t.numel(), seed, stream, offset, lo, hi, s)
    elif t.dtype == torch.float32:
        rc = lib.synth_integers_f32(t.data_ptr(), t.numel(), seed, stream, offset, lo, hi, s)
    else:
        raise TypeError(t.dtype)
    if rc != 0:
        raise RuntimeError(f"synth fill failed: cuda error {rc}")


def fill_normal_rows(t, seed: int, stream: int, lo: float = -3.0, hi: float = 3.0) -> None:
    """Fill a contiguous row-major 2-D float32 CUDA tensor with N(0,1) values
    (Box-Muller on two words per element) times a per-row scale
    10^(lo + (hi - lo) * u_i), u_i uniform in [0, 1) from stream + 1 (the
    reduced-precision GEMV workload: rows scaled log-uniformly)."""
    import torch
    assert t.is_cuda and t.is_contiguous() and t.dim() == 2 and t.dtype == torch.float32
    lib = _load()
    s = torch.cuda.current_stream(t.device).cuda_stream
    rc = lib.synth_normal_rows_f32(t.data_ptr(), t.shape[0], t.shape[1], seed, stream, lo, hi, s)
    if rc != 0:
        raise RuntimeError(f"synth fill failed: cuda error {rc}")


def build(nvcc: str = "nvcc") -> str:
    """Compile libsynth.so for sm_103a; returns its path."""
    import subprocess
    src = os.path.join(_HERE, "synth.cu")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-shared",
           "-Xcompiler", "-fPIC", "-o", LIB_PATH, src]
    subprocess.run(cmd, check=True)
    return LIB_PATH
