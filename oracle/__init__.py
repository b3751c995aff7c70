"""CPU oracle for GEMV / DOT / GER — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product path (the CUDA
library ``paper_2108_02025_gb300``) never imports it and shares no code with
it.

``oracle.c`` is the plain definition of each operation (Singh & Bassoy,
Sec. 3.1, Defs. DOT, GEM and GEMV) in FP64, in two forms: ``*_plain`` (index
order) and ``*_acc`` (compensated Dot2, the reference for tolerances).  This
module compiles it with gcc and wraps it with ctypes; arrays are numpy.
FP32 inputs are widened to FP64 here (exact) except for GER, which the oracle
computes in the working type because it is one rounding per element.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_HERE, "oracle.c")
LIB = os.path.join(_HERE, "liboracle.so")

ROW_MAJOR, COL_MAJOR = 0, 1

_lib = None


def build(cc: str = "gcc", src: str = SRC, out: str = LIB) -> str:
    """Compile the oracle (no fast-math, no FP contraction, OpenMP)."""
    cmd = [cc, "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True)
    return out


def _bind(lib):
    P, I64, D, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    for name in ("oracle_gemv_plain", "oracle_gemv_acc"):
        f = getattr(lib, name)
        f.argtypes = [I, I64, I64, D, P, I64, P, P]
        f.restype = None
    lib.oracle_gemv_scale.argtypes = [I, I64, I64, D, P, I64, P, P, P]
    lib.oracle_gemv_scale.restype = None
    for name in ("oracle_dot_plain", "oracle_dot_acc", "oracle_dot_scale"):
        f = getattr(lib, name)
        f.argtypes = [I64, P, P, D]
        f.restype = D
    lib.oracle_dger.argtypes = [I, I64, I64, D, P, P, P, I64]
    lib.oracle_dger.restype = None
    lib.oracle_sger.argtypes = [I, I64, I64, ctypes.c_float, P, P, P, I64]
    lib.oracle_sger.restype = None
    U8P = ctypes.POINTER(ctypes.c_uint8)
    lib.oracle_bf16_encode_array.argtypes = [I64, P, P]
    lib.oracle_bf16_encode_array.restype = None
    lib.oracle_e4m3_encode_array.argtypes = [I64, P, P]
    lib.oracle_e4m3_encode_array.restype = None
    lib.oracle_e4m3_decode_array.argtypes = [I64, P, P]
    lib.oracle_e4m3_decode_array.restype = None
    lib.oracle_quantize_e4m3_rows.argtypes = [I64, I64, P, I64, P, I64, P]
    lib.oracle_quantize_e4m3_rows.restype = None
    lib.oracle_threads.argtypes = []
    lib.oracle_threads.restype = I
    lib.oracle_set_threads.argtypes = [I]
    lib.oracle_set_threads.restype = None
    return lib


def load(path: str):
    """Bind an oracle shared library at ``path`` (used to test rebuilt copies)."""
    return Oracle(_bind(ctypes.CDLL(path)))


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
            build()
        _lib = _bind(ctypes.CDLL(LIB))
    return _lib


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check_matrix(layout, m, n, ld, size):
    if m > 0 and n > 0:
        need = (m - 1) * ld + n if layout == ROW_MAJOR else (n - 1) * ld + m
        if size < need:
            raise ValueError(f"matrix buffer of {size} elements is smaller than {need}")


class Oracle:
    """numpy-facing wrapper of one oracle library."""

    def __init__(self, lib=None):
        self._lib = lib

    @property
    def lib(self):
        return self._lib if self._lib is not None else _load()

    def threads(self) -> int:
        return self.lib.oracle_threads()

    def set_threads(self, t: int) -> None:
        self.lib.oracle_set_threads(int(t))

    def gemv(self, layout, m, n, alpha, A, lda, x, c, acc=True) -> np.ndarray:
        """Returns c + alpha*A*x in FP64 (A, x, c flat buffers; A with leading dim lda)."""
        A, x, out = _f64(A).ravel(), _f64(x).ravel(), _f64(c).ravel().copy()
        _check_matrix(layout, m, n, lda, A.size)
        assert x.size >= n and out.size >= m
        f = self.lib.oracle_gemv_acc if acc else self.lib.oracle_gemv_plain
        f(layout, m, n, float(alpha), _ptr(A), lda, _ptr(x), _ptr(out))
        return out

    def gemv_scale(self, layout, m, n, alpha, A, lda, x, c0) -> np.ndarray:
        """|c0_i| + |alpha| * sum_j |A_ij x_j| for every row i."""
        A, x, c0 = _f64(A).ravel(), _f64(x).ravel(), _f64(c0).ravel()
        _check_matrix(layout, m, n, lda, A.size)
        out = np.zeros(max(m, 0), dtype=np.float64)
        self.lib.oracle_gemv_scale(layout, m, n, float(alpha), _ptr(A), lda, _ptr(x), _ptr(c0),
                                   _ptr(out))
        return out

    def dot(self, n, x, y, alpha, acc=True) -> float:
        """Returns alpha + x.y in FP64."""
        x, y = _f64(x).ravel(), _f64(y).ravel()
        assert x.size >= n and y.size >= n
        f = self.lib.oracle_dot_acc if acc else self.lib.oracle_dot_plain
        return f(n, _ptr(x), _ptr(y), float(alpha))

    def dot_scale(self, n, x, y, alpha) -> float:
        x, y = _f64(x).ravel(), _f64(y).ravel()
        return self.lib.oracle_dot_scale(n, _ptr(x), _ptr(y), float(alpha))

    def ger(self, layout, m, n, alpha, x, y, C, ldc) -> np.ndarray:
        """Returns C + alpha * x y^T, one fma per element, in C's own type (f32/f64)."""
        C = np.asarray(C)
        dt = C.dtype
        if dt not in (np.float32, np.float64):
            raise TypeError(dt)
        out = np.ascontiguousarray(C).ravel().copy()
        x = np.ascontiguousarray(np.asarray(x), dtype=dt).ravel()
        y = np.ascontiguousarray(np.asarray(y), dtype=dt).ravel()
        _check_matrix(layout, m, n, ldc, out.size)
        assert x.size >= m and y.size >= n
        if dt == np.float64:
            self.lib.oracle_dger(layout, m, n, float(alpha), _ptr(x), _ptr(y), _ptr(out), ldc)
        else:
            self.lib.oracle_sger(layout, m, n, float(np.float32(alpha)), _ptr(x), _ptr(y),
                                 _ptr(out), ldc)
        return out

    # ---- reduced-precision storage of A (BF16, E4M3 with per-row scales)

    def bf16_encode(self, v) -> np.ndarray:
        """FP32 -> BF16 bits, round to nearest even."""
        v = np.ascontiguousarray(np.asarray(v), dtype=np.float32).ravel()
        q = np.empty(v.size, dtype=np.uint16)
        self.lib.oracle_bf16_encode_array(v.size, _ptr(v), _ptr(q))
        return q

    @staticmethod
    def bf16_decode(q) -> np.ndarray:
        """BF16 bits -> FP32 (exact)."""
        q = np.ascontiguousarray(np.asarray(q), dtype=np.uint16).ravel()
        return (q.astype(np.uint32) << np.uint32(16)).view(np.float32)

    def e4m3_encode(self, v) -> np.ndarray:
        """Real values -> E4M3 bits, round to nearest even, saturating at +-448."""
        v = _f64(v).ravel()
        q = np.empty(v.size, dtype=np.uint8)
        self.lib.oracle_e4m3_encode_array(v.size, _ptr(v), _ptr(q))
        return q

    def e4m3_decode(self, q) -> np.ndarray:
        q = np.ascontiguousarray(np.asarray(q), dtype=np.uint8).ravel()
        v = np.empty(q.size, dtype=np.float64)
        self.lib.oracle_e4m3_decode_array(q.size, _ptr(q), _ptr(v))
        return v

    def quantize_e4m3_rows(self, m, n, A, lda):
        """Row-major FP32 A -> (E4M3 bits with leading dimension n, FP32 scales)."""
        A = np.ascontiguousarray(np.asarray(A), dtype=np.float32).ravel()
        _check_matrix(ROW_MAJOR, m, n, lda, A.size)
        Q = np.zeros(max(m * n, 0), dtype=np.uint8)
        s = np.zeros(max(m, 0), dtype=np.float32)
        self.lib.oracle_quantize_e4m3_rows(m, n, _ptr(A), lda, _ptr(Q), n, _ptr(s))
        return Q, s


_default = Oracle()
threads = _default.threads
set_threads = _default.set_threads
gemv = _default.gemv
gemv_scale = _default.gemv_scale
dot = _default.dot
dot_scale = _default.dot_scale
ger = _default.ger
bf16_encode = _default.bf16_encode
bf16_decode = _default.bf16_decode
e4m3_encode = _default.e4m3_encode
e4m3_decode = _default.e4m3_decode
quantize_e4m3_rows = _default.quantize_e4m3_rows
