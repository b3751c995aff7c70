"""Python binding of libgbblas.so — GEMV, DOT and GER on one GB300 (sm_103a).

The functions ``gb_*`` have the names and argument order of the C ABI in
``include/gbblas.h`` and only marshal arguments: tensors become device
pointers, a ``torch.cuda.Stream`` becomes its handle, and the C status code
is returned unchanged.  ``gemv``, ``dot`` and ``ger`` are convenience calls
over them that pick the dtype variant, hold a zeroed workspace per device
and stream, and raise ``GbError`` on a non-zero status; ``quantize`` and
``gemv_q`` do the same for BF16 / E4M3 storage of A.  ``Batch`` plans and
launches many GEMVs (and GERs) as one persistent kernel, optionally from a
CUDA graph (``include/gbblas.h``, batched API), and ``Engine`` drives the
serving engine of ``include/gbserve.h`` (continuous batching under an HBM
budget, resident operand pools, row chunks).

The library must be built (``__graft_entry__.build()`` or
``python paper_2108_02025_gb300/build.py``); importing this package without
it raises.  There is no CPU implementation: every operation runs in the
library's kernels on the GPU.
"""
from __future__ import annotations

import ctypes
import os
import threading

# GBBLAS_LIB overrides where the library is loaded from.
LIB_PATH = os.environ.get("GBBLAS_LIB", os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                     "libgbblas.so"))

ROW_MAJOR, COL_MAJOR = 0, 1
OP_GEMV, OP_DOT, OP_GER, OP_GEMV_BF16, OP_GEMV_E4M3 = 0, 1, 2, 3, 4
F32, F64 = 0, 1

GB_OK = 0
GB_ERR_WORKSPACE = -100
GB_ERR_UNSUPPORTED = -101
GB_ERR_CUDA = -102
GB_ERR_INJECTED = -103


class GbError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: status {status} ({gb_status_string(status)})")
        self.status = status


def _load() -> ctypes.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() "
                          "(there is no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    I, I64, P, SZ = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_size_t
    D, F = ctypes.c_double, ctypes.c_float
    lib.gb_version.argtypes, lib.gb_version.restype = [], I
    lib.gb_status_string.argtypes, lib.gb_status_string.restype = [I], ctypes.c_char_p
    lib.gb_workspace_bytes.argtypes, lib.gb_workspace_bytes.restype = [I, I, I, I64, I64], SZ
    lib.gb_workspace_init.argtypes, lib.gb_workspace_init.restype = [P, SZ, P], I
    lib.gb_copy_to_host.argtypes, lib.gb_copy_to_host.restype = [P, P, SZ, P], I
    lib.gb_dgemv.argtypes = [I, I64, I64, D, P, I64, P, P, P, SZ, P]
    lib.gb_sgemv.argtypes = [I, I64, I64, F, P, I64, P, P, P, SZ, P]
    lib.gb_ddot.argtypes = [I64, P, P, P, P, SZ, P]
    lib.gb_sdot.argtypes = [I64, P, P, P, P, SZ, P]
    lib.gb_dger.argtypes = [I, I64, I64, D, P, P, P, I64, P]
    lib.gb_sger.argtypes = [I, I64, I64, F, P, P, P, I64, P]
    lib.gb_dgemv_noalloc.argtypes = [I, I64, I64, D, P, I64, P, P, P]
    lib.gb_quantize_bf16.argtypes = [I64, I64, P, I64, P, I64, P]
    lib.gb_quantize_e4m3.argtypes = [I64, I64, P, I64, P, I64, P, P]
    lib.gb_gemv_bf16.argtypes = [I64, I64, F, P, I64, P, P, P, SZ, P]
    lib.gb_gemv_e4m3.argtypes = [I64, I64, F, P, I64, P, P, P, P, SZ, P]
    lib.gb_sgemv_batch_default_tuning.argtypes = [P]
    lib.gb_sgemv_batch_default_tuning.restype = None
    lib.gb_sgemv_batch_plan_bytes.argtypes = [I64, P, P, P, P]
    lib.gb_sgemv_batch_plan_bytes.restype = SZ
    lib.gb_sgemv_batch_plan.argtypes = [I64, P, P, P, P, P, P, P, P, P, SZ]
    lib.gb_sgemv_batch.argtypes = [P, P, P]
    lib.gb_sgemv_batch_tiles.argtypes, lib.gb_sgemv_batch_tiles.restype = [P], I64
    lib.gb_batch_plan_bytes.argtypes, lib.gb_batch_plan_bytes.restype = [I64, P, P], SZ
    lib.gb_batch_plan.argtypes, lib.gb_batch_plan.restype = [I64, P, P, P, SZ], I
    for name in ("gb_dgemv", "gb_sgemv", "gb_ddot", "gb_sdot", "gb_dger", "gb_sger",
                 "gb_dgemv_noalloc", "gb_quantize_bf16", "gb_quantize_e4m3", "gb_gemv_bf16",
                 "gb_gemv_e4m3", "gb_sgemv_batch_plan", "gb_sgemv_batch"):
        getattr(lib, name).restype = I
    # serving engine (include/gbserve.h)
    lib.gb_engine_now_ns.argtypes, lib.gb_engine_now_ns.restype = [], I64
    lib.gb_engine_create.argtypes, lib.gb_engine_create.restype = [P, P], I
    lib.gb_engine_submit.argtypes, lib.gb_engine_submit.restype = [P, P], I
    lib.gb_engine_poll.argtypes, lib.gb_engine_poll.restype = [P, P, I], I
    lib.gb_engine_drain.argtypes, lib.gb_engine_drain.restype = [P, I64], I
    lib.gb_engine_stats_get.argtypes, lib.gb_engine_stats_get.restype = [P, P], I
    lib.gb_engine_request_bytes.argtypes, lib.gb_engine_request_bytes.restype = [P], SZ
    lib.gb_engine_destroy.argtypes, lib.gb_engine_destroy.restype = [P], None
    return lib


_lib = _load()

# Every symbol the header declares (checked by the tests against include/gbblas.h).
EXPORTS = ("gb_version", "gb_status_string", "gb_workspace_bytes", "gb_workspace_init", "gb_copy_to_host",
           "gb_dgemv", "gb_sgemv", "gb_ddot", "gb_sdot", "gb_dger", "gb_sger",
           "gb_dgemv_noalloc", "gb_quantize_bf16", "gb_quantize_e4m3", "gb_gemv_bf16",
           "gb_gemv_e4m3", "gb_sgemv_batch_default_tuning", "gb_sgemv_batch_plan_bytes",
           "gb_sgemv_batch_plan", "gb_sgemv_batch", "gb_sgemv_batch_tiles", "gb_batch_plan_bytes",
           "gb_batch_plan")


# Every symbol include/gbserve.h declares.
ENGINE_EXPORTS = ("gb_engine_now_ns", "gb_engine_create", "gb_engine_submit", "gb_engine_poll",
                  "gb_engine_drain", "gb_engine_stats_get", "gb_engine_request_bytes",
                  "gb_engine_destroy")


def lib() -> ctypes.CDLL:
    return _lib


# ------------------------------------------------------------ marshalling --

def _ptr(t) -> int | None:
    """Device pointer of a tensor, or an int passed through (None = NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(s) -> int | None:
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ------------------------------------------------------------------ C ABI --

def gb_version() -> int:
    return _lib.gb_version()


def gb_status_string(status: int) -> str:
    return _lib.gb_status_string(status).decode()


def gb_workspace_bytes(op: int, dtype: int, layout: int, m: int, n: int) -> int:
    return _lib.gb_workspace_bytes(op, dtype, layout, m, n)


def gb_workspace_init(ws, ws_bytes: int, stream=None) -> int:
    return _lib.gb_workspace_init(_ptr(ws), ws_bytes, _stream(stream))


def gb_copy_to_host(dst, src, nbytes: int, stream=None) -> int:
    return _lib.gb_copy_to_host(_ptr(dst), _ptr(src), nbytes, _stream(stream))


def gb_dgemv(layout, m, n, alpha, A, lda, x, c, ws, ws_bytes, stream=None) -> int:
    return _lib.gb_dgemv(layout, m, n, alpha, _ptr(A), lda, _ptr(x), _ptr(c), _ptr(ws), ws_bytes,
                         _stream(stream))


def gb_sgemv(layout, m, n, alpha, A, lda, x, c, ws, ws_bytes, stream=None) -> int:
    return _lib.gb_sgemv(layout, m, n, alpha, _ptr(A), lda, _ptr(x), _ptr(c), _ptr(ws), ws_bytes,
                         _stream(stream))


def gb_ddot(n, x, y, alpha, ws, ws_bytes, stream=None) -> int:
    return _lib.gb_ddot(n, _ptr(x), _ptr(y), _ptr(alpha), _ptr(ws), ws_bytes, _stream(stream))


def gb_sdot(n, x, y, alpha, ws, ws_bytes, stream=None) -> int:
    return _lib.gb_sdot(n, _ptr(x), _ptr(y), _ptr(alpha), _ptr(ws), ws_bytes, _stream(stream))


def gb_dger(layout, m, n, alpha, x, y, C, ldc, stream=None) -> int:
    return _lib.gb_dger(layout, m, n, alpha, _ptr(x), _ptr(y), _ptr(C), ldc, _stream(stream))


def gb_sger(layout, m, n, alpha, x, y, C, ldc, stream=None) -> int:
    return _lib.gb_sger(layout, m, n, alpha, _ptr(x), _ptr(y), _ptr(C), ldc, _stream(stream))


def gb_quantize_bf16(m, n, A, lda, Q, ldq, stream=None) -> int:
    return _lib.gb_quantize_bf16(m, n, _ptr(A), lda, _ptr(Q), ldq, _stream(stream))


def gb_quantize_e4m3(m, n, A, lda, Q, ldq, scales, stream=None) -> int:
    return _lib.gb_quantize_e4m3(m, n, _ptr(A), lda, _ptr(Q), ldq, _ptr(scales), _stream(stream))


def gb_gemv_bf16(m, n, alpha, Q, ldq, x, c, ws, ws_bytes, stream=None) -> int:
    return _lib.gb_gemv_bf16(m, n, alpha, _ptr(Q), ldq, _ptr(x), _ptr(c), _ptr(ws), ws_bytes,
                             _stream(stream))


def gb_gemv_e4m3(m, n, alpha, Q, ldq, scales, x, c, ws, ws_bytes, stream=None) -> int:
    return _lib.gb_gemv_e4m3(m, n, alpha, _ptr(Q), ldq, _ptr(scales), _ptr(x), _ptr(c), _ptr(ws),
                             ws_bytes, _stream(stream))


def gb_dgemv_noalloc(layout, m, n, alpha, A, lda, x, c, stream=None) -> int:
    """gb_dgemv with the library's own scratch array instead of a workspace,
    for callers that cannot allocate device memory."""
    return _lib.gb_dgemv_noalloc(layout, m, n, alpha, _ptr(A), lda, _ptr(x), _ptr(c),
                                 _stream(stream))


# ------------------------------------------------------- batched GEMV ----

BATCH_BUCKETS = 32


class BatchTuning(ctypes.Structure):
    """One entry of the batched GEMV tuning table (gb_batch_tuning)."""
    _fields_ = [("lanes_per_row", ctypes.c_int32), ("packs_per_iter", ctypes.c_int32),
                ("tile_bytes", ctypes.c_int32), ("reserved", ctypes.c_int32)]


TuningTable = BatchTuning * BATCH_BUCKETS
BATCH_GEMV_F32, BATCH_GEMV_BF16, BATCH_GER_F32, BATCH_DOT_F32 = 0, 1, 2, 3


class BatchItem(ctypes.Structure):
    """gb_batch_item: A = the matrix (GEMV A or BF16 codes; GER C), x = the
    n-vector (GEMV x; GER y), c = the m-vector (GEMV c; GER x)."""
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("m", ctypes.c_int64),
                ("n", ctypes.c_int64), ("lda", ctypes.c_int64), ("alpha", ctypes.c_float),
                ("reserved2", ctypes.c_int32), ("A", ctypes.c_void_p), ("x", ctypes.c_void_p),
                ("c", ctypes.c_void_p)]


def gb_batch_plan_bytes(count, items, table=None) -> int:
    return _lib.gb_batch_plan_bytes(count, _addr(items), _addr(table))


def gb_batch_plan(count, items, table, plan, plan_bytes) -> int:
    return _lib.gb_batch_plan(count, _addr(items), _addr(table), _addr(plan), plan_bytes)


def _addr(buf) -> int | None:
    """Address of a ctypes object, a numpy array or an int (None = NULL)."""
    if buf is None or isinstance(buf, int):
        return buf
    if hasattr(buf, "ctypes"):
        return buf.ctypes.data
    return ctypes.addressof(buf)


def gb_sgemv_batch_default_tuning(table) -> None:
    _lib.gb_sgemv_batch_default_tuning(_addr(table))


def gb_sgemv_batch_plan_bytes(count, m, n, alpha, table=None) -> int:
    """m, n: int64 host arrays; alpha: float32 host array (numpy or addresses)."""
    return _lib.gb_sgemv_batch_plan_bytes(count, _addr(m), _addr(n), _addr(alpha), _addr(table))


def gb_sgemv_batch_plan(count, m, n, lda, alpha, A, x, c, table, plan, plan_bytes) -> int:
    """m, n, lda int64, alpha float32, A/x/c uint64 (device addresses): host
    arrays; plan: host buffer (numpy uint8 array or address)."""
    return _lib.gb_sgemv_batch_plan(count, _addr(m), _addr(n), _addr(lda), _addr(alpha), _addr(A),
                                    _addr(x), _addr(c), _addr(table), _addr(plan), plan_bytes)


def gb_sgemv_batch(plan_host, plan_dev, stream=None) -> int:
    return _lib.gb_sgemv_batch(_addr(plan_host), _ptr(plan_dev), _stream(stream))


def gb_sgemv_batch_tiles(plan_host) -> int:
    return _lib.gb_sgemv_batch_tiles(_addr(plan_host))


def tuning_table(entries=None):
    """A ctypes tuning table: the built-in one, overridden bucket by bucket by
    ``entries`` ({bucket: (lanes_per_row, packs_per_iter, tile_bytes)})."""
    t = TuningTable()
    gb_sgemv_batch_default_tuning(t)
    for b, (lpr, u, tb) in (entries or {}).items():
        t[int(b)] = BatchTuning(int(lpr), int(u), int(tb), 0)
    return t


TUNING_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "batch_tuning.json")


def load_tuning(path: str | None = None):
    """The table written by the autotuner (``batch_tuning.json`` beside this
    file), or the built-in table when there is none."""
    import json
    path = TUNING_PATH if path is None else path
    if not os.path.exists(path):
        return tuning_table()
    with open(path) as f:
        d = json.load(f)
    return tuning_table({int(b): tuple(v) for b, v in d["buckets"].items()})


def _aligned_host(nbytes):
    import numpy as np
    raw = np.zeros(nbytes + 16, np.uint8)
    off = (-raw.ctypes.data) % 16
    return raw[off:off + nbytes]


class Batch:
    """A planned batch of FP32 row-major GEMVs c_p += alpha_p A_p x_p, run by
    one persistent launch (``launch``) or by replaying a captured CUDA graph
    of that launch (``capture`` then ``replay``).  ``problems`` is a list of
    (A, x, c, alpha) with A a 2-D CUDA tensor (unit column stride) or
    (A, x, c, alpha, m, n, lda) with A any tensor or device address."""

    def __init__(self, problems, table=None, device=None):
        import numpy as np
        import torch
        count = len(problems)
        m = np.zeros(count, np.int64)
        n = np.zeros(count, np.int64)
        lda = np.zeros(count, np.int64)
        alpha = np.zeros(count, np.float32)
        A = np.zeros(count, np.uint64)
        x = np.zeros(count, np.uint64)
        c = np.zeros(count, np.uint64)
        for i, pr in enumerate(problems):
            if len(pr) == 4:
                a, xv, cv, al = pr
                mi, ni = a.shape
                ld = a.stride(0) if mi > 1 else max(1, ni)
            else:
                a, xv, cv, al, mi, ni, ld = pr
            m[i], n[i], lda[i], alpha[i] = mi, ni, ld, al
            A[i], x[i], c[i] = _ptr(a) or 0, _ptr(xv) or 0, _ptr(cv) or 0
        self.table = tuning_table() if table is None else table
        nb = gb_sgemv_batch_plan_bytes(count, m, n, alpha, self.table)
        if nb == 0:
            raise GbError(-1, "sgemv_batch_plan_bytes")
        self.host = _aligned_host(nb)
        _check(gb_sgemv_batch_plan(count, m, n, lda, alpha, A, x, c, self.table, self.host, nb),
               "sgemv_batch_plan")
        self._upload(count, device)

    @classmethod
    def from_items(cls, items, table=None, device=None):
        """A mixed batch: ``items`` is a list of (kind, A, x, c, alpha, m, n, lda)
        with the gb_batch_item meaning of A, x and c (tensors or addresses)."""
        self = cls.__new__(cls)
        arr = (BatchItem * max(1, len(items)))()
        for i, (kind, a, xv, cv, al, mi, ni, ld) in enumerate(items):
            arr[i] = BatchItem(kind, 0, mi, ni, ld, al, 0, _ptr(a) or 0, _ptr(xv) or 0, _ptr(cv) or 0)
        self.table = tuning_table() if table is None else table
        nb = gb_batch_plan_bytes(len(items), arr, self.table)
        if nb == 0:
            raise GbError(-2, "batch_plan_bytes")
        self.host = _aligned_host(nb)
        _check(gb_batch_plan(len(items), arr, self.table, self.host, nb), "batch_plan")
        self._upload(len(items), device)
        return self

    def _upload(self, count, device):
        import torch
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.dev = torch.from_numpy(self.host.copy()).to(dev)
        torch.cuda.synchronize(dev)
        self.tiles = gb_sgemv_batch_tiles(self.host)
        self.count = count
        self.graph = None

    def launch(self, stream=None) -> None:
        _check(gb_sgemv_batch(self.host, self.dev, stream), "sgemv_batch")

    def capture(self, stream=None) -> None:
        """Capture one launch into a CUDA graph (torch.cuda.CUDAGraph)."""
        import torch
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream(self.dev.device) if stream is None else stream
        s.wait_stream(torch.cuda.current_stream(self.dev.device))
        with torch.cuda.graph(g, stream=s):
            self.launch(torch.cuda.current_stream(self.dev.device))
        self.graph = g

    def replay(self) -> None:
        self.graph.replay()


# -------------------------------------------------------- serving engine --

GB_ERR_BUDGET = -104
GB_ERR_TIMEOUT = -105
REQ_GEMV, REQ_DOT, REQ_GER = 0, 1, 2
FORM_F32, FORM_BF16 = 0, 1
ENGINE_HOST_ONLY = 1
REQ_POOL = 1


class EngineConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_size_t), ("streams", ctypes.c_int32),
                ("max_inflight", ctypes.c_int32), ("max_step_requests", ctypes.c_int32),
                ("flags", ctypes.c_int32), ("sim_bytes_per_ns", ctypes.c_double),
                ("table", ctypes.c_void_p), ("pool_elems", ctypes.c_int64), ("pool_seed", ctypes.c_uint64),
                ("chunk_bytes", ctypes.c_size_t)]


class Request(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("op", ctypes.c_int32), ("form", ctypes.c_int32),
                ("m", ctypes.c_int64), ("n", ctypes.c_int64), ("alpha", ctypes.c_float),
                ("flags", ctypes.c_int32), ("seed", ctypes.c_uint64), ("out", ctypes.c_void_p),
                ("arrival_ns", ctypes.c_int64)]


class Completion(ctypes.Structure):
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int32), ("op", ctypes.c_int32),
                ("arrival_ns", ctypes.c_int64), ("admitted_ns", ctypes.c_int64),
                ("launched_ns", ctypes.c_int64), ("done_ns", ctypes.c_int64),
                ("step", ctypes.c_int64), ("bytes", ctypes.c_int64)]


class EngineStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("failed", ctypes.c_int64), ("steps", ctypes.c_int64),
                ("inflight_peak", ctypes.c_int64), ("steps_inflight_peak", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_size_t), ("bytes_peak", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t), ("pool_bytes", ctypes.c_size_t)]


def gb_engine_now_ns() -> int:
    return _lib.gb_engine_now_ns()


def gb_engine_create(cfg, out) -> int:
    return _lib.gb_engine_create(_addr(cfg), _addr(out))


def gb_engine_submit(engine, request) -> int:
    return _lib.gb_engine_submit(engine, _addr(request))


def gb_engine_poll(engine, out, max_count) -> int:
    return _lib.gb_engine_poll(engine, _addr(out), max_count)


def gb_engine_drain(engine, timeout_ms) -> int:
    return _lib.gb_engine_drain(engine, timeout_ms)


def gb_engine_stats_get(engine, out) -> int:
    return _lib.gb_engine_stats_get(engine, _addr(out))


def gb_engine_request_bytes(request) -> int:
    return _lib.gb_engine_request_bytes(_addr(request))


def gb_engine_destroy(engine) -> None:
    _lib.gb_engine_destroy(engine)


class Engine:
    """The serving engine (continuous batching under an HBM budget).

    ``submit`` queues a request (op, m, n, alpha, seed, optional pinned host
    tensor for the result, arrival time on ``now_ns``'s clock); ``drain``
    waits for all of them; ``poll`` returns the completions as dicts.  With
    ``pool_elems`` > 0 the engine keeps resident operand pools and requests
    submitted with ``pool=True`` read their inputs from them."""

    def __init__(self, budget_bytes, streams=4, max_inflight=4096, max_step_requests=256,
                 host_only=False, sim_bytes_per_ns=1000.0, table=None, pool_elems=0, pool_seed=0,
                 chunk_bytes=0):
        self.table = table
        cfg = EngineConfig(budget_bytes, streams, max_inflight, max_step_requests,
                           ENGINE_HOST_ONLY if host_only else 0, sim_bytes_per_ns,
                           _addr(table) if table is not None else None, pool_elems, pool_seed, chunk_bytes)
        h = ctypes.c_void_p()
        _check(gb_engine_create(cfg, ctypes.addressof(h)), "engine_create")
        self.h = h.value
        self._keep = {}

    @staticmethod
    def now_ns() -> int:
        return gb_engine_now_ns()

    def submit(self, rid, op, m, n, alpha=1.0, seed=0, out=None, arrival_ns=0, form=FORM_F32,
               pool=False) -> int:
        """Returns the status (GB_OK, -2 invalid, GB_ERR_BUDGET)."""
        r = Request(rid, op, form, m, n, alpha, REQ_POOL if pool else 0, seed, _ptr(out), arrival_ns)
        st = gb_engine_submit(self.h, ctypes.addressof(r))
        if st == GB_OK and out is not None:
            self._keep[rid] = out  # the engine writes into it later
        return st

    def drain(self, timeout_ms=60000) -> int:
        return gb_engine_drain(self.h, timeout_ms)

    def poll(self, max_count=1 << 16):
        buf = (Completion * max_count)()
        k = gb_engine_poll(self.h, buf, max_count)
        if k < 0:
            raise GbError(k, "engine_poll")
        out = []
        for c in buf[:k]:
            out.append({f: getattr(c, f) for f, _ in Completion._fields_})
            self._keep.pop(c.id, None)
        return out

    def stats(self) -> dict:
        s = EngineStats()
        _check(gb_engine_stats_get(self.h, ctypes.addressof(s)), "engine_stats")
        return {f: getattr(s, f) for f, _ in EngineStats._fields_}

    def close(self) -> None:
        if self.h:
            gb_engine_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def request_bytes(op, m, n, form=FORM_F32, pool=False) -> int:
    r = Request(0, op, form, m, n, 1.0, REQ_POOL if pool else 0, 0, None, 0)
    return gb_engine_request_bytes(ctypes.addressof(r))


# ---------------------------------------------------------- convenience ----

_ws_lock = threading.Lock()
_ws_cache: dict = {}


def workspace(nbytes: int, device=None, stream=None):
    """A zero-filled uint8 device buffer of at least ``nbytes`` for ``stream``,
    kept and reused by later calls on the same (device, stream)."""
    import torch
    if nbytes <= 0:
        return None
    dev = torch.device("cuda", torch.cuda.current_device() if device is None else
                       torch.device(device).index or 0)
    key = (dev.index, _stream(stream))
    with _ws_lock:
        buf = _ws_cache.get(key)
        if buf is None or buf.numel() < nbytes:
            buf = torch.zeros(max(nbytes, 1 << 16), dtype=torch.uint8, device=dev)
            _ws_cache[key] = buf
    return buf


def _dtype_code(t) -> int:
    import torch
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _check(status: int, what: str) -> None:
    if status != GB_OK:
        raise GbError(status, what)


def gemv(A, x, c, alpha: float = 1.0, layout: int = ROW_MAJOR, m: int | None = None,
         n: int | None = None, lda: int | None = None, stream=None) -> None:
    """c += alpha * A @ x in place.  ``A`` is a 2-D CUDA tensor in its own
    memory order (row-major: stride (lda, 1); column-major: stride (1, lda)),
    or a flat buffer with m, n, lda given."""
    if A.dim() == 2 and m is None:
        m, n = A.shape
        if layout == ROW_MAJOR:
            assert A.stride(1) == 1 or n <= 1, "row-major A needs unit column stride"
            lda = A.stride(0) if m > 1 else max(1, n)
        else:
            assert A.stride(0) == 1 or m <= 1, "column-major A needs unit row stride"
            lda = A.stride(1) if n > 1 else max(1, m)
    dt = _dtype_code(A)
    nb = gb_workspace_bytes(OP_GEMV, dt, layout, m, n)
    ws = workspace(nb, A.device, stream)
    f = gb_dgemv if dt == F64 else gb_sgemv
    _check(f(layout, m, n, alpha, A, lda, x, c, ws, nb, stream), "gemv")


def dot(x, y, alpha, n: int | None = None, stream=None) -> None:
    """alpha += x . y in place; ``alpha`` is a one-element CUDA tensor."""
    n = x.numel() if n is None else n
    dt = _dtype_code(x)
    nb = gb_workspace_bytes(OP_DOT, dt, 0, 0, n)
    ws = workspace(nb, x.device, stream)
    f = gb_ddot if dt == F64 else gb_sdot
    _check(f(n, x, y, alpha, ws, nb, stream), "dot")


def ger(x, y, C, alpha: float = 1.0, layout: int = ROW_MAJOR, m: int | None = None,
        n: int | None = None, ldc: int | None = None, stream=None) -> None:
    """C += alpha * outer(x, y) in place (one fma per element)."""
    if C.dim() == 2 and m is None:
        m, n = C.shape
        if layout == ROW_MAJOR:
            ldc = C.stride(0) if m > 1 else max(1, n)
        else:
            ldc = C.stride(1) if n > 1 else max(1, m)
    dt = _dtype_code(C)
    f = gb_dger if dt == F64 else gb_sger
    _check(f(layout, m, n, alpha, x, y, C, ldc, stream), "ger")


def quantize(A, fmt: str, stream=None):
    """Row-major 2-D FP32 CUDA tensor -> (codes, scales or None); fmt 'bf16' or
    'e4m3'.  The code rows are padded to 16 bytes (the GEMV reads columns < n)."""
    import torch
    m, n = A.shape
    assert A.dtype == torch.float32 and A.stride(1) == 1
    if fmt == "bf16":
        ldq = (n + 7) // 8 * 8  # 16-byte rows
        Q = torch.empty((m, ldq), dtype=torch.int16, device=A.device)
        _check(gb_quantize_bf16(m, n, A, A.stride(0), Q, ldq, stream), "quantize_bf16")
        return Q, None
    ldq = (n + 15) // 16 * 16
    Q = torch.empty((m, ldq), dtype=torch.uint8, device=A.device)
    s = torch.empty(m, dtype=torch.float32, device=A.device)
    _check(gb_quantize_e4m3(m, n, A, A.stride(0), Q, ldq, s, stream), "quantize_e4m3")
    return Q, s


def gemv_q(Q, scales, x, c, alpha: float = 1.0, n: int | None = None, stream=None) -> None:
    """c += alpha * dequant(Q) @ x for codes from ``quantize`` (BF16 if scales is None)."""
    m = Q.shape[0]
    ldq = Q.stride(0)
    n = Q.shape[1] if n is None else n
    if scales is None:
        nb = gb_workspace_bytes(OP_GEMV_BF16, 0, ROW_MAJOR, m, n)
        ws = workspace(nb, Q.device, stream)
        _check(gb_gemv_bf16(m, n, alpha, Q, ldq, x, c, ws, nb, stream), "gemv_bf16")
    else:
        nb = gb_workspace_bytes(OP_GEMV_E4M3, 0, ROW_MAJOR, m, n)
        ws = workspace(nb, Q.device, stream)
        _check(gb_gemv_e4m3(m, n, alpha, Q, ldq, scales, x, c, ws, nb, stream), "gemv_e4m3")
