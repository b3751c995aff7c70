"""Helpers of the GPU parity tests: device buffers with guard elements,
deliberately misaligned views, and the condition-aware error metric."""
from __future__ import annotations

import numpy as np
import torch

GUARD = 16  # guard elements on each side of every output buffer
CANARY = {np.float64: -7.25e300, np.float32: -7.25e30}


def dev():
    return torch.device("cuda", 0)


def to_dev(a: np.ndarray, misalign: int = 0) -> torch.Tensor:
    """Copy to the device; with misalign=k the returned view starts k
    elements after a 256-byte aligned allocation."""
    a = np.ascontiguousarray(a)
    buf = torch.empty(a.size + misalign + 1, dtype=torch.from_numpy(a[:0]).dtype, device=dev())
    view = buf[misalign:misalign + a.size]
    view.copy_(torch.from_numpy(a))
    return view


class Guarded:
    """An output buffer with canary elements before and after it."""

    def __init__(self, a: np.ndarray, misalign: int = 0):
        a = np.ascontiguousarray(a)
        self.dtype = a.dtype.type
        full = np.full(a.size + 2 * GUARD + misalign, CANARY[self.dtype], dtype=a.dtype)
        full[GUARD + misalign:GUARD + misalign + a.size] = a
        self.buf = torch.from_numpy(full).to(dev())
        self.lo = GUARD + misalign
        self.n = a.size
        self.view = self.buf[self.lo:self.lo + self.n]

    def result(self) -> np.ndarray:
        full = self.buf.cpu().numpy()
        can = CANARY[self.dtype]
        assert np.all(full[:self.lo] == can), "write before the output buffer"
        assert np.all(full[self.lo + self.n:] == can), "write after the output buffer"
        return full[self.lo:self.lo + self.n]


def rel_err(got, want, scale) -> float:
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = np.asarray(scale, dtype=np.float64)
    if got.size == 0:
        return 0.0
    d = np.abs(got - want)
    d = np.where(scale > 0, d / np.where(scale > 0, scale, 1.0), np.where(d == 0, 0.0, np.inf))
    return float(np.max(d))


def workspace(nbytes: int) -> torch.Tensor | None:
    if nbytes == 0:
        return None
    return torch.zeros(nbytes + 256, dtype=torch.uint8, device=dev())
