"""gb_dgemv_noalloc: GEMV for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc or take memory from an allocator (a
runtime that owns the whole device heap, or code that must not allocate
once it is set up), so they cannot hand gb_dgemv the workspace its split
sums need.  gb_dgemv_noalloc takes no workspace: its split sums use a fixed
scratch array built into the library (GB_NOALLOC_SCRATCH_BYTES, 256 KiB per
GPU).  These tests call it through the C ABI on two calls in a row (the
second call finds the scratch left over from the first) and check every
output element against the FP64 oracle, with the tolerance of the other
FP64 GEMV tests, and against gb_dgemv, the entry point with a caller
workspace.  Shapes whose split sums need more scratch than the array holds
must be refused with GB_ERR_WORKSPACE, and an injected fault must enqueue
nothing; either way c stays untouched.

This file is collected last, so a run that stops at the first failure has
run every other test before it."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import oracle
import paper_2108_02025_gb300 as gb
import synth

pytestmark = pytest.mark.gpu

ROW, COL = gb.ROW_MAJOR, gb.COL_MAJOR
TOL = 1e-12
LIMIT = 256 << 10
CANDIDATES = [(64, 200003), (33, 250001), (300, 150001), (1000, 777), (4096, 4096),
              (2048, 65536), (64, 1048576), (8192, 8192)]


def needed(layout, m, n):
    return gb.gb_workspace_bytes(gb.OP_GEMV, gb.F64, layout, m, n)


def inputs(layout, m, n, seed):
    ld = n if layout == ROW else m
    A = torch.empty(m * n, dtype=torch.float64, device="cuda")
    x = torch.empty(n, dtype=torch.float64, device="cuda")
    c = torch.empty(m, dtype=torch.float64, device="cuda")
    synth.fill_uniform(A, seed, 1)
    synth.fill_uniform(x, seed, 2)
    synth.fill_uniform(c, seed, 3)
    return A, x, c, ld


@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
def test_matches_oracle_twice(layout):
    shapes = [(m, n) for (m, n) in CANDIDATES if 0 < needed(layout, m, n) <= LIMIT]
    assert shapes, "no candidate shape uses the scratch array"
    for (m, n) in shapes[:3]:
        A, x, c, ld = inputs(layout, m, n, seed=m + n)
        c_ref, c_new = c.clone(), c.clone()
        nb = needed(layout, m, n)
        ws = torch.zeros(nb, dtype=torch.uint8, device="cuda")
        c0 = c.cpu().numpy()
        A_h, x_h = A.cpu().numpy(), x.cpu().numpy()
        for call in range(2):
            before = c_new.cpu().numpy()
            assert gb.gb_dgemv_noalloc(layout, m, n, 0.75, A, ld, x, c_new) == gb.GB_OK
            assert gb.gb_dgemv(layout, m, n, 0.75, A, ld, x, c_ref, ws, nb) == gb.GB_OK
            torch.cuda.synchronize()
            got = c_new.cpu().numpy()
            want = oracle.gemv(layout, m, n, 0.75, A_h, ld, x_h, before)
            scale = oracle.gemv_scale(layout, m, n, 0.75, A_h, ld, x_h, before)
            err = np.max(np.abs(got - want) / scale)
            assert err <= TOL, (layout, m, n, call, err)
            # the same kernels as the workspace entry point: the same bits
            assert np.array_equal(got, c_ref.cpu().numpy()), (layout, m, n, call)
        assert not np.array_equal(c_new.cpu().numpy(), c0)


@pytest.mark.parametrize("layout", [ROW, COL], ids=["row", "col"])
def test_no_split_shape_needs_no_scratch(layout):
    m, n = next((m, n) for (m, n) in [(3000, 50), (100000, 8), (20000, 3)]
                if needed(layout, m, n) == 0)
    A, x, c, ld = inputs(layout, m, n, seed=5)
    c_ref, c_new = c.clone(), c.clone()
    assert gb.gb_dgemv(layout, m, n, -1.0, A, ld, x, c_ref, None, 0) == gb.GB_OK
    assert gb.gb_dgemv_noalloc(layout, m, n, -1.0, A, ld, x, c_new) == gb.GB_OK
    torch.cuda.synchronize()
    assert torch.equal(c_ref, c_new)


def test_refuses_shapes_beyond_the_scratch():
    big = [(lay, m, n) for lay in (ROW, COL) for (m, n) in CANDIDATES if needed(lay, m, n) > LIMIT]
    assert big, "no candidate shape exceeds the scratch array"
    lay, m, n = min(big, key=lambda s: s[1] * s[2])
    A, x, c, ld = inputs(lay, m, n, seed=7)
    before = c.clone()
    assert gb.gb_dgemv_noalloc(lay, m, n, 1.0, A, ld, x, c) == gb.GB_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert torch.equal(c, before)


def test_invalid_arguments_match_gb_dgemv():
    P, Q, R = 1 << 20, 1 << 30, 1 << 34   # never dereferenced: rejected on the host
    assert gb.gb_dgemv_noalloc(2, 4, 4, 1.0, P, 4, Q, R) == -1
    assert gb.gb_dgemv_noalloc(0, -1, 4, 1.0, P, 4, Q, R) == -2
    assert gb.gb_dgemv_noalloc(0, 4, 5, 1.0, P, 4, Q, R) == -6
    assert gb.gb_dgemv_noalloc(0, 4, 4, 1.0, None, 4, Q, R) == -5
    assert gb.gb_dgemv_noalloc(0, 4, 4, 1.0, P, 4, Q, P + 8) == -8
    assert gb.gb_dgemv_noalloc(0, 0, 4, 1.0, None, 4, None, None) == gb.GB_OK


_INJECT_CHILD = r"""
import sys, torch
sys.path.insert(0, {root!r})
import paper_2108_02025_gb300 as gb, synth
m, n = 64, 200003
A = torch.empty(m * n, dtype=torch.float64, device="cuda")
x = torch.empty(n, dtype=torch.float64, device="cuda")
c = torch.empty(m, dtype=torch.float64, device="cuda")
for t, s in ((A, 1), (x, 2), (c, 3)):
    synth.fill_uniform(t, 9, s)
before = c.clone()
assert 0 < gb.gb_workspace_bytes(gb.OP_GEMV, gb.F64, gb.ROW_MAJOR, m, n) <= (256 << 10)
st = gb.gb_dgemv_noalloc(gb.ROW_MAJOR, m, n, 1.0, A, n, x, c)
torch.cuda.synchronize()
assert st == gb.GB_ERR_INJECTED, st
assert torch.equal(c, before)
st = gb.gb_dgemv_noalloc(gb.ROW_MAJOR, m, n, 1.0, A, n, x, c)   # the next call runs
torch.cuda.synchronize()
assert st == gb.GB_OK, st
assert not torch.equal(c, before)
print("inject ok")
"""


def test_injected_fault_enqueues_nothing():
    """GB_FAULT_INJECT=gemv:1 fails the first GEMV call after every argument
    check: the call returns GB_ERR_INJECTED with c untouched, and the next
    call runs normally.  The variable is read once per process, so the
    check runs in a child process."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, GB_FAULT_INJECT="gemv:1")
    r = subprocess.run([sys.executable, "-c", _INJECT_CHILD.format(root=root)], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "inject ok" in r.stdout, r.stdout + r.stderr
