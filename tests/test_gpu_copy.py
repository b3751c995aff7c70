"""gb_copy_to_host: a kernel stores device bytes into page-locked host
memory through its device mapping.  Every size class (empty, under one
16-byte word, ragged tails, large), aligned and misaligned ends, the bytes
around the destination untouched, and the refusals (pageable or NULL
destination, NULL source)."""
import numpy as np
import pytest
import torch

import paper_2108_02025_gb300 as gb

pytestmark = pytest.mark.gpu

SIZES = [0, 1, 15, 16, 17, 4099, (1 << 20) + 5, 64 << 20]


@pytest.mark.parametrize("nbytes", SIZES)
@pytest.mark.parametrize("offsets", [(0, 0), (1, 0), (0, 3), (5, 7), (16, 32)], ids=str)
def test_copy_bytes(nbytes, offsets):
    so, do = offsets
    g = torch.Generator(device="cuda").manual_seed(nbytes + 31 * so + 7 * do)
    src = torch.randint(0, 256, (nbytes + so + 1,), dtype=torch.uint8, device="cuda", generator=g)
    host = torch.full((nbytes + do + 64,), 0xAB, dtype=torch.uint8, pin_memory=True)
    st = gb.gb_copy_to_host(host.data_ptr() + do, src.data_ptr() + so, nbytes, torch.cuda.current_stream())
    assert st == gb.GB_OK, gb.gb_status_string(st)
    torch.cuda.synchronize()
    h = host.numpy()
    want = src[so:so + nbytes].cpu().numpy()
    assert np.array_equal(h[do:do + nbytes], want)
    assert np.all(h[:do] == 0xAB) and np.all(h[do + nbytes:] == 0xAB)


def test_copy_on_a_side_stream_is_ordered_by_it():
    s = torch.cuda.Stream()
    src = torch.arange(1 << 22, dtype=torch.float32, device="cuda")
    host = torch.zeros(1 << 22, dtype=torch.float32, pin_memory=True)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        src.mul_(2.0)
        assert gb.gb_copy_to_host(host, src, src.numel() * 4, s) == gb.GB_OK
    s.synchronize()
    assert torch.equal(host, torch.arange(1 << 22, dtype=torch.float32) * 2.0)


def test_refusals():
    src = torch.zeros(64, dtype=torch.uint8, device="cuda")
    pageable = np.zeros(64, np.uint8)
    assert gb.gb_copy_to_host(pageable.ctypes.data, src, 64) == -1
    assert gb.gb_copy_to_host(None, src, 64) == -1
    host = torch.zeros(64, dtype=torch.uint8, pin_memory=True)
    assert gb.gb_copy_to_host(host, None, 64) == -2
    assert gb.gb_copy_to_host(None, None, 0) == gb.GB_OK
    torch.cuda.synchronize()
