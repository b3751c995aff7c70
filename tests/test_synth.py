"""The shared input generator: counter-based (any sub-range regenerates
alone), exact value maps, and the CUDA fill equal to the numpy one bit for
bit."""
import numpy as np
import pytest

import synth


def test_subrange_regenerates():
    a = synth.uniform(1000, 5, 2)
    assert np.array_equal(a[100:300], synth.uniform(200, 5, 2, offset=100))
    b = synth.integers(1000, 5, 2, -8, 8)
    assert np.array_equal(b[999:], synth.integers(1, 5, 2, -8, 8, offset=999))


def test_ranges_and_exactness():
    u = synth.uniform(1 << 16, 1, 1)
    assert u.min() >= -1.0 and u.max() < 1.0
    assert np.all((u + 1.0) * 2.0 ** 52 == np.floor((u + 1.0) * 2.0 ** 52))
    f = synth.uniform(1 << 16, 1, 1, np.float32)
    assert f.dtype == np.float32 and f.min() >= -1 and f.max() < 1
    i = synth.integers(1 << 16, 1, 1, -8, 8)
    assert set(np.unique(i).tolist()) == set(range(-8, 9))


def test_streams_and_seeds_differ():
    assert not np.array_equal(synth.uniform(64, 1, 1), synth.uniform(64, 1, 2))
    assert not np.array_equal(synth.uniform(64, 1, 1), synth.uniform(64, 2, 1))


def test_known_values():
    # the first words of seed 0 / stream 0, fixed once from the definition
    u = synth.raw(2, 0, 0)
    k = synth.key(0, 0)
    G = 0x9E3779B97F4A7C15
    mask = (1 << 64) - 1

    def mix(z):
        z ^= z >> 30
        z = (z * 0xBF58476D1CE4E5B9) & mask
        z ^= z >> 27
        z = (z * 0x94D049BB133111EB) & mask
        return z ^ (z >> 31)

    kk = mix(mix((0 + G) & mask) ^ 0)
    assert int(k) == kk
    assert [int(v) for v in u] == [mix((kk + 1 * G) & mask), mix((kk + 2 * G) & mask)]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_cuda_fill_matches_numpy(dtype):
    import torch
    tdt = getattr(torch, dtype)
    t = torch.empty(100003, dtype=tdt, device="cuda")
    synth.fill_uniform(t, 9, 4, offset=12345)
    assert np.array_equal(t.cpu().numpy(), synth.uniform(100003, 9, 4, np.dtype(dtype).type, offset=12345))
    synth.fill_integers(t, 9, 5, -8, 8)
    assert np.array_equal(t.cpu().numpy(), synth.integers(100003, 9, 5, -8, 8, np.dtype(dtype).type))


def test_uniform_pairs_definition():
    """Two FP32 uniforms per word: bits 63..40 then 39..16 of u_k, mapped to
    b * 2^-23 - 1; any sub-range regenerates on its own."""
    import numpy as np
    u = synth.raw(50, 9, 4)
    b = np.stack([u >> np.uint64(40), (u >> np.uint64(16)) & np.uint64(0xFFFFFF)], 1).ravel()
    want = b.astype(np.float64) * 2.0 ** -23 - 1.0
    got = synth.uniform_pairs(100, 9, 4)
    assert got.dtype == np.float32 and np.array_equal(got.astype(np.float64), want)
    for off, n in ((1, 10), (7, 33), (0, 1), (99, 1)):
        assert np.array_equal(synth.uniform_pairs(n, 9, 4, off), got[off:off + n])
    assert synth.uniform_pairs(0, 9, 4).size == 0
