"""Degenerate and extreme inputs of the batched and single-buffer paths.

Batches: no strings at all, one string (empty, one byte, exactly one chunk,
one chunk plus a byte, a string long enough for the chunk kernel), only empty
strings, a first offset that is not 8-byte aligned, and a tile that is only
partly filled. Single buffer: the longest string eight levels can hold is
accepted (it needs scratch), one more word needs a ninth level and is refused
with PMP_ETOOLONG before any memory is touched (Alg. 1: at most m^L - 1
words; Table 'properties').
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import pmo
from paper_1609_09840_gb300 import synth

pytestmark = pytest.mark.gpu

WIDTHS = (32, 64)


@pytest.fixture(scope="module")
def keys(native):
    ks = {w: native.Key(seed=13, width=w) for w in WIDTHS}
    yield ks
    for k in ks.values():
        k.close()


def pack_from(lengths, first):
    """offsets[0] = first, string i at [align8(offsets[i]), offsets[i + 1])."""
    off = [first]
    for n in lengths:
        off.append((off[-1] + 7) // 8 * 8 + int(n))
    return np.array(off, dtype=np.int64)


def run(native, key, width, lengths, first_offset=0, seed=77):
    lengths = np.asarray(lengths, dtype=np.int64)
    offsets = pack_from(lengths, first_offset)
    size = int(offsets[-1]) + 64
    host = np.asarray(synth.bytes_np(synth.derive(seed, synth.TAG_BYTES), 0, (size + 15) // 16 * 16), np.uint8)
    got = native.hash_batch(key, torch.from_numpy(host).cuda(), torch.from_numpy(offsets).cuda())
    torch.cuda.synchronize()
    P = pmo.width_params(width)
    want = pmo.hash_batch(P, pmo.key_expand(P, 13), host, offsets)
    return native.as_unsigned(got).astype(np.uint64), want


@pytest.mark.parametrize("width", WIDTHS)
def test_empty_batch(native, keys, width):
    out = torch.full((4,), 7, dtype=torch.int64, device="cuda")
    base = torch.zeros(16, dtype=torch.uint8, device="cuda")
    offsets = torch.zeros(1, dtype=torch.int64, device="cuda")
    native.hash_batch(keys[width], base, offsets, out=out)
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [7, 7, 7, 7]  # nothing written


@pytest.mark.parametrize("width", WIDTHS)
def test_single_string_batches(native, keys, width):
    CB = 128 * width // 8
    for length in (0, 1, 7, 8, CB - 1, CB, CB + 1, 40 * CB + 3):
        got, want = run(native, keys[width], width, [length])
        assert got.tolist() == want.tolist(), length


@pytest.mark.parametrize("width", WIDTHS)
def test_only_empty_strings(native, keys, width):
    got, want = run(native, keys[width], width, np.zeros(1000, np.int64))
    assert got.tolist() == want.tolist()
    assert len(set(got.tolist())) == 1  # every empty string hashes alike


@pytest.mark.parametrize("width", WIDTHS)
def test_unaligned_first_offset_and_partial_tile(native, keys, width):
    rng = np.random.default_rng(width)
    lengths = rng.integers(0, 300, 64 * 3 + 17)
    lengths[::9] = 0
    got, want = run(native, keys[width], width, lengths, first_offset=3)
    assert got.tolist() == want.tolist()


@pytest.mark.parametrize("width", WIDTHS)
def test_longest_accepted_length_and_the_first_refused(native, keys, width):
    """N0 = len / W + 1 words take ceil-log_m(N0) levels; L = 8 levels hold
    N0 <= m^8, i.e. len <= (m^8 - 1) W + W - 1."""
    W = width // 8
    ok_len = ((128 ** 8) - 1) * W + W - 1
    lib = native.load()
    fn = lib.pmp_hash32 if width == 32 else lib.pmp_hash64
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    k = keys[width]
    # accepted by the plan, so it asks for scratch (none given): PMP_EINVAL, no launch
    assert fn(k.handle, buf.data_ptr(), ctypes.c_uint64(ok_len), out.data_ptr(), None, 0, None) == native.PMP_EINVAL
    assert lib.pmp_hash_scratch_bytes(width, ctypes.c_uint64(ok_len)) > 0
    # one more word: a ninth level
    assert fn(k.handle, buf.data_ptr(), ctypes.c_uint64(ok_len + 1), out.data_ptr(), None, 0,
              None) == native.PMP_ETOOLONG
    assert native.device_status() == 0
