"""Fixed-length keys (pmp_hash_fixed32/64) against the oracle (needs a GPU).

Every key fits in one level-1 chunk, so its hash is the chunk value of
Sec. 5 (eq. 2wlinear) reduced by Sec. 6.2 / Alg. 2, then the output step:
the oracle's hash of the key alone, bit for bit, at every length class
(empty, partial last word, exact words, the largest one-chunk key) and at
strides with and without gaps between keys; where the batched layout can
express the same keys, the batched path must agree too.
"""
import numpy as np
import pytest
import torch

from oracle import pmo
from paper_1609_09840_gb300 import synth

pytestmark = pytest.mark.gpu

WIDTHS = (32, 64)


@pytest.fixture(scope="module")
def keys(native):
    ks = {w: native.Key(seed=9, width=w) for w in WIDTHS}
    yield ks
    for k in ks.values():
        k.close()


def key_lengths(width):
    CB = 128 * (width // 8)
    return [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 15, 16, 17, 23, 24, 25, 31, 32, 33, 39, 40, 41, 63, 64, 65,
            71, 72, 73, 100, CB - 9, CB - 8, CB - 1]


@pytest.mark.parametrize("width", WIDTHS)
def test_fixed_keys_match_oracle(native, keys, width):
    P = pmo.width_params(width)
    ok = pmo.key_expand(P, 9)
    n = 1037
    rng = np.random.default_rng(width)
    for L in key_lengths(width):
        a8 = (L + 7) // 8 * 8
        # 128: a multiple of 64, so that keys of 2..9 units take the 16-byte loads
        for stride in sorted({max(8, a8), a8 + 8, 128, 1024 + 8}):
            if stride < L:
                continue
            host = synth.bytes_np(synth.derive(500 + L + stride, synth.TAG_BYTES), 0, n * stride)
            dev = torch.from_numpy(host).cuda()
            got = native.as_unsigned(native.hash_fixed(keys[width], dev, n, L, stride)).astype(np.uint64)
            for i in list(rng.choice(n, size=48, replace=False)) + [0, n - 1]:
                i = int(i)
                want = pmo.hash_bytes(P, ok, host[i * stride: i * stride + L])
                assert int(got[i]) == want, (L, stride, i)


@pytest.mark.parametrize("width", WIDTHS)
def test_fixed_keys_equal_batched_path(native, keys, width):
    """Keys packed at stride align8(len) are also a batch (string i at
    [i * stride, i * stride + len)): both paths give the same values."""
    n = 100_003
    for L in [x for x in key_lengths(width) if x > 0]:
        stride = (L + 7) // 8 * 8
        dev = torch.empty((n * stride + 15) // 16 * 16, dtype=torch.uint8, device="cuda")
        synth.fill_bytes_torch(dev, synth.derive(600 + L, synth.TAG_BYTES))
        offsets = torch.arange(n + 1, dtype=torch.int64, device="cuda") * stride - (stride - L)
        offsets[0] = 0
        fixed = native.hash_fixed(keys[width], dev, n, L, stride)
        batched = native.hash_batch(keys[width], dev, offsets)
        assert torch.equal(fixed, batched), L


def test_fixed_keys_argument_errors(native, keys):
    dev = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    lib = native.load()
    k = keys[32]
    out = torch.empty(8, dtype=torch.int32, device="cuda")
    call = lambda base, n, L, stride: lib.pmp_hash_fixed32(k.handle, base, n, L, stride, out.data_ptr(), None)
    assert call(dev.data_ptr(), 4, 512, 512) == native.PMP_EINVAL      # not one chunk
    assert call(dev.data_ptr(), 4, 16, 8) == native.PMP_EINVAL         # stride < len
    assert call(dev.data_ptr(), 4, 16, 20) == native.PMP_EALIGN        # stride not a multiple of 8
    assert call(dev.data_ptr() + 4, 4, 16, 16) == native.PMP_EALIGN    # keys not 8-byte aligned
    assert call(dev.data_ptr(), 0, 16, 16) == native.PMP_OK            # nothing to do
    assert lib.pmp_hash_fixed64(keys[32].handle, dev.data_ptr(), 4, 16, 16, out.data_ptr(), None) == \
        native.PMP_EINVAL                                               # width of the key


@pytest.mark.parametrize("width", WIDTHS)
def test_fixed_keys_of_all_ones_up_to_nine_units(native, keys, width):
    """Keys of 0..73 bytes that are all 0xff (every word at its maximum, so
    every product and carry of the one-unit and few-unit kernels at its
    largest), and all zero: equal to the oracle."""
    P = pmo.width_params(width)
    ok = pmo.key_expand(P, 9)
    n = 300
    for fill in (0xFF, 0x00):
        for L in range(0, 74):
            stride = max(8, (L + 7) // 8 * 8)
            host = np.full(n * stride, fill, dtype=np.uint8)
            dev = torch.from_numpy(host).cuda()
            got = native.as_unsigned(native.hash_fixed(keys[width], dev, n, L, stride)).astype(np.uint64)
            want = pmo.hash_bytes(P, ok, host[:L])
            assert np.all(got == want), (fill, L)
