"""Component-wise regularity of PM+32, checked exhaustively on the device.

Sec. 5 (Lemma 7 and the table of properties in Sec. 6.1): for a fixed key,
changing one word of the input while the others stay fixed changes the tree
value h in [0, p) injectively (every level is an affine map of the changed
word modulo p with an invertible coefficient), so after the output step
z = h mod 2^32 every 32-bit value has at most two preimages, and at most
k = 15 values have two (only h in [2^32, p) folds onto [0, k)). The mixer of
Sec. 7 is a bijection, so the mixed outputs obey the same counts.

Each test hashes 2^32 strings that differ in one word only, once raw and once
mixed, through the batched C ABI, and counts the values with the device
(integer hashing: exact counts, no tolerance):
  - one level: 12-byte strings, the middle word takes every value;
  - two levels: 600-byte strings (two level-1 chunks), a word of the first
    chunk takes every value, so the level-1 value of that chunk runs through
    2^32 of the p residues, including values in [2^32, p) that the level-2
    chunk must take with their high bit.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

P32 = (1 << 32) + 15
K32 = 15
STEP = 1 << 26  # strings per batched call


def _need_bytes(stride):
    return 2 * 4 * P32 + STEP * (stride + 8 + 16 + 4) + (4 << 30)


def _run(native, length, stride, word, seed):
    """Counts of the raw values (size p) and of the mixed outputs (size 2^32)
    of the 2^32 strings that differ in word `word`."""
    dev = "cuda"
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < _need_bytes(stride):
        pytest.skip("needs %.0f GiB of free device memory" % (_need_bytes(stride) / 2 ** 30))
    key = native.Key(seed=seed, width=32)
    # every string: the same seeded bytes, except word `word`
    rng = np.random.default_rng(seed)
    row = torch.from_numpy(rng.integers(0, 256, size=stride, dtype=np.uint8)).to(dev)
    data = row.repeat(STEP)
    words = data.view(torch.int32).view(STEP, stride // 4)
    offsets = torch.arange(STEP + 1, dtype=torch.int64, device=dev) * stride - (stride - length)
    offsets[0] = 0  # string i occupies [stride * i, stride * i + length)
    counts_raw = torch.zeros(P32, dtype=torch.int32, device=dev)
    counts_mix = torch.zeros(1 << 32, dtype=torch.int32, device=dev)
    ones = torch.ones(STEP, dtype=torch.int32, device=dev)
    raw = torch.empty(2 * STEP, dtype=torch.int64, device=dev)
    mixed = torch.empty(STEP, dtype=torch.int32, device=dev)
    for c in range((1 << 32) // STEP):
        v = torch.arange(c * STEP, (c + 1) * STEP, dtype=torch.int64, device=dev)
        words[:, word] = (v - (v >= (1 << 31)).to(torch.int64) * (1 << 32)).to(torch.int32)
        native.hash_batch(key, data, offsets, out=raw, raw=True)
        native.hash_batch(key, data, offsets, out=mixed)
        h = raw[0::2]
        # range checks on the host before the values index anything
        assert int(raw[1::2].abs().max()) == 0
        assert 0 <= int(h.min()) and int(h.max()) < P32
        counts_raw.index_add_(0, h, ones)
        counts_mix.index_add_(0, mixed.to(torch.int64) & 0xFFFFFFFF, ones)
    torch.cuda.synchronize()
    assert native.device_status() == 0
    key.close()
    return counts_raw, counts_mix


def _check(counts_raw, counts_mix):
    # raw tree values: injective in the changed word
    assert int(counts_raw.sum(dtype=torch.int64)) == 1 << 32
    assert int(counts_raw.max()) == 1
    # z = h mod 2^32: at most two preimages, at most k values with two, and
    # exactly those j < k hit both as j and as 2^32 + j
    both = int(((counts_raw[:K32] == 1) & (counts_raw[1 << 32:] == 1)).sum())
    assert int(counts_mix.max()) <= 2
    twice = int((counts_mix == 2).sum(dtype=torch.int64))
    once = int((counts_mix == 1).sum(dtype=torch.int64))
    assert twice == both <= K32
    assert once + 2 * twice == 1 << 32


def test_pm32_regularity_one_level_exhaustive(native):
    counts_raw, counts_mix = _run(native, length=12, stride=16, word=1, seed=21)
    _check(counts_raw, counts_mix)


def test_pm32_regularity_two_levels_exhaustive(native):
    counts_raw, counts_mix = _run(native, length=600, stride=600, word=37, seed=22)
    _check(counts_raw, counts_mix)
