"""Avalanche statistics of the output step (Sec. 7), measured on the device.

Sec. 7: changing one input bit should flip about half of the output bits,
and the mixer applied to h mod 2^n is there to achieve that. For 2^16
random 16-byte keys and every one of their 128 input bits, the test hashes
the key and the key with that bit flipped (pmp_hash_fixed, one call of
129 * 2^16 keys) and measures, for every (input bit, output bit) pair, how
often the output bit flips.

Tolerances: each frequency is a mean of 2^16 fair coin flips if the mixer
does its job, so its standard deviation is 0.5 / 256 ~ 0.002, and the
largest deviation among the 4096 (PM+32) or 8192 (PM+64) pairs is about
4.3 of those, ~0.009. The test asks for: the mean over all pairs within
0.5 +- 0.005, every input bit's mean within 0.5 +- 0.02, and every pair
within 0.5 +- 0.02 (about ten standard deviations; measured on a GB300:
worst pair 0.0067 for PM+32 and 0.0085 for PM+64). The raw tree value h (no
mixer) is measured beside it and printed for contrast: being affine in each
input word (Sec. 5), it has pairs whose output bit flips almost always or
almost never (measured worst pair 0.495 / 0.4998).
"""
import numpy as np
import pytest
import torch

from paper_1609_09840_gb300 import synth

pytestmark = pytest.mark.gpu

NKEYS = 1 << 16
KLEN = 16


def flip_blocks(dev):
    base = torch.empty(NKEYS * KLEN, dtype=torch.uint8, device=dev)
    synth.fill_bytes_torch(base, synth.derive(700, synth.TAG_BYTES))
    allk = base.view(1, NKEYS, KLEN).repeat(1 + 8 * KLEN, 1, 1)
    for i in range(8 * KLEN):
        allk[1 + i, :, i // 8] ^= (1 << (i % 8))
    return allk.reshape(-1)


def flip_matrix(h, width):
    h = h.view(1 + 8 * KLEN, NKEYS).to(torch.int64)
    d = h[1:] ^ h[:1]
    cols = [((d >> j) & 1).to(torch.float32).mean(dim=1) for j in range(width)]
    return torch.stack(cols, dim=1).cpu().numpy()  # [input bit, output bit]


@pytest.mark.parametrize("width", (32, 64))
def test_mixed_output_avalanche(native, width):
    key = native.Key(seed=11, width=width)
    keys = flip_blocks("cuda")
    n = keys.numel() // KLEN
    h = native.hash_fixed(key, keys, n, KLEN, KLEN)
    if width == 32:
        h = h.to(torch.int64) & 0xFFFFFFFF
    m = flip_matrix(h, width)
    # raw tree values of the same keys (offsets at the fixed stride)
    offsets = torch.arange(n + 1, dtype=torch.int64, device="cuda") * KLEN
    raw = native.hash_batch(key, keys, offsets, raw=True).view(n, 2)[:, 0]
    if width == 32:
        raw = raw & 0xFFFFFFFF
    mr = flip_matrix(raw, width)
    key.close()
    print("\nPM+%d avalanche: mixed mean %.4f, worst input bit %.4f, worst pair bias %.4f; "
          "raw mean %.4f, worst pair bias %.4f" % (
              width, m.mean(), np.abs(m.mean(axis=1) - 0.5).max() + 0.5, np.abs(m - 0.5).max(),
              mr.mean(), np.abs(mr - 0.5).max()))
    assert abs(m.mean() - 0.5) < 0.005
    assert np.abs(m.mean(axis=1) - 0.5).max() < 0.02
    assert np.abs(m - 0.5).max() < 0.02
