"""Almost Delta-universality, measured over many keys on the device.

Sec. 5: PM+-Multilinear is 1/(p - 1 - kappa)-almost Delta-universal; by
Lemma 1 (Sec. 3) its values reduced mod 2^t then collide for two distinct
strings with probability at most eps_t = ceil((2p - 1) / 2^t) / (p - 1 -
kappa) over the random key (about 3.05e-5 at t = 16 for both widths).

pmp_count_collisions counts, for the keys of consecutive seeds, how often
the raw values of two one-chunk strings agree in their low t bits. It is
first pinned to the oracle (the same count, exactly, for 2,000 keys at t = 4,
every key expanded and every string hashed by oracle/pmo.c), then run on
10^8 keys for adversarial pairs: strings that differ in one word; a string
and the same string with one more zero byte (the 0x01 pad must separate
them); an all-zero word against two all-zero words; one word moved to
another position. Bar: the count stays below
n eps_t + 6 sqrt(n eps_t) (the bound plus six binomial standard deviations).
"""
import math

import numpy as np
import pytest
import torch

from oracle import pmo
from paper_1609_09840_gb300 import synth

pytestmark = pytest.mark.gpu

WIDTHS = (32, 64)


def eps_t(width, t):
    P = pmo.width_params(width)
    p = pmo.prime(P)
    return math.ceil((2 * p - 1) / 2 ** t) / (p - 1 - P.kappa)


def dev_bytes(b):
    buf = np.zeros(max(16, (len(b) + 15) // 16 * 16), dtype=np.uint8)
    buf[: len(b)] = np.frombuffer(bytes(b), dtype=np.uint8)
    return torch.from_numpy(buf).cuda()


def pairs(width):
    W = width // 8
    rnd = bytes(synth.bytes_np(synth.derive(800, synth.TAG_BYTES), 0, 64))
    a = rnd[:3 * W]
    b = bytearray(a)
    b[W + 1] ^= 0x5A
    word = rnd[32:32 + W]
    return {
        "one_word": (a, bytes(b)),
        "zero_tail": (rnd[:11], rnd[:11] + b"\0"),
        "zero_words": (bytes(W), bytes(2 * W)),
        "moved_word": (word + bytes(W), bytes(W) + word),
    }


@pytest.mark.parametrize("width", WIDTHS)
def test_collision_counter_matches_oracle(native, width):
    P = pmo.width_params(width)
    t, nkeys, seed0 = 4, 2000, 12345
    for name, (a, b) in pairs(width).items():
        want = 0
        for s in range(seed0, seed0 + nkeys):
            k = pmo.key_expand(P, s)
            ha = pmo.tree_bytes(P, k, np.frombuffer(a, dtype=np.uint8))
            hb = pmo.tree_bytes(P, k, np.frombuffer(b, dtype=np.uint8))
            want += (ha - hb) % (1 << t) == 0
        got = native.count_collisions(width, seed0, nkeys, dev_bytes(a), len(a), dev_bytes(b), len(b), t)
        assert got == want, name


@pytest.mark.parametrize("width", WIDTHS)
def test_truncated_collisions_within_the_universality_bound(native, width):
    t, nkeys = 16, 10 ** 8
    e = eps_t(width, t)
    bound = nkeys * e + 6 * math.sqrt(nkeys * e)
    for name, (a, b) in pairs(width).items():
        got = native.count_collisions(width, 1 << 40, nkeys, dev_bytes(a), len(a), dev_bytes(b), len(b), t)
        print("\nPM+%d %s: %d collisions in %d keys (rate %.3e, bound %.3e)" % (
            width, name, got, nkeys, got / nkeys, e))
        assert got <= bound, (name, got, bound)


@pytest.mark.parametrize("width", WIDTHS)
def test_full_width_collisions_reported(native, width):
    """Untruncated raw values (t = n bits): over 2^30 keys the count stays
    within the bound n eps_n plus six standard deviations (about 0.75 expected
    at most for PM+32, essentially none for PM+64); the count is printed."""
    t, nkeys = width, 1 << 30
    e = eps_t(width, t)
    a, b = pairs(width)["one_word"]
    got = native.count_collisions(width, 1 << 41, nkeys, dev_bytes(a), len(a), dev_bytes(b), len(b), t)
    print("\nPM+%d, t = %d: %d collisions in %d keys (bound %.3g per key)" % (width, t, got, nkeys, e))
    assert got <= nkeys * e + 6 * math.sqrt(nkeys * e) + 2
