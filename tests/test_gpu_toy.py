"""Toy members of the family on the device (p = 2^8 + 1 and 2^16 + 1, k = 1:
the first rows of Sec. 5's table of the smallest primes above powers of two).

Parity first: the raw tree values of every (key, word position, word value)
case equal oracle/pmo.c's, and the key-difference histogram of a one-chunk
function equals the one the oracle's chunk function gives key by key. Then the
enumerations the CPU cannot finish in seconds:
- component-wise regularity (Sec. 3, Sec. 5): for many keys and every whole
  word of multi-level strings, all 2^n values of the word give distinct raw
  values, and mod 2^n no value has more than two preimages and at most k = 1
  has two;
- almost Delta-universality (Sec. 5): over all (p - 1 - kappa)^m keys, no
  difference f(s) - f(t) occurs for more than (p - 1 - kappa)^(m - 1) keys,
  with the exact histogram where it has a closed form.
"""
import numpy as np
import pytest
import torch

from oracle import pmo
from paper_1609_09840_gb300 import synth

pytestmark = pytest.mark.gpu


def toy(n, kappa=0, m=4, L=4):
    return pmo.params(n, 1, kappa, m, L)


def string_bytes(seed, length):
    return np.asarray(synth.bytes_np(synth.derive(seed, synth.TAG_BYTES), 0, max(length, 1)),
                      dtype=np.uint8)[:length]


def dev(b):
    return torch.from_numpy(np.concatenate([b, np.zeros(8, np.uint8)])).cuda()


def oracle_raws(P, seed, buf, comp):
    key = pmo.key_expand(P, seed)
    W = P.n // 8
    out = []
    for x in range(1 << P.n):
        b = buf.copy()
        b[comp * W:(comp + 1) * W] = np.frombuffer(int(x).to_bytes(W, "little"), dtype=np.uint8)
        out.append(pmo.tree_bytes(P, key, b))
    return out


def expected_counts(raws, n):
    seen_raw, seen = set(), {}
    c = [0, 0, 0]
    for h in raws:
        c[0] += h in seen_raw
        seen_raw.add(h)
        z = h % (1 << n)
        seen[z] = seen.get(z, 0) + 1
        if seen[z] == 2:
            c[1] += 1
        elif seen[z] > 2:
            c[2] += 1
    return c


@pytest.mark.parametrize("kappa", [0, 100])
def test_regularity_raw_values_match_oracle_n8(native, kappa):
    n, m, L, length = 8, 4, 4, 9  # 10 words: 3 chunks, then the root (two levels)
    P = toy(n, kappa, m, L)
    buf = string_bytes(40 + kappa, length)
    seed0, nkeys = 17, 3
    counts, raw = native.toy_regularity(n, kappa, m, L, seed0, nkeys, dev(buf), length, 0, length, want_raw=True)
    counts, raw = counts.cpu().numpy(), raw.cpu().numpy()
    for q in range(nkeys):
        for c in range(length):
            want = oracle_raws(P, seed0 + q, buf, c)
            row = q * length + c
            assert raw[row].tolist() == want, (q, c)
            assert counts[row].tolist() == expected_counts(want, n), (q, c)


def test_regularity_raw_values_match_oracle_n16(native):
    n, m, L, length = 16, 4, 4, 4  # two words and the pad: one level
    P = toy(n, 0, m, L)
    buf = string_bytes(41, length)
    counts, raw = native.toy_regularity(n, 0, m, L, 23, 1, dev(buf), length, 0, 2, want_raw=True)
    raw, counts = raw.cpu().numpy(), counts.cpu().numpy()
    for c in range(2):
        want = oracle_raws(P, 23, buf, c)
        assert raw[c].tolist() == want, c
        assert counts[c].tolist() == expected_counts(want, n), c


@pytest.mark.parametrize("n,kappa,length", [(8, 0, 40), (8, 200, 63), (16, 0, 40), (16, 9000, 62)])
def test_every_component_regular_over_many_keys(native, n, kappa, length):
    """Three-level strings (m = 4), every whole word, 1024 keys: no raw value
    repeats; mod 2^n at most k = 1 value has two preimages, none has three."""
    m, L, nkeys = 4, 4, 1024
    W = n // 8
    assert pmo.levels(toy(n, kappa, m, L), length // W + 1) == 3
    buf = string_bytes(50 + n + kappa, length)
    ncomp = length // W
    counts, _ = native.toy_regularity(n, kappa, m, L, 1000 + kappa, nkeys, dev(buf), length, 0, ncomp)
    c = counts.cpu().numpy()
    assert c.shape == (nkeys * ncomp, 3)
    assert c[:, 0].max() == 0
    assert c[:, 1].max() <= 1
    assert c[:, 2].max() == 0


def oracle_delta_hist(P, s, t):
    p = pmo.prime(P)
    R = p - P.kappa - 1
    hist = np.zeros(p, dtype=np.int64)
    for a1 in range(1, R + 1):
        for a2 in range(1, R + 1):
            fk = [0, a1, a2]
            hist[(pmo.chunk(P, fk, list(s)) - pmo.chunk(P, fk, list(t))) % p] += 1
    return hist


@pytest.mark.parametrize("kappa", [0, 100])
def test_delta_histogram_matches_oracle_n8(native, kappa):
    P = pmo.params(8, 1, kappa, 2, 1)
    for s, t in [((7, 200), (100, 9)), ((256, 0), (0, 256))]:
        got = native.toy_delta_hist(8, kappa, 2, s, t).cpu().numpy()
        assert got.tolist() == oracle_delta_hist(P, s, t).tolist(), (s, t)


@pytest.mark.parametrize("n,kappa,m", [(8, 0, 3), (8, 57, 3), (16, 0, 2), (16, 1000, 2)])
def test_almost_delta_universal_over_every_key(native, n, kappa, m):
    """Every key of a one-chunk function: 2^24 (n = 8, m = 3) and 2^32 (n = 16,
    m = 2) keys at kappa = 0. Bound of Sec. 5: count * (p - 1 - kappa) <= keys."""
    p = (1 << n) + 1
    R = p - kappa - 1
    rng = np.random.default_rng(n * 100 + kappa)
    pairs = [
        ([1] + [0] * (m - 1), [0] * m),                                   # one component, difference 1
        ([p - 1] + [5] * (m - 1), [0] + [5] * (m - 1)),                   # largest value against 0
        ([int(v) for v in rng.integers(0, p, m)], [int(v) for v in rng.integers(0, p, m)]),
        ([0] * (m - 1) + [1 << n], [1 << n] + [0] * (m - 1)),            # a value moved
    ]
    for s, t in pairs:
        if s == t:
            continue
        h = native.toy_delta_hist(n, kappa, m, s, t).cpu().numpy()
        assert int(h.sum()) == R ** m
        assert int(h.max()) * R <= R ** m, (s, t)
        d = [(a - b) % p for a, b in zip(s, t)]
        if sum(1 for x in d if x) == 1 and kappa == 0:
            # f(s) - f(t) = a_i d_i: every non-zero residue for R^(m-1) keys each
            want = np.full(p, R ** (m - 1), dtype=np.int64)
            want[0] = 0
            assert h.tolist() == want.tolist(), (s, t)


def test_toy_arguments_are_checked(native):
    from paper_1609_09840_gb300.native import PmpError

    buf = dev(string_bytes(1, 8))
    with pytest.raises(PmpError):
        native.toy_regularity(12, 0, 4, 4, 1, 1, buf, 8, 0, 1)       # n not 8 or 16
    with pytest.raises(PmpError):
        native.toy_regularity(8, 0, 4, 4, 1, 1, buf, 8, 7, 2)        # position past the string words
    with pytest.raises(PmpError):
        native.toy_regularity(8, 0, 2, 1, 1, 1, buf, 8, 0, 1)        # needs more than L levels
    with pytest.raises(PmpError):
        native.toy_delta_hist(8, 0, 2, (1, 2), (1, 2))                # s == t
    with pytest.raises(PmpError):
        native.toy_delta_hist(8, 0, 2, (300, 2), (1, 2))              # value >= p
