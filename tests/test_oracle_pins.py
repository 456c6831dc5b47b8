"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: the paper's
tables and worked example (tests/golden/), closed forms, invariants the
paper proves, special cases that reduce to Python's arbitrary-precision
arithmetic, and brute force on toy parameters. A plausible slip in the oracle
(a dropped term, a wrong index or sign, a transposed operand, the wrong level
function, the wrong padding byte or byte order) fails at least one of them.
"""
import json
import os
import random

import numpy as np
import pytest
import sympy

from oracle import pmo

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def toy(n=8, k=1, kappa=0, m=4, L=4):
    return pmo.params(n, k, kappa, m, L)


# --------------------------------------------------------------------------
# Paper tables (tests/golden/paper_tables.json)
# --------------------------------------------------------------------------
def test_prime_table_is_smallest_primes_above_powers_of_two():
    """Table of smallest primes above 2^n (Sec. 5)."""
    for n, k in golden("paper_tables.json")["smallest_primes_above_power_of_two"]["rows"]:
        p = (1 << n) + k
        assert sympy.isprime(p)
        assert sympy.nextprime(1 << n) == p


def test_parameter_table_matches_oracle_and_kappa_rule():
    """Table 'parameters' (Sec. 6.1) and the word-fit rule (p-kappa-1)(p-1) < 2^2n
    of Sec. 6.1 (the printed inequality is off by one; the open interval for a_i
    makes the strict form hold), with kappa the smallest value that satisfies it."""
    rows = golden("paper_tables.json")["parameters"]["rows"]
    for row, P in zip(rows, (pmo.pm32(), pmo.pm64())):
        assert (P.n, P.k, P.kappa, P.m, P.L) == (row["n"], row["k"], row["kappa"], row["m"], row["L"])
        p = pmo.prime(P)
        assert (p - P.kappa - 1) * (p - 1) < 1 << (2 * P.n)
        assert (p - (P.kappa - 1) - 1) * (p - 1) >= 1 << (2 * P.n)
        # the exact slack: 2^2n - (k-1)^2
        assert (1 << (2 * P.n)) - (p - P.kappa - 1) * (p - 1) == (P.k - 1) ** 2


def test_properties_table_epsilon_and_max_length():
    """Table 'properties': eps = 3L/(p-1-kappa) after mod 2^n (Sec. 5 end) and a
    maximum length of m^L - 1 words (Algorithm 1 input bound)."""
    rows = golden("paper_tables.json")["properties"]["rows"]
    from fractions import Fraction

    for row, P in zip(rows, (pmo.pm32(), pmo.pm64())):
        p = pmo.prime(P)
        eps = Fraction(3 * P.L, p - 1 - P.kappa)
        assert eps == Fraction(row["eps_num"], (1 << row["eps_pow"]) - row["eps_sub"])
        assert P.m ** P.L - 1 == (1 << row["max_words_log2"]) - 1
        # the oracle accepts exactly sigma lengths up to m^L = N + 1
        assert pmo.levels(P, P.m ** P.L) == P.L
        assert pmo.levels(P, P.m ** P.L + 1) == 0


def test_reduction_bound_constants():
    """Sec. 6.2 bound terms for PM+32: k^2 m = 28800, k(k-1) = 210, slack 29023."""
    g = golden("paper_tables.json")["reduction_bound"]
    k, m = 15, 128
    assert k * k * m == g["k2m_pm32"]
    assert k * (k - 1) == g["kk1_pm32"]
    # (2^n - 1) + k^2 m + k(k-1) + (2^n + k - 1) = 2 * 2^n + slack
    assert -1 + g["k2m_pm32"] + g["kk1_pm32"] + (k - 1) == g["slack"]


# --------------------------------------------------------------------------
# Generic remainder against Python's '%'
# --------------------------------------------------------------------------
@pytest.mark.parametrize("P", [pmo.pm32(), pmo.pm64(), toy(8), toy(16)])
def test_generic_remainder_matches_python_mod(P):
    p = pmo.prime(P)
    rng = random.Random(7)
    xs = [0, 1, p - 1, p, p + 1, 2 * p - 1, 2 * p, (1 << 192) - 1, (1 << 256) - 1, (1 << P.n),
          (1 << (2 * P.n)) - 1, p * p - 1, p * (1 << 100) + 5]
    xs += [rng.getrandbits(rng.choice([8, 40, 72, 130, 200, 256])) for _ in range(400)]
    for x in xs:
        x &= (1 << 256) - 1
        assert pmo.mod(P, x) == x % p


# --------------------------------------------------------------------------
# Chunk function, eq. (2wlinear)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("P", [pmo.pm32(), pmo.pm64()])
def test_chunk_selector_keys_pick_one_component(P):
    """b = 0 and a = e_r makes f(s) = s_r: pins which key multiplies which word."""
    p = pmo.prime(P)
    rng = random.Random(1)
    s = [rng.randrange(p) for _ in range(P.m)]
    for r in (0, 1, 2, 63, 64, 126, 127):
        fkey = [0] * (P.m + 1)
        fkey[1 + r] = 1
        assert pmo.chunk(P, fkey, s) == s[r]
    fkey = [12345] + [0] * P.m
    assert pmo.chunk(P, fkey, s) == 12345


@pytest.mark.parametrize("P", [pmo.pm32(), pmo.pm64()])
def test_chunk_all_ones_key_is_sum_mod_p(P):
    p = pmo.prime(P)
    rng = random.Random(2)
    s = [rng.randrange(p) for _ in range(P.m)]
    assert pmo.chunk(P, [0] + [1] * P.m, s) == sum(s) % p


@pytest.mark.parametrize("P", [pmo.pm32(), pmo.pm64()])
def test_chunk_extremal_closed_form(P):
    """All a_i = p-kappa-1, all s_i = p-1, b = 2^n-1: the largest sum of Sec. 6.2,
    S = b + m (p-kappa-1)(p-1), which needs three words."""
    p = pmo.prime(P)
    a = p - P.kappa - 1
    b = (1 << P.n) - 1
    S = b + P.m * a * (p - 1)
    assert S >= 1 << (2 * P.n)  # a genuine three-word sum
    assert pmo.chunk(P, [b] + [a] * P.m, [p - 1] * P.m) == S % p


@pytest.mark.parametrize("P", [pmo.pm32(), pmo.pm64()])
def test_chunk_is_affine_in_each_component_with_slope_a_r(P):
    """f(s + e_r) - f(s) = a_r (mod p): the component-wise structure behind the
    regularity and universality proofs of Sec. 5."""
    p = pmo.prime(P)
    key = pmo.key_expand(P, 99)
    fkey = [int(x) for x in key[: P.m + 1]]
    rng = random.Random(3)
    s = [rng.randrange(p - 1) for _ in range(P.m)]
    f0 = pmo.chunk(P, fkey, s)
    for r in (0, 5, 77, 127):
        s2 = list(s)
        s2[r] += 1
        assert (pmo.chunk(P, fkey, s2) - f0) % p == fkey[1 + r] % p


# --------------------------------------------------------------------------
# Tree (Algorithm 1), worked example of Fig. 1, padding and byte order
# --------------------------------------------------------------------------
def test_figure1_worked_example_structure():
    """Fig. 1 with m = 4: 'ab' -> f1(a,b,1,0); 'abcde' -> f2(f1(a,b,c,d), f1(e,1,0,0), 0, 0)."""
    fig = golden("paper_tables.json")["figure1"]
    P = toy(n=8, k=1, kappa=0, m=fig["m"], L=3)
    key = pmo.key_expand(P, 2024)
    f = [list(map(int, key[j * (P.m + 1): (j + 1) * (P.m + 1)])) for j in range(P.L)]
    chars = {c: ord(c) for c in "abcde"}

    def resolve(x, env):
        return chars[x] if isinstance(x, str) and x in chars else env.get(x, x)

    for word, spec in (("ab", fig["ab"]), ("abcde", fig["abcde"])):
        env = {}
        l1 = [pmo.chunk(P, f[0], [resolve(x, env) for x in seg]) for seg in spec["level1"]]
        for i, v in enumerate(l1):
            env["L1_%d" % i] = v
        expect = l1[0] if spec["level2"] is None else pmo.chunk(
            P, f[1], [resolve(x, env) for x in spec["level2"][0]])
        words = [ord(c) for c in word]
        assert pmo.tree_words(P, key, words) == expect
        # with 8-bit words the byte padding of Sec. 4 appends exactly the value 1
        assert pmo.tree_bytes(P, key, word.encode()) == expect
        # and the same numbers with f written out as b + sum a_i s_i mod p
        p = pmo.prime(P)
        if spec["level2"] is None:
            seg = [chars["a"], chars["b"], 1, 0]
            assert expect == (f[0][0] + sum(a * s for a, s in zip(f[0][1:], seg))) % p


def selector_key(P, picks):
    """Key whose level-j function returns component picks[j] (b = 0)."""
    key = np.zeros((P.L, P.m + 1), dtype=np.uint64)
    for j, r in enumerate(picks):
        key[j, 1 + r] = 1
    return key.reshape(-1)


@pytest.mark.parametrize("P", [pmo.pm32(), pmo.pm64()])
def test_byte_padding_and_little_endian_words(P):
    """Sec. 4: pad with a 0x01 byte and zeros to the word boundary; words are
    little-endian. A selector key exposes one word of sigma."""
    W = P.n // 8
    data = bytes(range(1, 40))
    for length in range(0, 3 * W + 1):
        s = data[:length]
        padded = s + b"\x01" + b"\x00" * (W - 1 - (length % W))
        assert len(padded) % W == 0
        nwords = len(padded) // W
        assert nwords == length // W + 1
        for r in range(nwords + 1):
            expect = int.from_bytes(padded[r * W:(r + 1) * W], "little") if r < nwords else 0
            assert pmo.tree_bytes(P, selector_key(P, [r]), s) == expect


def test_level_count_boundaries():
    """levels(N0) under Algorithm 1 with at least one level applied."""
    for P in (pmo.pm32(), pmo.pm64()):
        m = P.m
        assert pmo.levels(P, 1) == 1
        assert pmo.levels(P, m) == 1
        assert pmo.levels(P, m + 1) == 2
        assert pmo.levels(P, m * m) == 2
        assert pmo.levels(P, m * m + 1) == 3
        assert pmo.levels(P, m ** 3 + 1) == 4
    P = toy(m=4, L=3)
    assert [pmo.levels(P, n) for n in (1, 4, 5, 16, 17, 64, 65)] == [1, 1, 2, 2, 3, 3, 0]


@pytest.mark.parametrize("P", [pmo.pm32(), pmo.pm64()])
def test_two_level_structure_with_selector_and_sum_keys(P):
    """Level 1 sums its chunk (a = 1), level 2 selects child 1: the hash is the sum
    of the second level-1 chunk's words mod p, so level order and chunking show."""
    W = P.n // 8
    key = np.zeros((P.L, P.m + 1), dtype=np.uint64)
    key[0, 1:] = 1
    key[1, 2] = 1  # a_{2,2}: picks the second level-1 value
    key = key.reshape(-1)
    rng = np.random.default_rng(5)
    length = (P.m + 30) * W + 3  # two level-1 chunks
    data = rng.integers(0, 256, length, dtype=np.uint8).tobytes()
    padded = data + b"\x01" + b"\x00" * (W - 1 - (length % W))
    words = [int.from_bytes(padded[i:i + W], "little") for i in range(0, len(padded), W)]
    assert len(words) > P.m
    expect = sum(words[P.m: 2 * P.m]) % pmo.prime(P)
    assert pmo.tree_bytes(P, key, data) == expect


def test_toy_tree_matches_nested_composition_by_brute_force():
    """Toy m = 3, n = 8: compare against the nested composition of Algorithm 1
    built from the one-chunk function for every string length 0..40."""
    P = toy(n=8, k=1, kappa=0, m=3, L=5)
    key = pmo.key_expand(P, 11)
    f = [list(map(int, key[j * 4:(j + 1) * 4])) for j in range(P.L)]
    rng = random.Random(8)
    for length in range(0, 41):
        s = [rng.randrange(256) for _ in range(length)]
        sigma = s + [1]
        j = 0
        while True:
            while len(sigma) % P.m:
                sigma.append(0)
            sigma = [pmo.chunk(P, f[j], sigma[i:i + P.m]) for i in range(0, len(sigma), P.m)]
            j += 1
            if len(sigma) == 1:
                break
        assert pmo.tree_bytes(P, key, bytes(s)) == sigma[0]


@pytest.mark.parametrize("P", [pmo.pm32(), pmo.pm64(), toy(8, m=4, L=8), toy(16, m=5, L=8)])
def test_streaming_order_equals_level_by_level(P):
    """Sec. 4: the bounded-memory order gives the same value as Algorithm 1."""
    key = pmo.key_expand(P, 3)
    W = P.n // 8
    rng = np.random.default_rng(6)
    m = P.m
    lengths = set(range(0, 3 * W))
    for nw in (m - 1, m, m + 1, 2 * m, m * m - 1, m * m, m * m + 1, m * m * 2 + 7):
        for d in (-W - 1, -1, 0, 1, W):
            lengths.add(max(0, nw * W + d))
    if m == 4:
        lengths.update(range(0, 300))
    for length in sorted(lengths):
        if length > 600000:
            continue
        data = rng.integers(0, 256, length, dtype=np.uint8)
        assert pmo.tree_bytes(P, key, data) == pmo.tree_bytes(P, key, data, streaming=True), length


# --------------------------------------------------------------------------
# Regularity and universality (Sec. 3, Sec. 5) by brute force
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nbits,levels_len", [(8, 3), (8, 9), (16, 2)])
def test_component_wise_regularity_exhaustive_toy(nbits, levels_len):
    """Fix a key and a string, vary one word over all 2^n values: the raw tree
    values are pairwise distinct (component-wise regular), and after mod 2^n no
    value has more than 2 preimages and at most k values have 2 (Sec. 3, Lemma on
    mod M; Table 'properties')."""
    P = toy(n=nbits, k=1, kappa=0, m=4, L=4)
    key = pmo.key_expand(P, 17)
    W = nbits // 8
    rng = np.random.default_rng(nbits + levels_len)
    base = rng.integers(0, 256, levels_len * W, dtype=np.uint8)
    comp = levels_len // 2
    raws = []
    for x in range(1 << nbits):
        buf = base.copy()
        buf[comp * W:(comp + 1) * W] = np.frombuffer(int(x).to_bytes(W, "little"), dtype=np.uint8)
        raws.append(pmo.tree_bytes(P, key, buf))
    assert len(set(raws)) == len(raws)
    outs = [r % (1 << nbits) for r in raws]
    counts = np.bincount(outs, minlength=1 << nbits)
    assert counts.max() <= 2
    assert (counts == 2).sum() <= P.k


@pytest.mark.parametrize("P", [pmo.pm32(), pmo.pm64()])
def test_component_wise_injectivity_sample(P):
    """Varying one word of a PM+32/PM+64 string never repeats a raw tree value."""
    key = pmo.key_expand(P, 21)
    W = P.n // 8
    rng = np.random.default_rng(22)
    base = rng.integers(0, 256, 200 * W, dtype=np.uint8)  # two levels
    seen = set()
    for x in rng.integers(0, 2 ** 32, 3000, dtype=np.uint64).tolist() + [0, 1, 2 ** 32 - 1]:
        buf = base.copy()
        buf[130 * W:130 * W + 4] = np.frombuffer(int(x).to_bytes(4, "little"), dtype=np.uint8)
        seen.add((x, pmo.tree_bytes(P, key, buf)))
    raws = {}
    for x, r in seen:
        raws.setdefault(r, set()).add(x)
    assert all(len(v) == 1 for v in raws.values())


def test_almost_delta_universality_exhaustive_toy():
    """Over every key (a_1, a_2) of a toy PM+ function with m = 2, n = 8, p = 257,
    kappa = 0, the difference f(s) - f(s') takes any value c for at most a
    1/(p-1-kappa) fraction of keys (Sec. 5: 1/(p-1-kappa)-almost Delta-universal)."""
    P = toy(n=8, k=1, kappa=0, m=2, L=1)
    p = pmo.prime(P)
    keys_a = range(1, p - P.kappa)  # (0, p - kappa)
    nkeys = len(keys_a) ** 2
    pairs = [((3, 5), (4, 5)), ((0, 0), (0, 1)), ((7, 200), (100, 9)), ((256, 0), (0, 256))]
    for s, t in pairs:
        diffs = np.zeros(p, dtype=np.int64)
        for a1 in keys_a:
            for a2 in keys_a:
                fk = [0, a1, a2]
                d = (pmo.chunk(P, fk, list(s)) - pmo.chunk(P, fk, list(t))) % p
                diffs[d] += 1
        assert diffs.max() * (p - 1 - P.kappa) <= nkeys


# --------------------------------------------------------------------------
# Output step (Sec. 5 end, Sec. 7)
# --------------------------------------------------------------------------
def _inv_xorshift(z, s, bits):
    mask = (1 << bits) - 1
    x = z
    for _ in range(bits // s + 1):
        x = z ^ (x >> s)
    return x & mask


@pytest.mark.parametrize("bits", [32, 64])
def test_mixer_is_a_bijection_with_explicit_inverse(bits):
    """Sec. 7: the mixers are invertible. The inverse undoes each step: the
    xorshift by s >= bits/2 and the odd multiplier (inverse mod 2^bits)."""
    g = golden("paper_tables.json")["mixer"]["pm%d" % bits]
    mult = int(g["mult"], 16)
    assert mult % 2 == 1
    inv = pow(mult, -1, 1 << bits)
    mix = pmo.mix32 if bits == 32 else pmo.mix64
    rng = random.Random(bits)
    xs = [0, 1, 2, (1 << bits) - 1, 1 << (bits - 1)] + [rng.getrandbits(bits) for _ in range(20000)]
    outs = set()
    for x in xs:
        z = mix(x)
        y = _inv_xorshift(z, g["s2"], bits)
        y = (y * inv) & ((1 << bits) - 1)
        y = _inv_xorshift(y, g["s1"], bits)
        assert y == x
        outs.add(z)
    assert len(outs) == len(set(xs))


@pytest.mark.parametrize("P", [pmo.pm32(), pmo.pm64()])
def test_output_step_reduces_mod_2n_before_mixing(P):
    p = pmo.prime(P)
    mix = pmo.mix32 if P.n == 32 else pmo.mix64
    for h in (0, 1, (1 << P.n) - 1, 1 << P.n, p - 1):
        assert pmo.output(P, h) == mix(h % (1 << P.n))


# --------------------------------------------------------------------------
# Key expansion convention
# --------------------------------------------------------------------------
def test_splitmix64_reference_outputs():
    g = golden("splitmix64.json")
    for i, v in enumerate(g["outputs"]):
        assert pmo.splitmix64_at(g["seed"], i) == int(v, 16)


@pytest.mark.parametrize("P", [pmo.pm32(), pmo.pm64()])
def test_key_ranges_follow_the_definition(P):
    """Definition (Sec. 5): b in [0, 2^n), a_i in (0, p - kappa)."""
    p = pmo.prime(P)
    for seed in (0, 1, 2, 3, 2 ** 64 - 1):
        key = pmo.key_expand(P, seed).reshape(P.L, P.m + 1)
        assert (key[:, 0].astype(object) < (1 << P.n)).all()
        a = key[:, 1:].astype(object)
        assert (a >= 1).all() and (a < p - P.kappa).all()
    # the first draws of the stream land where the convention says
    key = pmo.key_expand(P, 1)
    assert int(key[0]) == pmo.splitmix64_at(1, 0) >> (64 - P.n)


def test_key_rejection_sampling_skips_out_of_range_draws():
    """Toy n = 8 with kappa large enough that rejections are frequent."""
    P = pmo.params(8, 1, 100, 4, 2)  # a in [1, 257 - 101] = [1, 156]
    key = pmo.key_expand(P, 5)
    draws = iter(pmo.splitmix64_at(5, i) >> 56 for i in range(10000))
    for j in range(P.L):
        assert int(key[j * 5]) == next(draws)
        for i in range(1, 5):
            while True:
                a = next(draws)
                if 1 <= a <= 156:
                    break
            assert int(key[j * 5 + i]) == a


@pytest.mark.parametrize("P", [pmo.pm32(), pmo.pm64()])
def test_batch_wrapper_is_the_single_string_hash(P):
    """The oracle's batch entry point applies the single-string hash (pinned
    above) to each [align8(offsets[i]), offsets[i+1]) and, raw, the tree value;
    an end before the aligned start is refused."""
    key = pmo.key_expand(P, 31)
    lengths = np.array([0, 1, 7, 8, 9, 100, 0, 513, 1025, 3], dtype=np.int64)
    offsets = [3]
    for n in lengths:
        offsets.append((offsets[-1] + 7) // 8 * 8 + int(n))
    offsets = np.array(offsets, dtype=np.int64)
    base = np.random.default_rng(32).integers(0, 256, int(offsets[-1]) + 16, dtype=np.uint8)
    out = pmo.hash_batch(P, key, base, offsets)
    raw = pmo.hash_batch(P, key, base, offsets, raw=True)
    for i in range(lengths.size):
        s = (int(offsets[i]) + 7) // 8 * 8
        piece = base[s:int(offsets[i + 1])]
        assert int(out[i]) == pmo.hash_bytes(P, key, piece)
        assert int(raw[2 * i]) + (int(raw[2 * i + 1]) << 64) == pmo.tree_bytes(P, key, piece)
    bad = offsets.copy()
    bad[2] = bad[1] - 1  # string 1 would end before its aligned start
    with pytest.raises(ValueError):
        pmo.hash_batch(P, key, base, bad)


# --------------------------------------------------------------------------
# The whole hash in Python integers, with real seeded keys
# --------------------------------------------------------------------------
def bigint_tree(width, key, data):
    """h(s) by the definitions alone, in Python's arbitrary-precision
    integers: the bytes followed by 0x01 and zeros up to a word boundary,
    read as little-endian n-bit words (Sec. 4); then Algorithm 1: zero-pad to
    a multiple of m = 128 words and replace the string by the values
    (b_j + sum_i a_{j,i} s_i) mod p of its chunks (Sec. 5, eq. 2wlinear),
    with the key row of level j, until one value is left (at least one level
    is applied). Shares nothing with the oracle but the key words."""
    W = width // 8
    p = 2 ** width + (15 if width == 32 else 13)
    m = 128
    padded = bytes(data) + b"\x01"
    padded += b"\x00" * (-len(padded) % W)
    sigma = [int.from_bytes(padded[i:i + W], "little") for i in range(0, len(padded), W)]
    j = 0
    while True:
        sigma += [0] * (-len(sigma) % m)
        row = [int(x) for x in key[j * (m + 1):(j + 1) * (m + 1)]]
        b, a = row[0], row[1:]
        sigma = [(b + sum(ai * si for ai, si in zip(a, sigma[c:c + m]))) % p
                 for c in range(0, len(sigma), m)]
        j += 1
        if len(sigma) == 1:
            return sigma[0]


@pytest.mark.parametrize("width", [32, 64])
def test_whole_hash_matches_arbitrary_precision_restatement(width):
    """Every length 0..2*128*W + 16 and the lengths around m and m^2 words,
    with the seeded key of each width: the oracle's tree value equals the
    arbitrary-precision evaluation of eq. 2wlinear and Algorithm 1. Random
    full-width key words and message words exercise every limb and carry of
    the oracle's multi-level arithmetic."""
    from paper_1609_09840_gb300 import synth

    W = width // 8
    P = pmo.width_params(width)
    key = pmo.key_expand(P, 20260001 + width)
    buf = synth.bytes_np(synth.derive(77, synth.TAG_BYTES), 0, 128 * 128 * W + 4 * W)
    lengths = list(range(0, 2 * 128 * W + 17))
    for nw in (128, 128 * 128):
        lengths += [nw * W + d for d in (-W - 1, -W, -1, 0, 1, W - 1, W)]
    for L in lengths:
        want = bigint_tree(width, key, buf[:L].tobytes())
        assert pmo.tree_bytes(P, key, buf[:L]) == want, L


def test_arbitrary_precision_restatement_by_hand():
    """The restatement itself, on values worked out by hand: a string of
    fewer than four bytes is one word (its bytes, then the 0x01 pad), a
    four-byte string is one word followed by the pad word 1."""
    key = np.zeros(8 * 129, dtype=np.uint64)
    key[0], key[1], key[2] = 5, 7, 11
    p = 2 ** 32 + 15
    # "abc" -> word 0x01636261 (pad byte after the data), one chunk
    assert bigint_tree(32, key, b"abc") == (5 + 7 * 0x01636261) % p
    # four bytes: the pad is a word of its own, weight a_2
    assert bigint_tree(32, key, b"abcd") == (5 + 7 * 0x64636261 + 11 * 1) % p
