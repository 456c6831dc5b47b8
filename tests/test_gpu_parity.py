"""Bit-exact parity of the CUDA path with the CPU oracle (needs a GPU).

Every input is seeded and synthetic (paper_1609_09840_gb300.synth); every
expected value comes from the oracle (oracle/pmo.c). Integer hashing: the bar
is bit-exact equality.
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
    ks = {w: native.Key(seed=1, width=w) for w in WIDTHS}
    yield ks
    for k in ks.values():
        k.close()


BATCH_SCHEDULES = [("sorted", 512), ("sorted", 1024), ("tiles", 6), ("tiles", 8)]


@pytest.fixture(params=BATCH_SCHEDULES, ids=["sorted-512", "sorted-1024", "tiles-p1-6", "tiles-p1-8"])
def batch_kernel(native, request):
    """Run a batched test with each schedule of the one-chunk strings: the
    sorted ranges at each range size, and the tiles at each pass-1 depth
    (results must not depend on them)."""
    sched, v = request.param
    knobs = (native.KNOB_BATCH_SCHED, native.KNOB_BATCH_RANGE, native.KNOB_BATCH_P1)
    old = [native.tune_get(k) for k in knobs]
    if sched == "sorted":
        native.tune_set(native.KNOB_BATCH_SCHED, native.BATCH_SORTED)
        native.tune_set(native.KNOB_BATCH_RANGE, v)
    else:
        native.tune_set(native.KNOB_BATCH_SCHED, native.BATCH_TILES)
        native.tune_set(native.KNOB_BATCH_P1, v)
    yield request.param
    for k, o in zip(knobs, old):
        native.tune_set(k, o)


def okey(width, seed=1):
    return pmo.key_expand(pmo.width_params(width), seed)


def run_batch(native, key, batch, raw=False, plain=False):
    host = batch.host_bytes()
    base = torch.from_numpy(host).cuda()
    offsets = torch.from_numpy(batch.offsets).cuda()
    if plain:
        out = native.hash_batch_plain(key, base, offsets)
    else:
        out = native.hash_batch(key, base, offsets, raw=raw)
    torch.cuda.synchronize()
    return host, out


def expect_batch(width, host, batch, raw=False, seed=1):
    return pmo.hash_batch(pmo.width_params(width), okey(width, seed), host, batch.offsets, raw=raw)


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("seed", [0, 1, 2, 12345, 2 ** 64 - 1])
def test_key_expansion_matches_oracle(native, width, seed):
    k = native.Key(seed=seed, width=width)
    assert np.array_equal(k.export().astype(np.uint64), okey(width, seed))
    k.close()


@pytest.mark.parametrize("width", WIDTHS)
def test_device_reduction_matches_generic_remainder(native, width):
    """Sec. 6.2 + Algorithm 2 on the device vs the oracle's long division, on
    the branch boundaries of Algorithm 2 and on random three-word sums."""
    P = pmo.width_params(width)
    n, k = P.n, P.k
    p = pmo.prime(P)
    smax = ((1 << n) - 1) + 128 * ((1 << (2 * n)) - 1)
    rng = np.random.default_rng(width)
    cases = []
    for v1 in range(3):
        for v0 in list(range(0, 3 * k + 2)) + [(1 << n) - d for d in range(1, 5)]:
            cases.append(v0 + (v1 << n))
    for w2 in (0, 1, 127, 128):
        for w1 in (0, 1, (1 << n) - 1, (1 << n) - 2):
            for w0 in (0, 1, k, (1 << n) - 1):
                S = w0 + (w1 << n) + (w2 << (2 * n))
                if S <= smax:
                    cases.append(S)
    cases.append(smax)
    for _ in range(4000):
        cases.append(int.from_bytes(rng.bytes(40), "little") % (smax + 1))
    words = np.array([[(S >> (64 * i)) & (2 ** 64 - 1) for i in range(3)] for S in cases],
                     dtype=np.uint64)
    z = native.debug_reduce(width, torch.from_numpy(words.view(np.int64)).cuda())
    z = z.cpu().numpy().view(np.uint64)
    for S, (lo, hi) in zip(cases, z):
        got = int(lo) + (int(hi) << 64)
        assert got == pmo.mod(P, S), hex(S)
        assert got < p


def boundary_lengths(width):
    W = width // 8
    m = 128
    ls = set(range(0, 2 * m * W + 17))
    for nw in (m, m * m, 2 * m * m):
        for d in (-W - 1, -W, -1, 0, 1, W, W + 1):
            ls.add(nw * W + d)
    ls.update((65535, 65536, 65537))
    return np.array(sorted(x for x in ls if x >= 0), dtype=np.int64)


@pytest.mark.parametrize("width", WIDTHS)
def test_batch_boundary_lengths(native, keys, width, batch_kernel):
    """Every length up to two chunks plus the level boundaries (N0 crossing
    m and m^2), through the batched path (short and long strings)."""
    batch = synth.Batch("bounds", 101, boundary_lengths(width))
    host, out = run_batch(native, keys[width], batch)
    want = expect_batch(width, host, batch)
    got = native.as_unsigned(out).astype(np.uint64)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, [(int(batch.lengths[i]), hex(int(got[i])), hex(int(want[i]))) for i in bad[:10]]


@pytest.mark.parametrize("width", WIDTHS)
def test_batch_all_ones_content(native, keys, width, batch_kernel):
    """Strings of 0xff bytes of every length up to two chunks: every word at
    its maximum drives the carry-free accumulators and the limb sums of the
    reduction (Sec. 6.2) to their largest values."""
    batch = synth.Batch("ones", 0, boundary_lengths(width))
    host = np.full(batch.buffer_bytes, 0xFF, dtype=np.uint8)
    base = torch.from_numpy(host).cuda()
    offsets = torch.from_numpy(batch.offsets).cuda()
    raw = native.hash_batch(keys[width], base, offsets, raw=True).cpu().numpy().view(np.uint64)
    want = expect_batch(width, host, batch, raw=True)
    bad = np.nonzero(raw.reshape(-1, 2) != want.reshape(-1, 2))[0]
    assert bad.size == 0, [int(batch.lengths[i]) for i in bad[:10]]


@pytest.mark.parametrize("width", WIDTHS)
def test_batch_long_string_paths(native, keys, width, batch_kernel):
    """Strings around the split between the warp-inline path of the tile
    kernel and the per-chunk kernel (32 chunks), around one and two level-2 chunks
    (m and 2m chunks, where a third level starts), each preceded by strings
    of 1 and 8 bytes so that they start at 8 and 16 modulo 16."""
    W = width // 8
    CB = 128 * W
    around = []
    for chunks in (31, 32, 33, 127, 128, 129, 255, 256, 257):
        for d in (-9, -1, 0, 1, 7):
            around.append(chunks * CB + d)
    lengths = []
    for i, L in enumerate(around):
        lengths += [1 if i % 2 else 8, L]
    batch = synth.Batch("longpaths", 103, lengths)
    host, out = run_batch(native, keys[width], batch)
    want = expect_batch(width, host, batch)
    got = native.as_unsigned(out).astype(np.uint64)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, [int(batch.lengths[i]) for i in bad[:10]]
    starts = batch.starts[1::2] % 16
    assert set(int(x) for x in starts) == {0, 8}


@pytest.mark.parametrize("width", WIDTHS)
def test_batch_scratch_too_small_reports_escratch(native, keys, width, batch_kernel):
    """Scratch sized for far fewer bytes than the batch holds (a 16 MiB string
    needs more work items and tree storage than it covers): the string is
    refused, the device status reports PMP_ESCRATCH, and the strings of
    fewer than 32 chunks (which need no scratch) are still hashed."""
    W = width // 8
    lengths = [5, 17, 3 * 128 * W + 9, 40, (16 << 20) + 24, 63]
    batch = synth.Batch("small_scratch", 104, lengths)
    host = batch.host_bytes()
    base = torch.from_numpy(host).cuda()
    offsets = torch.from_numpy(batch.offsets).cuda()
    assert native.device_status() == 0
    scr = torch.empty(native.batch_scratch_bytes(width, batch.n, 64), dtype=torch.uint8, device="cuda")
    out = torch.empty(batch.n, dtype=torch.int32 if width == 32 else torch.int64, device="cuda")
    lib = native.load()
    fn = lib.pmp_hash_batch32 if width == 32 else lib.pmp_hash_batch64
    rc = fn(keys[width].handle, base.data_ptr(), offsets.data_ptr(), batch.n, out.data_ptr(),
            scr.data_ptr(), scr.numel(), None)  # through the C ABI: the binding would enlarge the scratch
    assert rc == native.PMP_OK
    assert native.device_status() == native.PMP_ESCRATCH
    want = expect_batch(width, host, batch)
    got = native.as_unsigned(out).astype(np.uint64)
    short = [i for i, L in enumerate(lengths) if L < 31 * 128 * W]
    assert np.array_equal(got[short], want[short])


@pytest.mark.parametrize("width", WIDTHS)
def test_batch_raw_values(native, keys, width, batch_kernel):
    batch = synth.Batch("raw", 102, boundary_lengths(width)[::7])
    host, out = run_batch(native, keys[width], batch, raw=True)
    want = expect_batch(width, host, batch, raw=True)
    assert np.array_equal(out.cpu().numpy().view(np.uint64), want)


@pytest.mark.parametrize("width", WIDTHS)
def test_c1_uniform_strings_batched_and_plain(native, keys, width, batch_kernel):
    """The 10,000-string case (lengths 1..256): batched and one launch per string."""
    batch = synth.workload_c1()
    host, out = run_batch(native, keys[width], batch)
    want = expect_batch(width, host, batch)
    assert np.array_equal(native.as_unsigned(out).astype(np.uint64), want)
    _, outp = run_batch(native, keys[width], batch, plain=True)
    assert np.array_equal(native.as_unsigned(outp).astype(np.uint64), want)


@pytest.mark.parametrize("width", WIDTHS)
def test_lognormal_batch_small(native, keys, width, batch_kernel):
    """200k strings with the batched case's length law (median 24 B, sigma 1,
    up to 64 KiB)."""
    batch = synth.workload_c3(n=200_000, seed=3)
    host, out = run_batch(native, keys[width], batch)
    want = expect_batch(width, host, batch)
    assert np.array_equal(native.as_unsigned(out).astype(np.uint64), want)


@pytest.mark.parametrize("width", WIDTHS)
def test_one_chunk_tiles(native, keys, width, batch_kernel):
    """Tiles of one-chunk strings only: all-empty tiles, tiles of 1-byte
    strings, tiles of the longest one-chunk strings (every string continues
    in pass 2), lengths that are multiples of 8 (the pad in a unit of its
    own), and random mixes with empty strings in between."""
    CB = 128 * width // 8
    rng = np.random.default_rng(width + 7)
    parts = [np.zeros(64, np.int64), np.ones(64, np.int64), np.full(64, CB - 1, np.int64),
             8 * rng.integers(0, CB // 8, 192), rng.integers(CB - 9, CB, 128),
             np.repeat(np.array([0, 1, 7, 8, 9, CB - 8, CB - 1, 0]), 24)]
    for _ in range(40):
        k = int(rng.integers(1, 200))
        mix = rng.choice([0, 1, 3, 8, 16, 24, 31, 64, 100, CB // 2, CB - 8, CB - 1], k)
        parts.append(np.where(rng.random(k) < 0.5, mix, rng.integers(0, CB, k)))
    lengths = np.concatenate(parts).astype(np.int64)
    batch = synth.Batch("tiles", 211, lengths)
    host, out = run_batch(native, keys[width], batch)
    want = expect_batch(width, host, batch)
    got = native.as_unsigned(out).astype(np.uint64)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, [(int(i), int(batch.lengths[i])) for i in bad[:10]]


@pytest.mark.parametrize("width", WIDTHS)
def test_staging_fills(native, keys, width, batch_kernel):
    """Batches whose one-chunk strings do not fit one staging fill of the
    sorted schedule (56 KiB per fill for ranges of 1024 strings, 28 KiB for
    ranges of 512): ranges of the
    longest one-chunk strings (a run cut into many fills, a fill starting in
    the middle of a run), runs of one string between strings of 3 and 31
    chunks, the first offset not 8-byte aligned, and a count that is not a
    multiple of the range size."""
    W = width // 8
    CB = 128 * W
    rng = np.random.default_rng(width + 31)
    parts = [np.full(2500, CB - 1, np.int64), rng.integers(CB - 64, CB, 1500),
             np.tile(np.array([CB - 1, 2 * CB + 5, 3, CB * 31 - 7, 0, CB - 8], np.int64), 300),
             np.tile(np.array([17, 2 * CB], np.int64), 700),
             rng.integers(0, 64, 3000), np.full(1024, 48, np.int64), np.full(777, 200, np.int64)]
    lengths = np.concatenate(parts).astype(np.int64)
    batch = synth.Batch("fills", 212, lengths)
    host = batch.host_bytes()
    # shift every string by 3 bytes: offsets[0] = 3, starts stay 8-byte aligned
    off = batch.offsets.copy()
    off[0] = 3
    base = torch.from_numpy(host).cuda()
    offsets = torch.from_numpy(off).cuda()
    out = native.hash_batch(keys[width], base, offsets)
    torch.cuda.synchronize()
    want = pmo.hash_batch(pmo.width_params(width), okey(width), host, off)
    got = native.as_unsigned(out).astype(np.uint64)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, [(int(i), int(lengths[i])) for i in bad[:10]]


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("n", [1, 2, 3, 511, 512, 513, 1023, 1024, 1025, 4097])
def test_offsets_at_8_mod_16(native, keys, width, n, batch_kernel):
    """An offsets array that starts 8 bytes past a 16-byte boundary (a view
    one entry into a larger array), at string counts that leave every
    parity of a range's entry count and a short last range: the oracle's
    values."""
    rng = np.random.default_rng(n + width)
    lengths = np.minimum(rng.lognormal(np.log(24), 1.0, n).astype(np.int64), 2000)
    batch = synth.Batch("off8", 213 + n, lengths)
    host = batch.host_bytes()
    base = torch.from_numpy(host).cuda()
    whole = torch.zeros(n + 2, dtype=torch.int64, device="cuda")
    whole[1:] = torch.from_numpy(batch.offsets).cuda()
    offsets = whole[1:]
    assert offsets.data_ptr() % 16 == 8
    out = native.hash_batch(keys[width], base, offsets)
    want = pmo.hash_batch(pmo.width_params(width), okey(width), host, batch.offsets)
    got = native.as_unsigned(out).astype(np.uint64)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, [(int(i), int(lengths[i])) for i in bad[:10]]


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("stages", [2, 3])
def test_chunk_kernel_every_staging_depth(native, keys, width, stages):
    """Strings of 32 or more level-1 chunks (one, two and three level-2
    segments, at 8 and 16 modulo 16) hashed by the chunk kernel at each
    staging depth the autotuner may pick: the oracle's values."""
    W = width // 8
    CB = 128 * W
    lengths = []
    for i, L in enumerate([32 * CB, 32 * CB + 9, 128 * CB - 1, 128 * CB + 5, 300 * CB + 17, 257 * CB]):
        lengths += [1 if i % 2 else 8, L]
    batch = synth.Batch("stages", 107, lengths)
    knob = native.KNOB_CHUNK_STAGES_32 if width == 32 else native.KNOB_CHUNK_STAGES_64
    old = native.tune_get(knob)
    native.tune_set(knob, stages)
    try:
        host, out = run_batch(native, keys[width], batch)
    finally:
        native.tune_set(knob, old)
    want = expect_batch(width, host, batch)
    assert np.array_equal(native.as_unsigned(out).astype(np.uint64), want)


@pytest.mark.parametrize("width", WIDTHS)
def test_skewed_batch_small(native, keys, width, batch_kernel):
    """The skewed mix at reduced size: short 8..64 B strings plus 1% long
    strings (64..700 KiB here), with zero and repeated-byte content."""
    batch = synth.workload_c4(n=20_000, seed=4, long_lo=64 << 10, long_hi=700 << 10)
    host, out = run_batch(native, keys[width], batch)
    want = expect_batch(width, host, batch)
    assert np.array_equal(native.as_unsigned(out).astype(np.uint64), want)


def single_lengths(width):
    W = width // 8
    m = 128
    ls = {0, 1, 2, 15, 16, 17, 100, m * W - 1, m * W, m * W + 1, m * W + 16, 2 * m * W,
          m * m * W - 16, m * m * W, m * m * W + 16, 128 * m * W * 3 + 48, m * m * W * 2,
          m * m * m * W - 16, m * m * m * W, m * m * m * W + 32, 5 * m * m * m * W // 2 + 64}
    return sorted(ls)


@pytest.mark.parametrize("width", WIDTHS)
def test_single_buffer_lengths(native, keys, width):
    """One buffer through the fused tree kernel: every level count from 1 to 4
    (5 for PM+32), tails of every kind, and level-2 tiles that are complete,
    partial or hold only the padding chunk."""
    P = pmo.width_params(width)
    ok = okey(width)
    maxlen = max(single_lengths(width))
    data = synth.bytes_np(synth.derive(77, synth.TAG_BYTES), 0, maxlen)
    dev = torch.from_numpy(data).cuda()
    for length in single_lengths(width):
        got = int(native.as_unsigned(native.hash(keys[width], dev[:length] if length else dev[:0],
                                                  length=length))[0])
        assert got == pmo.hash_bytes(P, ok, data[:length]), length
    assert native.device_status() == 0


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("stages", [2, 3, 4, 6])
def test_single_buffer_every_staging_depth(native, keys, width, stages):
    """Every staging depth the autotuner may pick gives the oracle's values."""
    P = pmo.width_params(width)
    ok = okey(width)
    knob = native.KNOB_TREE_STAGES_32 if width == 32 else native.KNOB_TREE_STAGES_64
    old = native.tune_get(knob)
    native.tune_set(knob, stages)
    try:
        W = width // 8
        lengths = [0, 5, 128 * W * 128 - 8, 128 * W * 128 * 3 + 40, 128 * W * 128 * 130 + 24]
        data = synth.bytes_np(synth.derive(78, synth.TAG_BYTES), 0, max(lengths))
        dev = torch.from_numpy(data).cuda()
        for length in lengths:
            got = int(native.as_unsigned(native.hash(keys[width], dev[:length], length=length))[0])
            assert got == pmo.hash_bytes(P, ok, data[:length]), (stages, length)
    finally:
        native.tune_set(knob, old)


def test_tuning_knobs_reject_bad_values(native):
    with pytest.raises(native.PmpError):
        native.tune_set(native.KNOB_TREE_STAGES_32, 5)
    with pytest.raises(native.PmpError):
        native.tune_set(native.KNOB_BATCH_P1, 7)
    with pytest.raises(native.PmpError):
        native.tune_set(native.KNOB_BATCH_SCHED, 2)
    with pytest.raises(native.PmpError):
        native.tune_set(native.KNOB_BATCH_RANGE, 768)
    with pytest.raises(native.PmpError):
        native.tune_set(native.KNOB_CHUNK_STAGES_64, 4)
    with pytest.raises(native.PmpError):
        native.tune_set(native.KNOB_CHUNK_STAGES_32, 1)
    with pytest.raises(native.PmpError):
        native.tune_set(99, 4)


def _solve_word(P, fkey, words, r, y):
    """Word s_r that makes f(words) == y, or None if it is not below 2^n
    (component-wise regularity, Sec. 5: s_r = a_r^{-1}(y - b - sum_{i!=r} a_i s_i))."""
    p = pmo.prime(P)
    rest = (fkey[0] + sum(int(a) * int(s) for i, (a, s) in enumerate(zip(fkey[1:], words)) if i != r)) % p
    s = (y - rest) * pow(int(fkey[1 + r]), -1, p) % p
    return s if s < (1 << P.n) else None


@pytest.mark.parametrize("width", WIDTHS)
def test_level_values_in_the_top_range(native, keys, width, batch_kernel):
    """Crafted strings whose level values lie in [2^n, p): a level-1 chunk value
    feeding level 2 (the extra high bit of Sec. 6.1), and a one-level hash whose
    output step maps it into [0, k)."""
    P = pmo.width_params(width)
    W = width // 8
    ok = okey(width)
    f1 = [int(x) for x in ok[:129]]
    rng = np.random.default_rng(width + 5)
    p = pmo.prime(P)
    strings = []
    for target in range(1 << P.n, p):
        # two-level string: first chunk (128 full words) has value `target`
        words = [int(x) for x in rng.integers(0, 1 << min(P.n, 63), 128, dtype=np.uint64)]
        s = _solve_word(P, f1, words, 77, target)
        if s is None:
            continue
        words[77] = s
        data = b"".join(w.to_bytes(W, "little") for w in words) + rng.bytes(40 * W + 3)
        strings.append(data)
        # one-level string: 20 data words + pad; solve word 3 for the tree value
        short = [int(x) for x in rng.integers(0, 1 << min(P.n, 63), 20, dtype=np.uint64)]
        sigma = short + [1] + [0] * 107
        s = _solve_word(P, f1, sigma, 3, target)
        if s is not None:
            short[3] = s
            strings.append(b"".join(w.to_bytes(W, "little") for w in short))
    assert len(strings) >= 2 * (p - (1 << P.n)) - 4
    lengths = np.array([len(x) for x in strings], dtype=np.int64)
    batch = synth.Batch("top", 0, lengths)
    host = np.zeros(batch.buffer_bytes, dtype=np.uint8)
    for i, x in enumerate(strings):
        st = int(batch.starts[i])
        host[st:st + len(x)] = np.frombuffer(x, dtype=np.uint8)
    base = torch.from_numpy(host).cuda()
    offs = torch.from_numpy(batch.offsets).cuda()
    raw = native.hash_batch(keys[width], base, offs, raw=True).cpu().numpy().view(np.uint64)
    want_raw = pmo.hash_batch(P, ok, host, batch.offsets, raw=True)
    assert np.array_equal(raw, want_raw)
    # the one-level strings really produced values >= 2^n
    hi = raw.reshape(-1, 2)
    vals = [int(lo) + (int(h) << 64) for lo, h in hi]
    assert sum(v >= (1 << P.n) for v in vals) >= p - (1 << P.n) - 2
    out = native.as_unsigned(native.hash_batch(keys[width], base, offs)).astype(np.uint64)
    assert np.array_equal(out, pmo.hash_batch(P, ok, host, batch.offsets))


@pytest.mark.parametrize("width", WIDTHS)
def test_single_buffer_1gib(native, keys, width):
    """The 1 GiB single-buffer case (seed 2), hashed through all levels."""
    P = pmo.width_params(width)
    seed = synth.workload_c2_bytes(2)
    dev = torch.empty(synth.C2_BYTES, dtype=torch.uint8, device="cuda")
    synth.fill_bytes_torch(dev, seed)
    key = native.Key(seed=2, width=width)
    got = int(native.as_unsigned(native.hash(key, dev))[0])
    host = synth.bytes_np(seed, 0, synth.C2_BYTES)
    assert np.array_equal(host[:4096], dev[:4096].cpu().numpy())
    want = pmo.hash_bytes(P, okey(width, 2), host)
    assert got == want
    key.close()


def test_device_status_clean(native):
    assert native.device_status() == 0


@pytest.mark.parametrize("width", WIDTHS)
def test_cuda_graph_replay_matches_direct_calls(native, keys, width):
    """A captured batched call and a captured single-buffer call give the
    oracle's values on every replay, also after the input bytes change."""
    P = pmo.width_params(width)
    ok = okey(width)
    batch = synth.workload_c3(n=50_000, seed=31)
    host = batch.host_bytes()
    base = torch.from_numpy(host).cuda()
    offs = torch.from_numpy(batch.offsets).cuda()
    out = torch.empty(batch.n, dtype=torch.int32 if width == 32 else torch.int64, device="cuda")
    g = native.graph_batch(keys[width], base, offs, out)
    for rep in range(3):
        if rep == 2:  # new content, same layout
            host = synth.bytes_np(synth.derive(99, synth.TAG_BYTES), 0, host.size)
            base.copy_(torch.from_numpy(host))
        out.fill_(0)
        g.launch()
        torch.cuda.synchronize()
        want = pmo.hash_batch(P, ok, host, batch.offsets)
        assert np.array_equal(native.as_unsigned(out).astype(np.uint64), want)
    g.close()
    buf = torch.from_numpy(host[: 3 * 128 * 128 * (width // 8) + 40].copy()).cuda()
    out1 = torch.zeros(1, dtype=torch.int32 if width == 32 else torch.int64, device="cuda")
    g1 = native.graph_hash(keys[width], buf, out1)
    g1.launch()
    g1.launch()
    torch.cuda.synchronize()
    assert int(native.as_unsigned(out1)[0]) == pmo.hash_bytes(P, ok, buf.cpu().numpy())
    g1.close()
