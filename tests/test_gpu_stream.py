"""Streaming hashing (pmp_stream_*) against the oracle (needs a GPU).

Sec. 4: the tree of Algorithm 1 can be evaluated while the string is read
once. The hash of a string fed in pieces must equal the oracle's hash of the
whole string (and the single-buffer path's), bit for bit, for every split:
pieces at every alignment, empty pieces, byte-at-a-time feeding, and
updates that span many update segments and several tree levels.
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
    ks = {w: native.Key(seed=7, width=w) for w in WIDTHS}
    yield ks
    for k in ks.values():
        k.close()


def okey(width):
    return pmo.key_expand(pmo.width_params(width), 7)


def expect(width, data):
    return pmo.hash_bytes(pmo.width_params(width), okey(width), data)


def stream_hash(native, key, dev_bytes, cuts, offset=0):
    """Feed dev_bytes[offset:] cut at `cuts` (positions relative to the string)."""
    s = native.Stream(key)
    n = dev_bytes.numel() - offset
    bounds = [0] + sorted(cuts) + [n]
    for a, b in zip(bounds[:-1], bounds[1:]):
        s.update(dev_bytes[offset + a: offset + b])
    out = s.final()
    s.close()
    return int(native.as_unsigned(out)[0])


def lengths(width):
    CB = 128 * (width // 8)
    return [0, 1, 7, 8, 9, CB - 1, CB, CB + 1, 3 * CB + 5, 128 * CB - 3, 128 * CB, 128 * CB + 9,
            2 * 128 * CB + 17]


@pytest.mark.parametrize("width", WIDTHS)
def test_stream_random_splits_match_oracle(native, keys, width):
    rng = np.random.default_rng(width)
    for L in lengths(width):
        host = synth.bytes_np(synth.derive(300 + L, synth.TAG_BYTES), 0, L + 16)
        dev = torch.from_numpy(host).cuda()
        want = expect(width, host[3: 3 + L])
        for trial in range(3):
            k = int(rng.integers(0, 6)) if L else 0
            cuts = sorted(int(x) for x in rng.integers(0, L + 1, size=k))
            got = stream_hash(native, keys[width], dev[: 3 + L], cuts, offset=3)  # odd start address
            assert got == want, (L, cuts)


@pytest.mark.parametrize("width", WIDTHS)
def test_stream_equals_single_buffer_at_every_alignment(native, keys, width):
    CB = 128 * (width // 8)
    L = 5 * CB + 77
    host = synth.bytes_np(synth.derive(401, synth.TAG_BYTES), 0, L + 32)
    dev = torch.from_numpy(host).cuda()
    for off in range(8):
        want = expect(width, host[off: off + L])
        for first in (1, 3, 8, CB - 1, CB, CB + 5):
            got = stream_hash(native, keys[width], dev[: off + L], [first, first + CB + 3], offset=off)
            assert got == want, (off, first)


@pytest.mark.parametrize("width", WIDTHS)
def test_stream_byte_at_a_time_and_empty_pieces(native, keys, width):
    CB = 128 * (width // 8)
    L = CB + 40
    host = synth.bytes_np(synth.derive(402, synth.TAG_BYTES), 0, L)
    dev = torch.from_numpy(host).cuda()
    s = native.Stream(keys[width])
    for i in range(L):
        s.update(dev[i: i + 1])
        if i % 97 == 0:
            s.update(dev[i: i])  # empty piece
    assert len(s) == L
    got = int(native.as_unsigned(s.final())[0])
    s.close()
    assert got == expect(width, host)


@pytest.mark.parametrize("width", WIDTHS)
def test_stream_final_keeps_state_and_reset(native, keys, width):
    CB = 128 * (width // 8)
    host = synth.bytes_np(synth.derive(403, synth.TAG_BYTES), 0, 200 * CB + 11)
    dev = torch.from_numpy(host).cuda()
    s = native.Stream(keys[width])
    s.update(dev[: 130 * CB + 5])
    mid = int(native.as_unsigned(s.final())[0])
    assert mid == expect(width, host[: 130 * CB + 5])
    s.update(dev[130 * CB + 5:])
    assert int(native.as_unsigned(s.final())[0]) == expect(width, host)
    s.reset()
    assert len(s) == 0
    assert int(native.as_unsigned(s.final())[0]) == expect(width, host[:0])
    s.update(dev[:7])
    assert int(native.as_unsigned(s.final())[0]) == expect(width, host[:7])
    s.close()


@pytest.mark.parametrize("width", WIDTHS)
def test_stream_raw_value_in_top_range_path(native, keys, width):
    """The raw tree value of a streamed string equals the oracle's tree value."""
    P = pmo.width_params(width)
    CB = 128 * (width // 8)
    host = synth.bytes_np(synth.derive(404, synth.TAG_BYTES), 0, 3 * CB + 1)
    dev = torch.from_numpy(host).cuda()
    s = native.Stream(keys[width])
    s.update(dev[:CB + 2])
    s.update(dev[CB + 2:])
    raw = torch.zeros(2, dtype=torch.int64, device="cuda")
    s.final(raw=raw)
    s.close()
    lo, hi = (int(x) for x in raw.cpu().numpy().view(np.uint64))
    assert lo + (hi << 64) == pmo.tree_bytes(P, okey(width), host)


@pytest.fixture(params=[1 << 17, 1 << 18, 1 << 19], ids=["seg-2^17", "seg-2^18", "seg-2^19"])
def segment(native, request):
    """Every update segment size the autotuner may pick."""
    old = native.tune_get(native.KNOB_STREAM_SEGMENT)
    native.tune_set(native.KNOB_STREAM_SEGMENT, request.param)
    yield request.param
    native.tune_set(native.KNOB_STREAM_SEGMENT, old)


@pytest.mark.parametrize("width", WIDTHS)
def test_stream_large_updates_across_segments(native, keys, width, segment):
    """Updates of 2^17 and more chunks (several update segments), cut at odd
    places, through three levels, from a start address that is not even
    2-byte aligned; checked against the single-buffer path on a 16-byte
    aligned copy of the same bytes (that path is pinned to the oracle by the
    parity tests)."""
    CB = 128 * (width // 8)
    L = (3 << 16) * CB + 12345  # about 100 MiB (PM+32) / 200 MiB (PM+64)
    buf = torch.empty((L + 16 + 7) // 8 * 8, dtype=torch.uint8, device="cuda")
    synth.fill_bytes_torch(buf, synth.derive(405, synth.TAG_BYTES))
    aligned = buf[5: 5 + L].clone()
    want = int(native.as_unsigned(native.hash(keys[width], aligned))[0])
    got = stream_hash(native, keys[width], buf[: 5 + L], [3, (1 << 17) * CB + 1001, L - 17], offset=5)
    assert got == want


@pytest.mark.parametrize("width", WIDTHS)
def test_stream_level2_mode_and_lazy_folds(native, keys, width):
    """Pieces of thousands of whole chunks that start a level-2 chunk go
    through the tree kernel's level-2 mode (their level-2 values wait to be
    folded into level 3); a piece that ends inside a level-2 chunk leaves a
    partial sum; the next piece starts mid-chunk (level-1 mode, after the
    waiting values are folded); a result asked for half way folds them too
    and the string continues. Checked against the single-buffer path on the
    same bytes, for the prefix and the whole string."""
    CB = 128 * (width // 8)
    T = 128 * CB  # bytes of one level-2 chunk
    L = 300 * T + 777
    buf = torch.empty((L + 16 + 7) // 8 * 8, dtype=torch.uint8, device="cuda")
    synth.fill_bytes_torch(buf, synth.derive(406, synth.TAG_BYTES))
    cuts = [0, 40 * T, 73 * T + 50 * CB, 73 * T + 50 * CB + 4096 * CB + 3, 200 * T, 232 * T, 260 * T + 5, L]
    s = native.Stream(keys[width])
    for a, b in zip(cuts[:-1], cuts[1:]):
        s.update(buf[a:b])
        if b == 200 * T:
            mid = int(native.as_unsigned(s.final())[0])
    whole = int(native.as_unsigned(s.final())[0])
    s.close()
    assert mid == int(native.as_unsigned(native.hash(keys[width], buf[:200 * T].clone()))[0])
    assert whole == int(native.as_unsigned(native.hash(keys[width], buf[:L].clone()))[0])


@pytest.mark.parametrize("width", WIDTHS)
def test_stream_result_with_waiting_level2_values(native, keys, width):
    """Results asked for while level-2 values of the tree kernel's level-2
    mode still wait (their fold into level 3 and up and the final chunk run
    in one launch): after 64 level-2 chunks (level 3 partial), after 150
    (a level-3 chunk completed), after 300, and after a short tail appended
    to the carried bytes; each equals the single-buffer hash of the prefix."""
    CB = 128 * (width // 8)
    T = 128 * CB  # bytes of one level-2 chunk
    L = 300 * T + 777
    buf = torch.empty((L + 16 + 7) // 8 * 8, dtype=torch.uint8, device="cuda")
    synth.fill_bytes_torch(buf, synth.derive(407, synth.TAG_BYTES))
    s = native.Stream(keys[width])
    got, want = [], []
    for a, b in ((0, 64 * T), (64 * T, 150 * T), (150 * T, 300 * T), (300 * T, L)):
        s.update(buf[a:b])
        got.append(int(native.as_unsigned(s.final())[0]))
        want.append(int(native.as_unsigned(native.hash(keys[width], buf[:b].clone()))[0]))
    s.close()
    assert got == want


@pytest.mark.parametrize("width", WIDTHS)
def test_stream_level2_updates_keep_stream_order(native, keys, width):
    """Level-2 mode updates overlap one another (each is a programmatic
    dependent of the one before), but stream order holds for everything
    else. One piece buffer is refilled on the same CUDA stream before every
    update, so an update that read its piece early, or a refill that ran
    before the previous update had read it, would change the hash. Two
    strings' updates are interleaved with a batch call (whose chunk kernel
    follows it) and a single-buffer hash on the same stream."""
    CB = 128 * (width // 8)
    T = 128 * CB  # bytes of one level-2 chunk
    P = 40 * T    # 40 level-2 chunks per piece (at least 4096 level-1 chunks)
    src = torch.empty(6 * P, dtype=torch.uint8, device="cuda")
    synth.fill_bytes_torch(src, synth.derive(408, synth.TAG_BYTES))
    piece = torch.empty(P, dtype=torch.uint8, device="cuda")
    batch = synth.Batch("order", 409, np.array([17, 40 * CB + 9, 3, 200 * CB + 1], dtype=np.int64))
    bbase = torch.from_numpy(batch.host_bytes()).cuda()
    boffs = torch.from_numpy(batch.offsets).cuda()
    a, b = native.Stream(keys[width]), native.Stream(keys[width])
    outs = []
    for k in range(6):
        piece.copy_(src[k * P:(k + 1) * P])
        (a if k % 2 == 0 else b).update(piece)
        if k == 2:
            outs.append(native.hash_batch(keys[width], bbase, boffs))
        if k == 3:
            outs.append(native.hash(keys[width], src[:P]))
    got_a = int(native.as_unsigned(a.final())[0])
    got_b = int(native.as_unsigned(b.final())[0])
    a.close()
    b.close()
    even = torch.cat([src[k * P:(k + 1) * P] for k in (0, 2, 4)])
    odd = torch.cat([src[k * P:(k + 1) * P] for k in (1, 3, 5)])
    assert got_a == int(native.as_unsigned(native.hash(keys[width], even))[0])
    assert got_b == int(native.as_unsigned(native.hash(keys[width], odd))[0])
    want_batch = pmo.hash_batch(pmo.width_params(width), okey(width), batch.host_bytes(), batch.offsets)
    assert np.array_equal(native.as_unsigned(outs[0]).astype(np.uint64), want_batch)
    assert int(native.as_unsigned(outs[1])[0]) == int(native.as_unsigned(native.hash(keys[width], src[:P].clone()))[0])


@pytest.mark.parametrize("width", WIDTHS)
def test_stream_results_back_to_back_without_sync(native, keys, width):
    """Results are launched as programmatic dependents of the update before
    them (they may start while a level-2 update drains, and wait for it
    before reading its values). Strings are hashed back to back on one CUDA
    stream with no host synchronisation: a result right after a level-2
    update, a result half way through a string that then grows, a reset
    after a result, a result after an unaligned update that only carries
    bytes, and the empty string. The one piece buffer is refilled on the
    stream before every update. Every result must equal the oracle's."""
    CB = 128 * (width // 8)
    P = 40 * 128 * CB  # 40 level-2 chunks per piece: level-2 mode updates
    src = torch.empty(7 * P, dtype=torch.uint8, device="cuda")
    synth.fill_bytes_torch(src, synth.derive(411, synth.TAG_BYTES))
    piece = torch.empty(P, dtype=torch.uint8, device="cuda")
    res = torch.zeros(5, dtype=torch.int32 if width == 32 else torch.int64, device="cuda")
    cs = torch.cuda.current_stream()
    lib = native.load()
    s = native.Stream(keys[width])

    def feed(k, n=P):
        piece[:n].copy_(src[k * P:k * P + n])
        s.update(piece[:n], stream=cs)

    def result(i):
        assert lib.pmp_stream_final(s._h, res[i:i + 1].data_ptr(), None, cs.cuda_stream) == 0

    feed(0)
    feed(1)
    result(0)  # string A = pieces 0, 1
    feed(2)
    result(1)  # string A + piece 2 (a result keeps the state)
    s.reset(stream=cs)
    feed(3)
    result(2)  # string B = piece 3
    feed(4)
    feed(5)
    feed(6, 1000 * 8 + 3)  # an unaligned tail: carried bytes only
    result(3)  # string B + pieces 4, 5 and the tail
    s.reset(stream=cs)
    result(4)  # the empty string
    torch.cuda.synchronize()
    s.close()
    host = src.cpu().numpy()
    want = [host[:2 * P], host[:3 * P], host[3 * P:4 * P],
            np.concatenate([host[3 * P:6 * P], host[6 * P:6 * P + 1000 * 8 + 3]]), host[:0]]
    got = native.as_unsigned(res)
    for i, data in enumerate(want):
        assert int(got[i]) == expect(width, data), i
