"""The seeded input module: host and device generators agree, packing is as documented."""
import numpy as np
import torch

from oracle import pmo
from paper_1609_09840_gb300 import synth


def test_stream_is_splitmix64():
    for seed in (0, 1, 12345, 2 ** 64 - 1):
        xs = synth.u64_np(seed, 0, 5)
        for i in range(5):
            assert int(xs[i]) == pmo.splitmix64_at(seed, i)
        assert synth.mix64((seed + synth.GAMMA) & synth.MASK64) == int(xs[0])


def test_numpy_and_torch_bytes_agree():
    seed = synth.derive(9, synth.TAG_BYTES)
    a = synth.bytes_np(seed, 0, 4096)
    t = torch.empty(4096, dtype=torch.uint8)
    synth.fill_bytes_torch(t, seed, block_words=37)
    assert np.array_equal(a, t.numpy())
    # arbitrary windows of the same stream
    for start, n in ((3, 10), (8, 1), (1000, 333), (4095, 1)):
        assert np.array_equal(synth.bytes_np(seed, start, n), a[start:start + n])


def test_packing_convention():
    lengths = np.array([0, 1, 7, 8, 9, 16, 3], dtype=np.int64)
    off = synth.pack_offsets(lengths)
    starts = synth.align8(off[:-1])
    assert (starts % 8 == 0).all()
    assert np.array_equal(off[1:] - starts, lengths)
    assert (starts[1:] >= off[1:-1]).all()


def test_batch_host_device_bytes_agree_with_special_strings():
    b = synth.workload_c4(n=3000, seed=4, long_lo=5000, long_hi=9000)
    assert (b.kind == synth.KIND_ZERO).any() and (b.kind == synth.KIND_REPEAT).any()
    host = b.host_bytes()
    dev = b.device_bytes("cpu").numpy()
    assert np.array_equal(host, dev)
    for i in range(0, b.n, 97):
        s, e = int(b.starts[i]), int(b.offsets[i + 1])
        assert np.array_equal(b.string_bytes(i), host[s:e])


def test_workload_shapes():
    c1 = synth.workload_c1()
    assert c1.n == 10_000 and c1.lengths.min() >= 1 and c1.lengths.max() <= 256
    c3 = synth.workload_c3(n=200_000)
    med = np.median(c3.lengths)
    assert 20 <= med <= 28 and c3.lengths.min() >= 1 and c3.lengths.max() <= 65536
    c4 = synth.workload_c4(n=100_000)
    frac_long = (c4.lengths > 64).mean()
    assert 0.005 < frac_long < 0.015
    reqs = synth.serving_requests(20, rate_per_s=100.0)
    assert all(1 <= r.batch.n <= 100_000 for r in reqs)
    assert sorted(r.arrival_s for r in reqs) == [r.arrival_s for r in reqs]
