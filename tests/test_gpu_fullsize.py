"""Parity at full size: the 4M-string batched case and the ~174 GiB skewed mix,
hashed on the device in the configuration the benchmark times, with a seeded
sample of outputs recomputed one by one by the oracle from host-generated
bytes of the same strings (integer hashing: bit-exact)."""
import numpy as np
import pytest
import torch

from oracle import pmo
from paper_1609_09840_gb300 import synth

pytestmark = pytest.mark.gpu


def sample_indices(n, count, seed, must=()):
    rng = np.random.default_rng(seed)
    idx = set(int(x) for x in rng.choice(n, size=min(count, n), replace=False))
    idx.update(int(x) for x in must)
    return sorted(idx)


@pytest.mark.parametrize("width", (32, 64))
def test_batched_4m_strings_sampled(native, width):
    batch = synth.workload_c3()
    base = batch.device_bytes("cuda")
    offs = torch.from_numpy(batch.offsets).cuda()
    key = native.Key(seed=3, width=width)
    out = native.as_unsigned(native.hash_batch(key, base, offs)).astype(np.uint64)
    P = pmo.width_params(width)
    okey = pmo.key_expand(P, 3)
    longest = np.argsort(batch.lengths)[-50:]  # the multi-chunk strings
    for i in sample_indices(batch.n, 5000, seed=width, must=longest):
        assert int(out[i]) == pmo.hash_bytes(P, okey, batch.string_bytes(i)), i
    key.close()
    del base
    torch.cuda.empty_cache()


def test_skewed_mix_full_size_sampled(native):
    batch = synth.workload_c4()
    need = batch.buffer_bytes + 64 * batch.n
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < need + (4 << 30):
        pytest.skip("needs %.0f GiB of free device memory" % (need / 2 ** 30))
    base = batch.device_bytes("cuda")
    offs = torch.from_numpy(batch.offsets).cuda()
    key = native.Key(seed=4, width=64)
    out = native.as_unsigned(native.hash_batch(key, base, offs)).astype(np.uint64)
    assert native.device_status() == 0
    del base
    torch.cuda.empty_cache()
    P = pmo.pm64()
    okey = pmo.key_expand(P, 4)
    long_idx = np.nonzero(batch.lengths > 64)[0]
    rng = np.random.default_rng(44)
    picks = [int(x) for x in rng.choice(long_idx, size=12, replace=False)]
    for kind in (synth.KIND_ZERO, synth.KIND_REPEAT):  # long strings of every content kind
        cand = long_idx[batch.kind[long_idx] == kind]
        picks += [int(x) for x in cand[:2]]
    for i in sample_indices(batch.n, 3000, seed=4, must=picks):
        assert int(out[i]) == pmo.hash_bytes(P, okey, batch.string_bytes(i)), i
    key.close()
