"""The serving loop (continuous batching): every result is the same when the
request runs alone through the batched API and when it runs mixed with other
requests in the server, and equals the oracle (integer hashing: bit-exact);
requests are in flight together (their admission-to-completion spans
overlap), not served one after another."""
import numpy as np
import pytest
import torch

from oracle import pmo
from paper_1609_09840_gb300 import synth

pytestmark = pytest.mark.gpu


def make_requests(count, seed=55, max_strings=3000):
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(count):
        n = int(rng.integers(1, max_strings))
        width = 32 if r % 2 == 0 else 64
        batch = synth.Batch("req%d" % r, seed * 1000 + r, synth.lognormal_lengths(seed * 1000 + r, n))
        host = torch.from_numpy(batch.host_bytes()).pin_memory()
        offs = torch.from_numpy(batch.offsets).pin_memory()
        out = torch.zeros(n, dtype=torch.int32 if width == 32 else torch.int64).pin_memory()
        reqs.append((width, batch, host, offs, out))
    return reqs


def test_server_results_alone_and_in_the_mix(native):
    k32, k64 = native.Key(seed=5, width=32), native.Key(seed=5, width=64)
    keys = {32: k32, 64: k64}
    reqs = make_requests(24)
    # a budget that holds only a few requests at a time, so admission waits
    server = native.Server(k32, k64, budget_bytes=2 << 20, slots=3)
    tickets = [server.submit(w, host, offs, out) for (w, _, host, offs, out) in reqs]
    for t in tickets:
        assert server.wait(t, timeout_s=60.0)
    spans = []
    for t, (w, batch, host, offs, out) in zip(tickets, reqs):
        mixed = native.as_unsigned(out).astype(np.uint64)
        alone = native.as_unsigned(native.hash_batch(keys[w], host.cuda(), offs.cuda())).astype(np.uint64)
        assert np.array_equal(mixed, alone)
        want = pmo.hash_batch(pmo.width_params(w), pmo.key_expand(pmo.width_params(w), 5),
                              batch.host_bytes(), batch.offsets)
        assert np.array_equal(mixed, want)
        sub, adm, done = server.times(t)
        assert sub <= adm <= done
        spans.append((adm, done))
        server.release(t)
    server.close()
    assert native.device_status() == 0
    # continuous batching, not a queue: requests were in flight on the device
    # together (admitted before another one had completed)
    together = sum(1 for i, a in enumerate(spans) for b in spans[i + 1:] if a[0] < b[1] and b[0] < a[1])
    assert together > 0


def test_server_refuses_a_request_larger_than_its_budget(native):
    k32, k64 = native.Key(seed=5, width=32), native.Key(seed=5, width=64)
    server = native.Server(k32, k64, budget_bytes=64 << 10, slots=2)
    batch = synth.Batch("big", 9, np.full(2000, 100, dtype=np.int64))
    host = batch.host_bytes()
    out = np.zeros(batch.n, dtype=np.uint64)
    with pytest.raises(native.PmpError) as e:
        server.submit(64, host, batch.offsets, out)
    assert e.value.code == native.PMP_ENOMEM
    server.close()
