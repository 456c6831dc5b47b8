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


def test_server_string_in_pieces_across_requests(native):
    """Two strings (PM+32 and PM+64) held by the server are appended to piece
    by piece in separate requests, interleaved with batch requests on the
    same slots; their partial tree state stays on the device between
    requests (Sec. 4's bounded-memory order). A result asked for half way is
    the hash of the prefix, and the string continues after it; the final
    results equal the oracle's hash of the whole byte strings."""
    k32, k64 = native.Key(seed=6, width=32), native.Key(seed=6, width=64)
    server = native.Server(k32, k64, budget_bytes=64 << 20, slots=3)
    data = synth.bytes_np(synth.derive(66, synth.TAG_BYTES), 0, 3_000_000 + 77)
    cuts = [0, 1, 7, 8, 513, 4096, 4099, 70_000, 1_000_003, 1_500_000, 2_999_999, len(data)]
    sids = {w: server.stream_open(w) for w in (32, 64)}
    batches = make_requests(10, seed=66, max_strings=2000)
    outs, tickets, mids = {}, [], {}
    for i in range(len(cuts) - 1):
        piece = torch.from_numpy(data[cuts[i]:cuts[i + 1]].copy()).pin_memory()
        for w in (32, 64):
            final = i == len(cuts) - 2 or i == 5
            out = torch.zeros(1, dtype=torch.int32 if w == 32 else torch.int64).pin_memory() if final else None
            t = server.submit_piece(sids[w], piece, final=final, out=out)
            tickets.append(t)
            if final:
                (outs if i == len(cuts) - 2 else mids)[w] = (t, out)
        if i < len(batches):
            w, batch, host, offs, out = batches[i]
            tickets.append(server.submit(w, host, offs, out))
    for t in tickets:
        assert server.wait(t, timeout_s=60.0)
    for w in (32, 64):
        P = pmo.width_params(w)
        okey = pmo.key_expand(P, 6)
        got = int(native.as_unsigned(outs[w][1])[0])
        assert got == pmo.hash_bytes(P, okey, data), w
        mid = int(native.as_unsigned(mids[w][1])[0])
        assert mid == pmo.hash_bytes(P, okey, data[:cuts[6]]), w
        server.stream_close(sids[w])
    for (w, batch, host, offs, out) in batches:
        want = pmo.hash_batch(pmo.width_params(w), pmo.key_expand(pmo.width_params(w), 6),
                              batch.host_bytes(), batch.offsets)
        assert np.array_equal(native.as_unsigned(out).astype(np.uint64), want)
    for t in tickets:
        server.release(t)
    with pytest.raises(native.PmpError) as e:
        server.submit_piece(sids[32], torch.zeros(4, dtype=torch.uint8))
    assert e.value.code == native.PMP_EINVAL  # a closed string
    server.close()
    assert native.device_status() == 0


def test_server_wait_rejects_bad_timeouts(native):
    k32, k64 = native.Key(seed=5, width=32), native.Key(seed=5, width=64)
    server = native.Server(k32, k64, budget_bytes=1 << 20, slots=1)
    batch = synth.Batch("t", 3, np.array([5, 17, 40]))
    host = torch.from_numpy(batch.host_bytes()).pin_memory()
    offs = torch.from_numpy(batch.offsets).pin_memory()
    out = torch.zeros(batch.n, dtype=torch.int32).pin_memory()
    t = server.submit(32, host, offs, out)
    for bad in (-1.0, float("nan")):
        done, rc = server.wait_status(t, bad)
        assert rc == native.PMP_EINVAL
    done, rc = server.wait_status(t, 1e30)  # taken as 1e9 s: returns when done
    assert done and rc == native.PMP_OK
    server.release(t)
    server.close()


def test_batch_status_word_names_the_failing_call(native):
    """Two batch calls in flight on two streams, one given far too little
    scratch for its 16 MiB string: only that call's status word reports
    PMP_ESCRATCH (the serving loop reports it on the request's own ticket);
    the other call's word stays 0 and its hashes equal the oracle's."""
    lib = native.load()
    k = native.Key(seed=8, width=64)
    good = synth.Batch("good", 81, synth.lognormal_lengths(81, 5000))
    bad = synth.Batch("bad", 82, np.array([5, 40, (16 << 20) + 24, 63]))
    status = torch.zeros(2, dtype=torch.int32, device="cuda")
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    assert native.device_status() == 0
    for idx, (b, data_bytes) in enumerate(((good, good.buffer_bytes), (bad, 64))):
        base = torch.from_numpy(b.host_bytes()).cuda()
        offs = torch.from_numpy(b.offsets).cuda()
        out = torch.zeros(b.n, dtype=torch.int64, device="cuda")
        scr = torch.empty(native.batch_scratch_bytes(64, b.n, data_bytes), dtype=torch.uint8, device="cuda")
        torch.cuda.synchronize()
        rc = lib.pmp_hash_batch_status(k.handle, base.data_ptr(), offs.data_ptr(), b.n, out.data_ptr(),
                                       status.data_ptr() + 4 * idx, scr.data_ptr(), scr.numel(),
                                       streams[idx].cuda_stream)
        assert rc == native.PMP_OK
        outs.append((b, base, offs, out, scr))
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0, native.PMP_ESCRATCH]
    assert native.device_status() == native.PMP_ESCRATCH  # the device-wide word too (read and cleared)
    b, base, offs, out, _ = outs[0]
    want = pmo.hash_batch(pmo.width_params(64), pmo.key_expand(pmo.width_params(64), 8), b.host_bytes(), b.offsets)
    assert np.array_equal(native.as_unsigned(out).astype(np.uint64), want)
