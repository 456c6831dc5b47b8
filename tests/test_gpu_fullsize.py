"""Parity at full size, element by element: the 4M-string batched case (every
output, both widths, every batch schedule), the ~174 GiB skewed mix (every
short string, and long strings of each content kind), and the serving
case's pool of 48 seeded requests run through the server (every output of
every request). The oracle's values come from a pool of host processes
(tests/_oracle_pool.py) that regenerate the same seeded strings; integer
hashing: the bar is bit-exact equality."""
import numpy as np
import pytest
import torch

import _oracle_pool as op
from paper_1609_09840_gb300 import synth

pytestmark = pytest.mark.gpu

SCHEDULES = (("sorted", 512), ("sorted", 1024), ("tiles", 6), ("tiles", 8))


@pytest.fixture(scope="module")
def procs():
    with op.pool() as p:
        yield p


@pytest.fixture(scope="module")
def c3_oracle(procs):
    n = 4 * 1024 * 1024
    c = op.cuts(n, 64)
    res = {}
    for w in (32, 64):
        out = np.zeros(n, dtype=np.uint64)
        for a, vals in procs.map(op.c3_part, [(c[i], c[i + 1], w, n) for i in range(64)], chunksize=1):
            out[a:a + vals.size] = vals
        res[w] = out
    return res


def set_schedule(native, sched, v):
    if sched == "sorted":
        native.tune_set(native.KNOB_BATCH_SCHED, native.BATCH_SORTED)
        native.tune_set(native.KNOB_BATCH_RANGE, v)
    else:
        native.tune_set(native.KNOB_BATCH_SCHED, native.BATCH_TILES)
        native.tune_set(native.KNOB_BATCH_P1, v)


def test_batched_4m_strings_every_output(native, c3_oracle):
    batch = synth.workload_c3()
    base = batch.device_bytes("cuda")
    offs = torch.from_numpy(batch.offsets).cuda()
    knobs = (native.KNOB_BATCH_SCHED, native.KNOB_BATCH_RANGE, native.KNOB_BATCH_P1)
    old = [native.tune_get(k) for k in knobs]
    try:
        for width in (32, 64):
            key = native.Key(seed=3, width=width)
            for sched, v in SCHEDULES:
                set_schedule(native, sched, v)
                out = native.as_unsigned(native.hash_batch(key, base, offs)).astype(np.uint64)
                bad = np.nonzero(out != c3_oracle[width])[0]
                assert bad.size == 0, (width, sched, v, bad[:10])
            key.close()
    finally:
        for k, o in zip(knobs, old):
            native.tune_set(k, o)
    assert native.device_status() == 0
    del base
    torch.cuda.empty_cache()


def test_skewed_mix_full_size(native, procs):
    """Every one of the ~2.08M short strings, the longest string, and eight
    long strings of each content kind (random, all-zero, repeated byte)."""
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
    key.close()
    del base
    torch.cuda.empty_cache()
    c = op.cuts(batch.n, 64)
    checked = 0
    for idx, vals in procs.map(op.c4_short_part, [(c[i], c[i + 1]) for i in range(64)], chunksize=1):
        bad = np.nonzero(out[idx] != vals)[0]
        assert bad.size == 0, idx[bad[:10]]
        checked += idx.size
    assert checked == int((batch.lengths <= 64).sum())
    long_idx = np.nonzero(batch.lengths > 64)[0]
    picks = [int(long_idx[np.argmax(batch.lengths[long_idx])])]
    for kind in (synth.KIND_RANDOM, synth.KIND_ZERO, synth.KIND_REPEAT):
        picks += [int(x) for x in long_idx[batch.kind[long_idx] == kind][:8]]
    for i, want in procs.map(op.c4_string, picks, chunksize=1):
        assert int(out[i]) == want, i


def test_serving_pool_every_request(native, procs):
    """The benchmark's pool of 48 seeded requests (1..100,000 strings each,
    log-normal lengths, PM+32 or PM+64) submitted together to a server with
    the benchmark's budget and slots: every output of every request equals
    the oracle's."""
    reqs = synth.serving_requests(48, rate_per_s=1.0, seed=5)
    k32, k64 = native.Key(seed=5, width=32), native.Key(seed=5, width=64)
    server = native.Server(k32, k64, budget_bytes=16 << 30, slots=4)
    bufs, tickets = [], []
    for r in reqs:
        host = torch.from_numpy(r.batch.host_bytes()).pin_memory()
        offs = torch.from_numpy(r.batch.offsets).pin_memory()
        out = torch.zeros(r.batch.n, dtype=torch.int32 if r.width == 32 else torch.int64).pin_memory()
        bufs.append(out)
        tickets.append(server.submit(r.width, host, offs, out))
    for t in tickets:
        done, rc = server.wait_status(t, 120.0)
        assert done and rc == native.PMP_OK
    for r, want in procs.map(op.c5_request, range(len(reqs)), chunksize=1):
        got = native.as_unsigned(bufs[r]).astype(np.uint64)
        assert np.array_equal(got, want), r
    for t in tickets:
        server.release(t)
    server.close()
    assert native.device_status() == 0
