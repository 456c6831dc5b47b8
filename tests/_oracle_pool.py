"""Oracle workers for the full-size parity tests: each regenerates its strings
from the seeded workload recipe (paper_1609_09840_gb300.synth) and hashes
them with the CPU oracle, so that a pool of spawned processes covers a whole
configuration in seconds. Test infrastructure: nothing here runs on a GPU.
"""
import multiprocessing as mp
import os

import numpy as np


def pool():
    """A process pool over every host core (spawned: safe next to CUDA)."""
    return mp.get_context("spawn").Pool(os.cpu_count() or 1)


def cuts(n, parts):
    return [n * i // parts for i in range(parts + 1)]


def _hash_span(width, key_seed, buf, offs):
    from oracle import pmo

    P = pmo.width_params(width)
    return pmo.hash_batch(P, pmo.key_expand(P, key_seed), buf, offs)


def c3_part(task):
    """Oracle hashes of strings [a, b) of the 4M-string log-normal batch."""
    a, b, width, n = task
    from paper_1609_09840_gb300 import synth

    lengths = synth.lognormal_lengths(3, n)[:b]
    offs = synth.pack_offsets(lengths)
    s0 = int(offs[a]) & ~7
    sub = np.ascontiguousarray(offs[a:] - s0)
    buf = synth.bytes_np(synth.derive(3, synth.TAG_BYTES), s0, (int(sub[-1]) + 31) // 16 * 16)
    return a, _hash_span(width, 3, buf, sub)


def c4_short_part(task):
    """Oracle hashes of the short strings (at most 64 bytes) among strings
    [a, b) of the skewed mix, PM+64: each run of consecutive short strings
    is regenerated as one byte span (content kinds applied) and hashed as a
    sub-batch."""
    a, b = task
    from paper_1609_09840_gb300 import synth

    batch = synth.workload_c4()
    short = batch.lengths <= 64
    starts = batch.starts
    idx, vals = [], []
    i = a
    while i < b:
        if not short[i]:
            i += 1
            continue
        j = i
        while j < b and short[j]:
            j += 1
        s0 = int(starts[i])
        sub = np.ascontiguousarray(batch.offsets[i:j + 1] - s0)
        sub[0] = 0
        buf = synth.bytes_np(synth.derive(4, synth.TAG_BYTES), s0, (int(sub[-1]) + 31) // 16 * 16)
        for q in range(i, j):
            if batch.kind[q] != synth.KIND_RANDOM:
                lo, hi = int(starts[q]) - s0, int(batch.offsets[q + 1]) - s0
                buf[lo:hi] = 0 if batch.kind[q] == synth.KIND_ZERO else batch.fill[q]
        idx.append(np.arange(i, j))
        vals.append(_hash_span(64, 4, buf, sub))
        i = j
    if not idx:
        return np.zeros(0, np.int64), np.zeros(0, np.uint64)
    return np.concatenate(idx), np.concatenate(vals)


def c4_string(i):
    """Oracle hash of string i of the skewed mix (PM+64)."""
    from oracle import pmo
    from paper_1609_09840_gb300 import synth

    batch = synth.workload_c4()
    P = pmo.pm64()
    return i, pmo.hash_bytes(P, pmo.key_expand(P, 4), batch.string_bytes(i))


def c5_request(r):
    """Oracle hashes of request r of the serving pool (48 requests, seed 5)."""
    from paper_1609_09840_gb300 import synth

    req = synth.serving_requests(48, rate_per_s=1.0, seed=5)[r]
    return r, _hash_span(req.width, 5, req.batch.host_bytes(), req.batch.offsets)
