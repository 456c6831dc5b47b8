"""pmp_hash64_noalloc: the PM+64 single-buffer hash for callers that may not
allocate device memory (for example code running under a host allocator that
owns all device memory, or a latency-critical path that cannot take the
device-wide synchronisation of cudaMalloc). It uses the library's fixed 1 MiB
per-device scratch array instead of caller scratch.

The test calls it through the C ABI twice in a row on different inputs, so
the second call runs on the scratch the first one left behind, and compares
each result with the existing pmp_hash64 entry point (integer hashing: the
results must be equal bit for bit). It also checks that an input too long
for the fixed array is refused with PMP_ESCRATCH before anything runs.
This file is collected last on purpose.
"""
import ctypes

import pytest
import torch

from paper_1609_09840_gb300 import synth

pytestmark = pytest.mark.gpu


def test_noalloc_matches_hash64_twice_in_a_row(native):
    key = native.Key(seed=2, width=64)
    lib = native.load()
    data = torch.empty(96 << 20, dtype=torch.uint8, device="cuda")
    synth.fill_bytes_torch(data, synth.derive(55, synth.TAG_BYTES))
    # 3-level and 2-level inputs: both use the scratch (level values, counters)
    for length in ((96 << 20) - 40, (5 << 20) + 24, (96 << 20) - 40):
        want = native.as_unsigned(native.hash(key, data[:length]))[0]
        for _ in range(2):
            out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
            rc = lib.pmp_hash64_noalloc(key.handle, ctypes.c_void_p(data.data_ptr()), length,
                                        ctypes.c_void_p(out.data_ptr()),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert rc == native.PMP_OK
            assert native.as_unsigned(out)[0] == want
    assert native.device_status() == 0
    key.close()


def test_noalloc_refuses_inputs_beyond_its_scratch(native):
    key = native.Key(seed=2, width=64)
    lib = native.load()
    limit = native.hash_noalloc_max_len()
    assert limit >= 4 << 30  # at least 4 GiB fit in the fixed array
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    small = torch.zeros(16, dtype=torch.uint8, device="cuda")
    # refused on the host before any launch: the buffer is never read
    rc = lib.pmp_hash64_noalloc(key.handle, ctypes.c_void_p(small.data_ptr()), limit + 1,
                                ctypes.c_void_p(out.data_ptr()), None)
    assert rc == native.PMP_ESCRATCH
    assert b"no-allocation" in lib.pmp_strerror(rc)
    key.close()
