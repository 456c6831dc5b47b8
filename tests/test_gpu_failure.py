"""Failure detection on the device without a fault.

Every wait of the TMA pipelines is bounded in wall time: a wait that runs out
records PMP_ETIMEOUT in the device status word, raises the block's abort flag
and lets the kernel return. Here a wait is made to run out on purpose (an
mbarrier phase that nothing completes), the status is read on the host, and
the context is shown to be still usable: a hash after it equals the oracle's.
"""
import time

import numpy as np
import pytest
import torch

from oracle import pmo
from paper_1609_09840_gb300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_reports_and_the_context_survives(native):
    assert native.device_status() == 0
    t0 = time.perf_counter()
    ok = native.debug_wait_timeout()
    dt = time.perf_counter() - t0
    assert ok == 0                      # the wait reported failure
    assert 1.5 < dt < 60                # after its limit (2 s), not at once, not never
    assert native.device_status() == native.PMP_ETIMEOUT
    assert native.device_status() == 0  # reading clears it
    data = np.asarray(synth.bytes_np(synth.derive(9, synth.TAG_BYTES), 0, 4096), dtype=np.uint8)
    for width in (32, 64):
        key = native.Key(seed=9, width=width)
        got = native.hash(key, torch.from_numpy(data).cuda())
        torch.cuda.synchronize()
        want = pmo.hash_bytes(pmo.width_params(width), pmo.key_expand(pmo.width_params(width), 9), data)
        assert int(native.as_unsigned(got.cpu())[0]) == want
        key.close()
    assert native.device_status() == 0
