"""Exhaustive device checks of the 32-bit arithmetic.

Sec. 6.2 and Algorithm 2 (n = 32) and the 32-bit mixer of Sec. 7 take 32-bit
inputs, so the device code is checked on every input rather than on samples:
- Algorithm 2 as read for this library (v0 - k v1 if k v1 <= v0, else
  v0 + 2^n if v1 = 1, else v0 + 2^n - k) on all 3 * 2^32 inputs
  v0 + 2^32 v1, v1 <= 2, against the integer remainder;
- the whole reduction of three-word sums S = r0 + 2^32 r1 + 2^64 r2 for every
  r0 and (r1, r2) pairs at the carry and branch boundaries (r2 up to m = 128,
  the bound of Sec. 6.2), against the integer remainder;
- the mixer followed by its inverse (the inverse of the odd multiplier mod
  2^32 computed here by Python) on all 2^32 inputs: a bijection, as Sec. 7
  requires so that regularity and universality carry over.
"""
import json
import os

import pytest

pytestmark = pytest.mark.gpu

with open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")) as _f:
    MIX32 = json.load(_f)["mixer"]["pm32"]  # Sec. 7: shifts and multiplier of the 32-bit mixer


def test_algorithm2_every_input(native):
    assert native.check_alg2_32() == 0


def test_reduction_every_low_word(native):
    k = 15
    r1s = [0, 1, k - 1, k, k + 1, (1 << 31) - 1, 1 << 31, 0x9E3779B9, (1 << 32) - k - 1, (1 << 32) - 1]
    pairs = [(r1, r2) for r1 in r1s for r2 in (0, 1, 128)]
    for i in range(0, len(pairs), 32):
        assert native.check_reduce32(pairs[i:i + 32]) == 0


def test_mixer_round_trip_every_input(native):
    assert (MIX32["s1"], MIX32["s2"]) == (13, 16)  # the inverse shifts in the kernel
    a = int(MIX32["mult"], 16)
    a_inv = pow(a, -1, 1 << 32)
    assert (a * a_inv) % (1 << 32) == 1
    assert native.check_mix32(a_inv) == 0
    # a wrong inverse must be caught (the check is not vacuous)
    assert native.check_mix32(a_inv ^ 2) > 0


def test_check_arguments(native):
    with pytest.raises(native.PmpError):
        native.check_reduce32([(0, 129)])
    with pytest.raises(native.PmpError):
        native.check_reduce32([(0, 0)] * 33)
