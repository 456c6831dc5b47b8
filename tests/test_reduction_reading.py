"""The reading of Sec. 6.2 and Algorithm 2 used by the device reduction.

The printed listing of Algorithm 2 names its inputs (v1, v2) but uses (v0, v1)
and ends with "return v0 - k". The library reads it as: with input v0 + 2^n v1
(v1 <= 2), return v0 - k v1 if k v1 <= v0; else v0 + 2^n if v1 == 1; else
v0 + 2^n - k (since 2 * 2^n == 2^n - k mod p). This test restates that reading
in Python and checks it against '%' on every branch boundary, and checks the
two-word bound v1 <= 2 of Sec. 6.2 at the extreme three-word sums.
"""
import random

import pytest


def reduce_reading(n, k, S):
    w0 = S & ((1 << n) - 1)
    w1 = (S >> n) & ((1 << n) - 1)
    w2 = S >> (2 * n)
    u = k * w1
    u0, u1 = u & ((1 << n) - 1), u >> n
    T = (w0 + k * k * w2 + k * u1) + ((1 << n) + k - u0)
    v0, v1 = T & ((1 << n) - 1), T >> n
    assert v1 <= 2
    if k * v1 <= v0:
        return v0 - k * v1
    if v1 == 1:
        return v0 + (1 << n)
    return v0 + (1 << n) - k


@pytest.mark.parametrize("n,k", [(32, 15), (64, 13)])
def test_reading_matches_mod_on_branch_boundaries(n, k):
    p = (1 << n) + k
    m = 128
    smax = ((1 << n) - 1) + m * ((1 << (2 * n)) - 1)
    cases = set()
    for v1 in range(3):
        for v0 in list(range(0, 3 * k + 2)) + [(1 << n) - d for d in range(1, 4)]:
            cases.add(v0 + (v1 << n))
    rng = random.Random(n)
    for _ in range(20000):
        cases.add(rng.randrange(smax + 1))
    for w2 in (0, 1, m - 1, m):
        for w1 in (0, 1, (1 << n) - 1):
            for w0 in (0, k, (1 << n) - 1):
                S = w0 + (w1 << n) + (w2 << (2 * n))
                if S <= smax:
                    cases.add(S)
    cases.add(smax)
    for S in cases:
        z = reduce_reading(n, k, S)
        assert 0 <= z < p
        assert z == S % p
