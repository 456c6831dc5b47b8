"""Host logic of the C ABI that needs no device: the single-buffer plan
against the level structure of Algorithm 1 (level counts from the oracle),
the batch scratch sizes, the tuning knobs, the no-allocation bound and the
status strings."""
import ctypes

import pytest

from oracle import pmo

M = 128
LMAX = 8


@pytest.fixture(scope="module")
def lib():
    from paper_1609_09840_gb300 import build

    lib = ctypes.CDLL(build.build())
    lib.pmp_hash_scratch_bytes.restype = ctypes.c_size_t
    lib.pmp_hash_scratch_bytes.argtypes = [ctypes.c_int, ctypes.c_uint64]
    lib.pmp_batch_scratch_bytes.restype = ctypes.c_size_t
    lib.pmp_batch_scratch_bytes.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_uint64]
    lib.pmp_hash_noalloc_max_len.restype = ctypes.c_uint64
    lib.pmp_strerror.restype = ctypes.c_char_p
    lib.pmp_tune_get.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    return lib


def level_sizes(n0):
    """Chunks per level of Algorithm 1 (at least one level)."""
    c = [n0]
    while True:
        c.append((c[-1] + M - 1) // M)
        if c[-1] <= 1:
            return c


def lengths(width):
    W = width // 8
    out = {0, 1, W - 1, W, M * W - 1, M * W, M * W + 1}
    for lv in range(1, 6):
        edge = M ** lv  # N0 = m^lv words fit lv levels, one more word needs another
        out.update({(edge - 1) * W, (edge - 1) * W + W - 1, edge * W})
    out.update({123456789, 1 << 30, (1 << 30) + 5, 3 << 33})
    return sorted(out)


@pytest.mark.parametrize("width", [32, 64])
def test_single_buffer_plan_follows_the_levels(lib, width):
    """Scratch holds the values of levels 2 .. L-1 (16 bytes each) and an
    arrival counter per chunk of levels 3 .. L (4 bytes), plus an 8-byte
    tile counter when level 2 has more than one chunk: zero for L <= 2."""
    P = pmo.width_params(width)
    W = width // 8
    for length in lengths(width):
        n0 = length // W + 1
        c = level_sizes(n0)
        L = len(c) - 1
        assert L == pmo.levels(P, n0), length
        got = lib.pmp_hash_scratch_bytes(width, length)
        if L <= 2:
            assert got == 0, length
            continue
        vals = 16 * sum(c[j] for j in range(2, L))
        ctrs = 4 * sum(c[j] for j in range(3, L + 1)) + (8 if c[2] > 1 else 0)
        assert vals + ctrs <= got <= vals + 255 + ctrs, (length, got, vals, ctrs)


@pytest.mark.parametrize("width", [32, 64])
def test_plan_refuses_a_ninth_level(lib, width):
    W = width // 8
    longest = (M ** LMAX - 1) * W + W - 1  # N0 = m^8 words: eight levels
    assert lib.pmp_hash_scratch_bytes(width, longest) > 0
    assert lib.pmp_hash_scratch_bytes(width, longest + 1) == 0  # the plan fails: nine levels


@pytest.mark.parametrize("width", [32, 64])
def test_batch_scratch_grows_with_the_data(lib, width):
    sizes = [lib.pmp_batch_scratch_bytes(width, 1000, d) for d in (0, 1 << 20, 1 << 30, 1 << 36)]
    assert sizes[0] >= 256  # the counter header
    assert sizes == sorted(sizes) and sizes[-1] > sizes[0]
    assert lib.pmp_batch_scratch_bytes(width, -1, 1 << 20) == 0
    assert lib.pmp_batch_scratch_bytes(48, 10, 1 << 20) == 0


def test_tuning_knobs_without_a_device(lib):
    v = ctypes.c_int()
    for knob, allowed in ((0, (2, 3, 4, 6)), (1, (2, 3, 4, 6)), (2, (6, 8))):
        assert lib.pmp_tune_get(knob, ctypes.byref(v)) == 0
        old = v.value
        assert old in allowed
        assert lib.pmp_tune_set(knob, 5) == 1  # PMP_EINVAL
        for a in allowed:
            assert lib.pmp_tune_set(knob, a) == 0
            assert lib.pmp_tune_get(knob, ctypes.byref(v)) == 0 and v.value == a
        assert lib.pmp_tune_set(knob, old) == 0
    assert lib.pmp_tune_set(99, 4) == 1


def test_noalloc_bound_and_status_strings(lib):
    n = lib.pmp_hash_noalloc_max_len()
    assert n >= 1 << 32
    texts = [lib.pmp_strerror(c) for c in range(8)]
    assert texts[0] == b"ok" and all(texts) and len(set(texts)) == 8
    assert lib.pmp_strerror(99)
