"""ctypes wrapper for the plain C oracle (oracle/pmo.c).

TEST INFRASTRUCTURE: only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module. The GPU library never
imports it and shares no code with it.

The oracle computes PM+ hashes (arXiv 1609.09840) from the paper's
definitions: eq. (2wlinear) of Sec. 5, Algorithm 1 of Sec. 4 with the byte
padding of Sec. 4, the output step ``h mod 2^n`` and the mixer of Sec. 7,
using exact multi-limb arithmetic and a generic remainder.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pmo.c")
_LIB = os.path.join(_HERE, "libpmo.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/libpmo.so (plain C99, -O2)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pmo.h"))
    ):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(
            ["gcc", "-std=c99", "-O2", "-Wall", "-fPIC", "-shared", "-o", tmp, _SRC]
        )
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("k", ctypes.c_uint64),
        ("kappa", ctypes.c_uint64),
        ("m", ctypes.c_int),
        ("L", ctypes.c_int),
    ]


class Val(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_uint64)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.POINTER(Params)
        u64p = ctypes.POINTER(ctypes.c_uint64)
        _lib.pmo_key_words.argtypes = [P]
        _lib.pmo_key_words.restype = ctypes.c_size_t
        _lib.pmo_key_expand.argtypes = [P, ctypes.c_uint64, u64p]
        _lib.pmo_splitmix64_at.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        _lib.pmo_splitmix64_at.restype = ctypes.c_uint64
        _lib.pmo_levels.argtypes = [P, ctypes.c_uint64]
        for fn in ("pmo_tree_bytes", "pmo_tree_bytes_streaming"):
            getattr(_lib, fn).argtypes = [P, u64p, ctypes.c_void_p, ctypes.c_uint64,
                                          ctypes.POINTER(Val)]
        _lib.pmo_tree_words.argtypes = [P, u64p, u64p, ctypes.c_uint64, ctypes.POINTER(Val)]
        _lib.pmo_chunk.argtypes = [P, u64p, ctypes.POINTER(Val)]
        _lib.pmo_chunk.restype = Val
        _lib.pmo_output.argtypes = [P, Val]
        _lib.pmo_output.restype = ctypes.c_uint64
        _lib.pmo_mix32.argtypes = [ctypes.c_uint32]
        _lib.pmo_mix32.restype = ctypes.c_uint32
        _lib.pmo_mix64.argtypes = [ctypes.c_uint64]
        _lib.pmo_mix64.restype = ctypes.c_uint64
        _lib.pmo_hash_bytes.argtypes = [P, u64p, ctypes.c_void_p, ctypes.c_uint64, u64p]
        _lib.pmo_hash_batch.argtypes = [P, u64p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_int, u64p]
        _lib.pmo_mod_limbs.argtypes = [P, ctypes.POINTER(ctypes.c_uint32), ctypes.c_int]
        _lib.pmo_mod_limbs.restype = Val
    return _lib


def params(n: int, k: int, kappa: int, m: int, L: int) -> Params:
    return Params(n, k, kappa, m, L)


def pm32() -> Params:
    """PM+32: p = 2^32+15, kappa = 28, m = 128, L = 8 (Table 'parameters')."""
    return Params(32, 15, 28, 128, 8)


def pm64() -> Params:
    """PM+64: p = 2^64+13, kappa = 24, m = 128, L = 8 (Table 'parameters')."""
    return Params(64, 13, 24, 128, 8)


def width_params(width: int) -> Params:
    return {32: pm32, 64: pm64}[width]()


def prime(P: Params) -> int:
    return (1 << P.n) + P.k


def _u64p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _check(rc: int):
    if rc != 0:
        raise ValueError("oracle error code %d" % rc)


def key_expand(P: Params, seed: int) -> np.ndarray:
    key = np.zeros(lib().pmo_key_words(ctypes.byref(P)), dtype=np.uint64)
    _check(lib().pmo_key_expand(ctypes.byref(P), ctypes.c_uint64(seed & (2**64 - 1)), _u64p(key)))
    return key


def splitmix64_at(seed: int, i: int) -> int:
    return int(lib().pmo_splitmix64_at(seed & (2**64 - 1), i))


def levels(P: Params, n0: int) -> int:
    return int(lib().pmo_levels(ctypes.byref(P), n0))


def _as_bytes(data) -> np.ndarray:
    if isinstance(data, (bytes, bytearray)):
        return np.frombuffer(bytes(data), dtype=np.uint8)
    return np.ascontiguousarray(np.asarray(data, dtype=np.uint8))


def tree_bytes(P: Params, key: np.ndarray, data, streaming: bool = False) -> int:
    """Raw tree value h(s) in [0, p) of a byte string (before the output step)."""
    buf = _as_bytes(data)
    out = Val()
    fn = lib().pmo_tree_bytes_streaming if streaming else lib().pmo_tree_bytes
    key = np.ascontiguousarray(key, dtype=np.uint64)
    _check(fn(ctypes.byref(P), _u64p(key), buf.ctypes.data if buf.size else None,
              buf.size, ctypes.byref(out)))
    return int(out.lo) + (int(out.hi) << 64)


def tree_words(P: Params, key: np.ndarray, words) -> int:
    """Algorithm 1 on a word string s_1..s_N (the value 1 is appended)."""
    w = np.ascontiguousarray(np.asarray(words, dtype=np.uint64))
    out = Val()
    key = np.ascontiguousarray(key, dtype=np.uint64)
    _check(lib().pmo_tree_words(ctypes.byref(P), _u64p(key), _u64p(w) if w.size else None,
                                w.size, ctypes.byref(out)))
    return int(out.lo) + (int(out.hi) << 64)


def chunk(P: Params, fkey, s) -> int:
    """f(s) = (b + sum a_i s_i) mod p with fkey = [b, a_1..a_m], s = m values."""
    fk = np.ascontiguousarray(np.asarray(fkey, dtype=np.uint64))
    vals = (Val * P.m)()
    for i, v in enumerate(s):
        vals[i].lo = int(v) & (2**64 - 1)
        vals[i].hi = int(v) >> 64
    r = lib().pmo_chunk(ctypes.byref(P), _u64p(fk), vals)
    return int(r.lo) + (int(r.hi) << 64)


def output(P: Params, h: int) -> int:
    return int(lib().pmo_output(ctypes.byref(P), Val(h & (2**64 - 1), h >> 64)))


def mix32(z: int) -> int:
    return int(lib().pmo_mix32(z))


def mix64(z: int) -> int:
    return int(lib().pmo_mix64(z))


def hash_bytes(P: Params, key: np.ndarray, data) -> int:
    buf = _as_bytes(data)
    out = ctypes.c_uint64()
    key = np.ascontiguousarray(key, dtype=np.uint64)
    _check(lib().pmo_hash_bytes(ctypes.byref(P), _u64p(key), buf.ctypes.data if buf.size else None,
                                buf.size, ctypes.byref(out)))
    return int(out.value)


def hash_batch(P: Params, key: np.ndarray, base: np.ndarray, offsets: np.ndarray,
               raw: bool = False) -> np.ndarray:
    """Hash every string i = base[align8(offsets[i]) : offsets[i+1]]."""
    base = np.ascontiguousarray(base, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    n = offsets.size - 1
    out = np.zeros(2 * n if raw else n, dtype=np.uint64)
    key = np.ascontiguousarray(key, dtype=np.uint64)
    _check(lib().pmo_hash_batch(ctypes.byref(P), _u64p(key), base.ctypes.data if base.size else None,
                                offsets.ctypes.data, n, 1 if raw else 0, _u64p(out)))
    return out


def mod(P: Params, x: int) -> int:
    """Generic remainder x mod p of the oracle (x < 2^256)."""
    limbs = (ctypes.c_uint32 * 8)(*[(x >> (32 * i)) & 0xFFFFFFFF for i in range(8)])
    r = lib().pmo_mod_limbs(ctypes.byref(P), limbs, 8)
    return int(r.lo) + (int(r.hi) << 64)
