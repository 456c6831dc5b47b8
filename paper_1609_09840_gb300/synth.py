"""Seeded synthetic inputs for PM+ hashing workloads.

This module is the ONE piece shared by the CUDA path's tests and benchmarks
and the CPU oracle's tests: it only produces input bytes, string lengths and
offsets. It contains none of the hashing arithmetic.

Every random quantity comes from the counter-based splitmix64 stream
(Steele, Lea, Flood 2014): output i of the stream with seed s is
mix64(s + (i + 1) * 0x9e3779b97f4a7c15). Being counter based, any byte of a
buffer can be produced independently on the host (numpy) or on the device
(torch integer ops), with identical results.

Derived streams: each purpose (bytes, lengths, ...) of a workload seed uses
its own stream seed ``derive(seed, tag)``.

Packing convention of the batched API: string i occupies bytes
[align8(offsets[i]), offsets[i+1]) of one buffer; offsets is int64[n+1].
Buffers are padded so that every 8-byte word that holds string bytes is
inside the allocation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

MASK64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB

TAG_BYTES = 0x42
TAG_LENGTHS = 0x4C
TAG_KIND = 0x4B
TAG_FILL = 0x46
TAG_ARRIVALS = 0x41
TAG_REQUESTS = 0x52

KIND_RANDOM, KIND_ZERO, KIND_REPEAT = 0, 1, 2


def mix64(z: int) -> int:
    z &= MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def derive(seed: int, tag: int) -> int:
    """Seed of the stream used for one purpose of one workload seed."""
    return mix64((seed & MASK64) ^ ((tag * 0xD1B54A32D192ED03) & MASK64))


# --------------------------------------------------------------------------
# numpy (host) generators
# --------------------------------------------------------------------------
def u64_np(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the splitmix64 stream `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & MASK64) + i * np.uint64(GAMMA)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
        return z ^ (z >> np.uint64(31))


def bytes_np(seed: int, start: int, nbytes: int) -> np.ndarray:
    """Bytes start .. start+nbytes-1 of the byte stream: byte q is byte q%8
    (little-endian) of stream output q//8."""
    if nbytes <= 0:
        return np.zeros(0, dtype=np.uint8)
    w0 = start // 8
    w1 = (start + nbytes + 7) // 8
    words = u64_np(seed, w0, w1 - w0).astype("<u8")
    b = words.view(np.uint8)
    off = start - 8 * w0
    return b[off:off + nbytes].copy()


def uniform01_np(seed: int, start: int, count: int) -> np.ndarray:
    """Doubles in (0, 1] from the top 53 bits of each draw."""
    x = u64_np(seed, start, count) >> np.uint64(11)
    return (x.astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


# --------------------------------------------------------------------------
# torch (host or device) generator of the same byte stream
# --------------------------------------------------------------------------
def _signed(c: int) -> int:
    c &= MASK64
    return c - (1 << 64) if c >= 1 << 63 else c


def _srl(x, s: int):
    """Logical right shift of an int64 tensor holding 64-bit patterns."""
    return (x >> s) & ((1 << (64 - s)) - 1)


def u64_torch(seed: int, start: int, count: int, device):
    """Same values as u64_np, as int64 bit patterns, computed on `device`."""
    import torch

    i = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = i * _signed(GAMMA) + _signed(seed)
    z = (z ^ _srl(z, 30)) * _signed(MIX1)
    z = (z ^ _srl(z, 27)) * _signed(MIX2)
    return z ^ _srl(z, 31)


def fill_bytes_torch(out, seed: int, start: int = 0, block_words: int = 1 << 26):
    """Fill the uint8 tensor `out` (length a multiple of 8) with stream bytes
    start .. start+len-1 (start a multiple of 8), in blocks to bound memory."""
    import torch

    assert out.dtype == torch.uint8 and out.numel() % 8 == 0 and start % 8 == 0
    words = out.view(torch.int64)
    n = words.numel()
    for w in range(0, n, block_words):
        c = min(block_words, n - w)
        words[w:w + c] = u64_torch(seed, start // 8 + w, c, out.device)
    return out


# --------------------------------------------------------------------------
# Batches of strings
# --------------------------------------------------------------------------
def align8(x):
    return (x + 7) & ~7


def pack_offsets(lengths: np.ndarray) -> np.ndarray:
    """int64[n+1] offsets of the 8-byte-aligned packing of `lengths`."""
    lengths = np.asarray(lengths, dtype=np.int64)
    n = lengths.size
    starts = np.zeros(n, dtype=np.int64)
    if n > 1:
        np.cumsum(align8(lengths[:-1]), out=starts[1:])
    offsets = np.zeros(n + 1, dtype=np.int64)
    offsets[1:] = starts + lengths
    return offsets


@dataclass
class Batch:
    """A packed batch of strings with seeded content.

    Byte q of the buffer is stream byte q of derive(seed, TAG_BYTES), except
    inside strings whose kind is KIND_ZERO (all zero) or KIND_REPEAT (every
    byte equal to fill[i])."""

    name: str
    seed: int
    lengths: np.ndarray
    offsets: np.ndarray = field(init=False)
    kind: Optional[np.ndarray] = None
    fill: Optional[np.ndarray] = None

    def __post_init__(self):
        self.lengths = np.asarray(self.lengths, dtype=np.int64)
        self.offsets = pack_offsets(self.lengths)

    @property
    def n(self) -> int:
        return int(self.lengths.size)

    @property
    def starts(self) -> np.ndarray:
        return align8(self.offsets[:-1])

    @property
    def data_bytes(self) -> int:
        return int(self.lengths.sum())

    @property
    def buffer_bytes(self) -> int:
        """Allocation size: the packed extent rounded up to 16 bytes."""
        return int((int(self.offsets[-1]) + 15) // 16 * 16) if self.n else 16

    def _special(self):
        if self.kind is None:
            return []
        return np.nonzero(self.kind != KIND_RANDOM)[0]

    def host_bytes(self) -> np.ndarray:
        buf = bytes_np(derive(self.seed, TAG_BYTES), 0, self.buffer_bytes)
        starts = self.starts
        for i in self._special():
            s, e = int(starts[i]), int(self.offsets[i + 1])
            buf[s:e] = 0 if self.kind[i] == KIND_ZERO else self.fill[i]
        return buf

    def device_bytes(self, device):
        import torch

        buf = torch.empty(self.buffer_bytes, dtype=torch.uint8, device=device)
        fill_bytes_torch(buf, derive(self.seed, TAG_BYTES))
        special = self._special()
        if len(special):
            starts = self.starts
            lens = self.lengths[special]
            short = special[lens <= 4096]
            long_ = special[lens > 4096]
            for i in long_:
                s, e = int(starts[i]), int(self.offsets[i + 1])
                buf[s:e] = 0 if self.kind[i] == KIND_ZERO else int(self.fill[i])
            if len(short):
                ls = self.lengths[short]
                idx = np.repeat(starts[short], ls) + (
                    np.arange(int(ls.sum())) - np.repeat(np.cumsum(ls) - ls, ls))
                vals = np.repeat(np.where(self.kind[short] == KIND_ZERO, 0, self.fill[short]), ls)
                buf[torch.from_numpy(idx).to(device)] = torch.from_numpy(
                    vals.astype(np.uint8)).to(device)
        return buf

    def string_bytes(self, i: int) -> np.ndarray:
        """Host copy of string i alone, without materialising the buffer."""
        s, e = int(self.starts[i]), int(self.offsets[i + 1])
        if self.kind is not None and self.kind[i] != KIND_RANDOM:
            v = 0 if self.kind[i] == KIND_ZERO else int(self.fill[i])
            return np.full(e - s, v, dtype=np.uint8)
        return bytes_np(derive(self.seed, TAG_BYTES), s, e - s)


def lognormal_lengths(seed: int, n: int, median: float = 24.0, sigma: float = 1.0,
                      lo: int = 1, hi: int = 65536, start: int = 0) -> np.ndarray:
    """round(exp(ln median + sigma Z)) clipped to [lo, hi]; Z ~ N(0, 1) by
    Box-Muller on two draws per string (draws 2i and 2i+1 of the stream)."""
    u = uniform01_np(derive(seed, TAG_LENGTHS), 2 * start, 2 * n).reshape(n, 2)
    z = np.sqrt(-2.0 * np.log(u[:, 0])) * np.cos(2.0 * math.pi * u[:, 1])
    lens = np.rint(np.exp(math.log(median) + sigma * z))
    return np.clip(lens, lo, hi).astype(np.int64)


# --------------------------------------------------------------------------
# The benchmark workloads
# --------------------------------------------------------------------------
def workload_c1(n: int = 10_000, seed: int = 1) -> Batch:
    """Plain per-string PM+32 case: lengths uniform in 1..256."""
    x = u64_np(derive(seed, TAG_LENGTHS), 0, n)
    return Batch("c1_uniform_1_256", seed, (x % np.uint64(256)).astype(np.int64) + 1)


def workload_c2_bytes(seed: int = 2) -> int:
    """The single-buffer case is 1 GiB of stream bytes of derive(seed, TAG_BYTES)."""
    return derive(seed, TAG_BYTES)


C2_BYTES = 1 << 30


def workload_c3(n: int = 4 * 1024 * 1024, seed: int = 3) -> Batch:
    """Batched ragged case: log-normal lengths, median 24 B, sigma_ln 1, 1..64 KiB."""
    return Batch("c3_lognormal_4M", seed, lognormal_lengths(seed, n))


def workload_c4(n: int = 2 * 1024 * 1024, seed: int = 4, long_frac: float = 0.01,
                long_lo: int = 1 << 20, long_hi: int = 16 << 20) -> Batch:
    """Skewed mix: 99% of lengths uniform in 8..64, 1% uniform in
    [long_lo, long_hi]; content 80% random, 10% zero, 10% one repeated byte."""
    ks = derive(seed, TAG_KIND)
    sel = uniform01_np(ks, 0, n)
    lx = u64_np(derive(seed, TAG_LENGTHS), 0, n)
    is_long = sel < long_frac
    short_len = 8 + (lx % np.uint64(57)).astype(np.int64)
    long_len = long_lo + (lx % np.uint64(long_hi - long_lo + 1)).astype(np.int64)
    lengths = np.where(is_long, long_len, short_len)
    c = uniform01_np(ks, n, n)
    kind = np.where(c < 0.8, KIND_RANDOM, np.where(c < 0.9, KIND_ZERO, KIND_REPEAT)).astype(np.uint8)
    fill = (u64_np(derive(seed, TAG_FILL), 0, n) & np.uint64(0xFF)).astype(np.uint8)
    return Batch("c4_skewed_2M", seed, lengths, kind=kind, fill=fill)


@dataclass
class Request:
    rid: int
    arrival_s: float
    width: int
    batch: Batch


def serving_requests(n_requests: int, rate_per_s: float, seed: int = 5,
                     max_strings: int = 100_000) -> list:
    """Poisson arrivals (exponential gaps) of requests with 1..max_strings
    strings each, log-normal lengths as in the batched case, and a 32- or
    64-bit output chosen with probability 1/2."""
    gaps = -np.log(uniform01_np(derive(seed, TAG_ARRIVALS), 0, n_requests)) / rate_per_s
    t = np.cumsum(gaps) - gaps[0]
    rs = u64_np(derive(seed, TAG_REQUESTS), 0, 2 * n_requests).reshape(n_requests, 2)
    reqs = []
    for r in range(n_requests):
        ns = 1 + int(rs[r, 0] % np.uint64(max_strings))
        width = 32 if int(rs[r, 1]) & 1 else 64
        rseed = derive(seed, 1000 + r)
        reqs.append(Request(r, float(t[r]), width,
                            Batch("req%d" % r, rseed, lognormal_lengths(rseed, ns))))
    return reqs
