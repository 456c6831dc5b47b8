"""Python binding of the PM+ CUDA library (libpmplus.so, C ABI in include/pmplus.h).

Argument marshalling only: every step of the hashing runs in the library's
CUDA kernels. PyTorch supplies device memory and streams. There is no CPU
fallback: if the compiled library is missing, load() raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpmplus.so")

PMP_OK, PMP_EINVAL, PMP_ENOMEM, PMP_ECUDA, PMP_ETOOLONG, PMP_ETIMEOUT, PMP_EALIGN, PMP_ESCRATCH = range(8)
KEY_WORDS = 8 * 129

_lib = None


class PmpError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.pmp_strerror(code).decode() if _lib is not None else str(code)
        super().__init__("%s failed: %s (status %d)" % (where, msg, code))


def load():
    """Load libpmplus.so (raises RuntimeError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libpmplus.so is missing: build it with __graft_entry__.build()")
    import torch  # noqa: F401  (initialise torch's CUDA runtime first)

    lib = ctypes.CDLL(LIB_PATH)
    vp, u64, i64, sz, ci = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_size_t, ctypes.c_int
    sig = {
        "pmp_key_create": (ci, [u64, ci, ctypes.POINTER(vp)]),
        "pmp_key_export": (ci, [vp, vp, sz]),
        "pmp_key_width": (ci, [vp]),
        "pmp_key_destroy": (None, [vp]),
        "pmp_hash_scratch_bytes": (sz, [ci, u64]),
        "pmp_hash32": (ci, [vp, vp, u64, vp, vp, sz, vp]),
        "pmp_hash64": (ci, [vp, vp, u64, vp, vp, sz, vp]),
        "pmp_batch_scratch_bytes": (sz, [ci, i64, u64]),
        "pmp_hash_batch32": (ci, [vp, vp, vp, i64, vp, vp, sz, vp]),
        "pmp_hash_batch64": (ci, [vp, vp, vp, i64, vp, vp, sz, vp]),
        "pmp_hash_batch_raw": (ci, [vp, vp, vp, i64, vp, vp, sz, vp]),
        "pmp_hash_batch32_plain": (ci, [vp, vp, vp, i64, vp, vp]),
        "pmp_hash_batch64_plain": (ci, [vp, vp, vp, i64, vp, vp]),
        "pmp_debug_reduce": (ci, [ci, vp, i64, vp, vp]),
        "pmp_check_alg2_32": (ci, [vp, vp]),
        "pmp_check_reduce32": (ci, [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32), ci, vp, vp]),
        "pmp_check_mix32": (ci, [ctypes.c_uint32, vp, vp]),
        "pmp_debug_wait_timeout": (ci, [vp, vp]),
        "pmp_hash64_noalloc": (ci, [vp, vp, u64, vp, vp]),
        "pmp_hash_noalloc_max_len": (u64, []),
        "pmp_tune_set": (ci, [ci, ci]),
        "pmp_graph_hash": (ci, [vp, vp, u64, vp, vp, sz, ctypes.POINTER(vp)]),
        "pmp_graph_batch": (ci, [vp, vp, vp, i64, vp, vp, sz, ctypes.POINTER(vp)]),
        "pmp_graph_launch": (ci, [vp, vp]),
        "pmp_graph_destroy": (None, [vp]),
        "pmp_server_create": (ci, [vp, vp, sz, ci, ctypes.POINTER(vp)]),
        "pmp_server_submit": (ci, [vp, ci, vp, vp, i64, vp, ctypes.POINTER(u64)]),
        "pmp_server_wait": (ci, [vp, u64, ctypes.c_double, ctypes.POINTER(ci)]),
        "pmp_server_ticket_times": (ci, [vp, u64, ctypes.POINTER(u64), ctypes.POINTER(u64),
                                         ctypes.POINTER(u64)]),
        "pmp_server_release": (ci, [vp, u64]),
        "pmp_server_stream_open": (ci, [vp, ci, ctypes.POINTER(u64)]),
        "pmp_server_submit_piece": (ci, [vp, u64, vp, u64, ci, vp, ctypes.POINTER(u64)]),
        "pmp_server_stream_close": (ci, [vp, u64]),
        "pmp_hash_batch_status": (ci, [vp, vp, vp, i64, vp, vp, vp, sz, vp]),
        "pmp_server_destroy": (None, [vp]),
        "pmp_hash_fixed32": (ci, [vp, vp, i64, ctypes.c_uint32, u64, vp, vp]),
        "pmp_hash_fixed64": (ci, [vp, vp, i64, ctypes.c_uint32, u64, vp, vp]),
        "pmp_count_collisions": (ci, [ci, u64, u64, vp, ctypes.c_uint32, vp, ctypes.c_uint32, ci, vp, vp]),
        "pmp_toy_regularity": (ci, [ci, ci, ci, ci, u64, ctypes.c_uint32, vp, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_uint32, vp, vp, vp]),
        "pmp_toy_delta_hist": (ci, [ci, ci, ci, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                    vp, vp]),
        "pmp_stream_create": (ci, [vp, ctypes.POINTER(vp)]),
        "pmp_stream_update": (ci, [vp, vp, u64, vp]),
        "pmp_stream_final": (ci, [vp, vp, vp, vp]),
        "pmp_stream_reset": (ci, [vp, vp]),
        "pmp_stream_length": (u64, [vp]),
        "pmp_stream_destroy": (None, [vp]),
        "pmp_tune_get": (ci, [ci, ctypes.POINTER(ci)]),
        "pmp_device_status": (ci, [ctypes.POINTER(ci)]),
        "pmp_strerror": (ctypes.c_char_p, [ci]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(rc: int, where: str):
    if rc != PMP_OK:
        raise PmpError(rc, where)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    import torch

    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _out_dtype(width: int):
    import torch

    return torch.int32 if width == 32 else torch.int64


def as_unsigned(t) -> np.ndarray:
    """Host numpy view of a result tensor with the unsigned dtype of its width."""
    a = t.detach().cpu().numpy()
    return a.view(np.uint32 if a.dtype == np.int32 else np.uint64)


class Key:
    """A PM+ key (8 levels of b_j, a_{j,1..128}) resident on a CUDA device."""

    def __init__(self, seed: int, width: int, device=None):
        import torch

        lib = load()
        self.width = int(width)
        self.seed = int(seed) & (2 ** 64 - 1)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.pmp_key_create(self.seed, self.width, ctypes.byref(h)), "pmp_key_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def export(self) -> np.ndarray:
        """The key words, level-major, as uint32 (width 32) or uint64 (width 64)."""
        out = np.zeros(KEY_WORDS, dtype=np.uint32 if self.width == 32 else np.uint64)
        _check(load().pmp_key_export(self._h, out.ctypes.data, out.nbytes), "pmp_key_export")
        return out

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().pmp_key_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hash_scratch_bytes(width: int, length: int) -> int:
    return int(load().pmp_hash_scratch_bytes(width, length))


def batch_scratch_bytes(width: int, n: int, data_bytes: int) -> int:
    """Scratch of a batch of n strings in a buffer of data_bytes bytes."""
    return int(load().pmp_batch_scratch_bytes(width, n, data_bytes))


def _scratch(nbytes: int, device, scratch=None):
    import torch

    if nbytes == 0:
        return None
    if scratch is not None and scratch.numel() >= nbytes:
        return scratch
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def hash(key: Key, buf, length: int = None, out=None, scratch=None, stream=None):
    """Hash one device byte buffer (16-byte aligned). Returns a 1-element
    int32/int64 tensor holding the uint32/uint64 hash."""
    import torch

    lib = load()
    n = buf.numel() if length is None else int(length)
    if out is None:
        out = torch.empty(1, dtype=_out_dtype(key.width), device=buf.device)
    scr = _scratch(hash_scratch_bytes(key.width, n), buf.device, scratch)
    fn = lib.pmp_hash32 if key.width == 32 else lib.pmp_hash64
    _check(fn(key.handle, _ptr(buf) if n else None, n, _ptr(out), _ptr(scr),
              scr.numel() if scr is not None else 0, _stream(stream)), fn.__name__)
    return out


def hash64_noalloc(key: Key, buf, length: int = None, out=None, stream=None):
    """PM+64 hash of one device buffer without any device allocation: the
    library's fixed per-device scratch array is used instead of caller scratch
    (for callers that may not allocate device memory). Calls that could overlap
    on the GPU must be serialised by the caller."""
    import torch

    n = buf.numel() if length is None else int(length)
    if out is None:
        out = torch.empty(1, dtype=torch.int64, device=buf.device)
    _check(load().pmp_hash64_noalloc(key.handle, _ptr(buf) if n else None, n, _ptr(out),
                                     _stream(stream)), "pmp_hash64_noalloc")
    return out


def hash_noalloc_max_len() -> int:
    return int(load().pmp_hash_noalloc_max_len())


def hash_batch(key: Key, base, offsets, out=None, scratch=None, stream=None, raw=False):
    """Hash the packed strings [align8(offsets[i]), offsets[i+1]) of `base`."""
    import torch

    lib = load()
    n = offsets.numel() - 1
    if out is None:
        out = (torch.empty(2 * n, dtype=torch.int64, device=base.device) if raw else
               torch.empty(n, dtype=_out_dtype(key.width), device=base.device))
    scr = _scratch(batch_scratch_bytes(key.width, n, base.numel()), base.device, scratch)
    if raw:
        fn = lib.pmp_hash_batch_raw
    else:
        fn = lib.pmp_hash_batch32 if key.width == 32 else lib.pmp_hash_batch64
    _check(fn(key.handle, _ptr(base), _ptr(offsets), n, _ptr(out), _ptr(scr),
              scr.numel() if scr is not None else 0, _stream(stream)), fn.__name__)
    return out


def hash_fixed(key: Key, keys, n: int, length: int, stride: int, out=None, stream=None):
    """Hash n keys of `length` bytes at `stride` in the uint8 device tensor `keys`."""
    import torch

    if out is None:
        out = torch.empty(n, dtype=_out_dtype(key.width), device=keys.device)
    lib = load()
    fn = lib.pmp_hash_fixed32 if key.width == 32 else lib.pmp_hash_fixed64
    _check(fn(key.handle, _ptr(keys), int(n), int(length), int(stride), _ptr(out), _stream(stream)), fn.__name__)
    return out


def count_collisions(width: int, seed0: int, nkeys: int, a, len_a: int, b, len_b: int, t_bits: int,
                     stream=None) -> int:
    """Keys of seeds seed0 .. seed0 + nkeys - 1 whose raw values of the
    one-chunk strings a and b (uint8 device tensors) agree in t_bits low bits."""
    import torch

    cnt = torch.zeros(1, dtype=torch.int64, device=a.device)
    _check(load().pmp_count_collisions(int(width), int(seed0), int(nkeys), _ptr(a), int(len_a), _ptr(b),
                                       int(len_b), int(t_bits), _ptr(cnt), _stream(stream)),
           "pmp_count_collisions")
    return int(cnt.item())


def toy_regularity(n: int, kappa: int, m: int, L: int, seed0: int, nkeys: int, data, length: int, comp0: int,
                   ncomp: int, want_raw: bool = False, stream=None):
    """Component-wise regularity of a toy member (p = 2^n + 1, n = 8 or 16):
    for each key and word position, counts (already-seen raw values, values
    mod 2^n seen twice, seen three times or more) as an (nkeys * ncomp, 3)
    int32 tensor, and the raw values ((nkeys * ncomp, 2^n)) when asked."""
    import torch

    dev = data.device if data is not None else torch.device("cuda")
    counts = torch.empty((nkeys * ncomp, 3), dtype=torch.int32, device=dev)
    raw = torch.empty((nkeys * ncomp, 1 << n), dtype=torch.int32, device=dev) if want_raw else None
    _check(load().pmp_toy_regularity(int(n), int(kappa), int(m), int(L), int(seed0), int(nkeys), _ptr(data),
                                     int(length), int(comp0), int(ncomp), _ptr(counts), _ptr(raw), _stream(stream)),
           "pmp_toy_regularity")
    return counts, raw


def toy_delta_hist(n: int, kappa: int, m: int, s, t, device="cuda", stream=None):
    """Histogram over every key in [1, p - kappa - 1]^m of f(s) - f(t) mod p
    for a toy one-chunk function (p = 2^n + 1): a (p,) int64 tensor."""
    import torch

    p = (1 << n) + 1
    hist = torch.empty(p, dtype=torch.int64, device=device)
    S = (ctypes.c_uint32 * m)(*[int(v) for v in s])
    T = (ctypes.c_uint32 * m)(*[int(v) for v in t])
    _check(load().pmp_toy_delta_hist(int(n), int(kappa), int(m), S, T, _ptr(hist), _stream(stream)),
           "pmp_toy_delta_hist")
    return hist


def hash_batch_plain(key: Key, base, offsets, out=None, stream=None):
    """Same results as hash_batch, one kernel launch per string."""
    import torch

    lib = load()
    n = offsets.numel() - 1
    if out is None:
        out = torch.empty(n, dtype=_out_dtype(key.width), device=base.device)
    fn = lib.pmp_hash_batch32_plain if key.width == 32 else lib.pmp_hash_batch64_plain
    _check(fn(key.handle, _ptr(base), _ptr(offsets), n, _ptr(out), _stream(stream)), fn.__name__)
    return out


def debug_reduce(width: int, S, stream=None):
    """Device reduction (Sec. 6.2 + Algorithm 2) of n sums given as (n, 3)
    int64 words; returns (n, 2) int64 words (low 64 bits, high bit)."""
    import torch

    n = S.shape[0]
    z = torch.empty((n, 2), dtype=torch.int64, device=S.device)
    _check(load().pmp_debug_reduce(width, _ptr(S), n, _ptr(z), _stream(stream)), "pmp_debug_reduce")
    return z


def _bad_counter():
    import torch

    return torch.zeros(1, dtype=torch.int64, device="cuda")


def check_alg2_32(stream=None) -> int:
    """Inputs (v0 < 2^32, v1 <= 2) where the device's Algorithm 2 differs
    from the integer remainder."""
    bad = _bad_counter()
    _check(load().pmp_check_alg2_32(_ptr(bad), _stream(stream)), "pmp_check_alg2_32")
    return int(bad.item())


def check_reduce32(pairs, stream=None) -> int:
    """Inputs r0 < 2^32 where the device reduction of r0 + 2^32 r1 + 2^64 r2
    differs from the integer remainder, over the given (r1, r2) pairs."""
    bad = _bad_counter()
    r1 = (ctypes.c_uint32 * len(pairs))(*[int(a) for a, _ in pairs])
    r2 = (ctypes.c_uint32 * len(pairs))(*[int(b) for _, b in pairs])
    _check(load().pmp_check_reduce32(r1, r2, len(pairs), _ptr(bad), _stream(stream)), "pmp_check_reduce32")
    return int(bad.item())


def check_mix32(a_inv: int, stream=None) -> int:
    """Inputs x where inverse(mix32(x)) != x, given the multiplier's inverse."""
    bad = _bad_counter()
    _check(load().pmp_check_mix32(int(a_inv), _ptr(bad), _stream(stream)), "pmp_check_mix32")
    return int(bad.item())


def debug_wait_timeout(stream=None) -> int:
    """Run the bounded-wait failure probe (about 2 s); returns 1 if the wait
    reported success, 0 if it gave up (the device status then holds
    PMP_ETIMEOUT)."""
    import torch

    res = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    _check(load().pmp_debug_wait_timeout(_ptr(res), _stream(stream)), "pmp_debug_wait_timeout")
    return int(res.item())


KNOB_TREE_STAGES_32, KNOB_TREE_STAGES_64, KNOB_BATCH_P1, KNOB_BATCH_SCHED, KNOB_BATCH_RANGE = 0, 1, 2, 3, 4
KNOB_CHUNK_STAGES_32, KNOB_STREAM_SEGMENT, KNOB_CHUNK_STAGES_64 = 5, 6, 7
BATCH_SORTED, BATCH_TILES = 0, 1


def tune_set(knob: int, value: int):
    _check(load().pmp_tune_set(knob, value), "pmp_tune_set")


def tune_get(knob: int) -> int:
    v = ctypes.c_int()
    _check(load().pmp_tune_get(knob, ctypes.byref(v)), "pmp_tune_get")
    return v.value


def device_status() -> int:
    v = ctypes.c_int()
    _check(load().pmp_device_status(ctypes.byref(v)), "pmp_device_status")
    return v.value


class Graph:
    """An executable CUDA graph of one hashing call (pmp_graph_*). Keeps the
    tensors it was captured with alive."""

    def __init__(self, handle, keep):
        self._h = handle
        self._keep = keep

    def launch(self, stream=None):
        _check(load().pmp_graph_launch(self._h, _stream(stream)), "pmp_graph_launch")

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().pmp_graph_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def graph_batch(key: Key, base, offsets, out, scratch=None) -> Graph:
    """Capture hash_batch(key, base, offsets, out) into a CUDA graph."""
    n = offsets.numel() - 1
    scr = _scratch(batch_scratch_bytes(key.width, n, base.numel()), base.device, scratch)
    h = ctypes.c_void_p()
    _check(load().pmp_graph_batch(key.handle, _ptr(base), _ptr(offsets), n, _ptr(out), _ptr(scr),
                                  scr.numel() if scr is not None else 0, ctypes.byref(h)),
           "pmp_graph_batch")
    return Graph(h, (key, base, offsets, out, scr))


def graph_hash(key: Key, buf, out, scratch=None) -> Graph:
    """Capture hash(key, buf, out=out) into a CUDA graph."""
    n = buf.numel()
    scr = _scratch(hash_scratch_bytes(key.width, n), buf.device, scratch)
    h = ctypes.c_void_p()
    _check(load().pmp_graph_hash(key.handle, _ptr(buf) if n else None, n, _ptr(out), _ptr(scr),
                                 scr.numel() if scr is not None else 0, ctypes.byref(h)),
           "pmp_graph_hash")
    return Graph(h, (key, buf, out, scr))


class Stream:
    """One string hashed from pieces (pmp_stream_*): update() appends device
    bytes, final() returns the hash of everything appended so far."""

    def __init__(self, key: Key):
        import torch

        lib = load()
        h = ctypes.c_void_p()
        with torch.cuda.device(key.device):
            _check(lib.pmp_stream_create(key.handle, ctypes.byref(h)), "pmp_stream_create")
        self._h = h
        self._key = key  # the key must outlive the stream
        self._pieces = []  # pieces stay alive until the next final()

    def update(self, piece, length: int = None, stream=None):
        """Append `length` bytes (default: all) of the uint8 device tensor `piece`."""
        n = piece.numel() if length is None else int(length)
        _check(load().pmp_stream_update(self._h, _ptr(piece) if n else None, n, _stream(stream)),
               "pmp_stream_update")
        self._pieces.append(piece)

    def final(self, out=None, raw=None, stream=None):
        """Queue the hash of the bytes so far into `out` (a one-element device
        tensor, created when None); `raw` optionally receives (lo, hi)."""
        import torch

        if out is None:
            out = torch.empty(1, dtype=_out_dtype(self._key.width), device=self._key.device)
        _check(load().pmp_stream_final(self._h, _ptr(out), _ptr(raw), _stream(stream)), "pmp_stream_final")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        self._pieces = []
        return out

    def reset(self, stream=None):
        _check(load().pmp_stream_reset(self._h, _stream(stream)), "pmp_stream_reset")

    def __len__(self):
        return int(load().pmp_stream_length(self._h))

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().pmp_stream_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Request loop with continuous batching (pmp_server_*): requests are
    packed batches in host memory; results land in host memory."""

    def __init__(self, key32: Key, key64: Key, budget_bytes: int, slots: int = 4):
        import torch

        lib = load()
        h = ctypes.c_void_p()
        with torch.cuda.device(key32.device):
            _check(lib.pmp_server_create(key32.handle, key64.handle, int(budget_bytes), int(slots),
                                         ctypes.byref(h)), "pmp_server_create")
        self._h = h
        self._keys = (key32, key64)  # the keys must outlive the server
        self._live = {}

    def submit(self, width: int, base, offsets, out) -> int:
        """base: uint8 host array/tensor; offsets: int64 host (n+1); out: host
        array of n uint32/uint64 (int32/int64 tensors are fine). Keeps the
        buffers alive until the ticket is released."""
        n = len(offsets) - 1
        t = ctypes.c_uint64()
        _check(load().pmp_server_submit(self._h, width, _host_ptr(base), _host_ptr(offsets), n,
                                        _host_ptr(out), ctypes.byref(t)), "pmp_server_submit")
        self._live[t.value] = (base, offsets, out)
        return t.value

    def wait(self, ticket: int, timeout_s: float = 60.0) -> bool:
        done = ctypes.c_int()
        _check(load().pmp_server_wait(self._h, ticket, timeout_s, ctypes.byref(done)),
               "pmp_server_wait")
        return bool(done.value)

    def wait_status(self, ticket: int, timeout_s: float = 60.0):
        """(done, status code) of a ticket, without raising on a failed request."""
        done = ctypes.c_int()
        rc = load().pmp_server_wait(self._h, ticket, timeout_s, ctypes.byref(done))
        return bool(done.value), rc

    def stream_open(self, width: int) -> int:
        """A string held by the server (device-resident tree state)."""
        sid = ctypes.c_uint64()
        _check(load().pmp_server_stream_open(self._h, width, ctypes.byref(sid)), "pmp_server_stream_open")
        return sid.value

    def submit_piece(self, stream_id: int, piece, final: bool = False, out=None) -> int:
        """Append a host piece (uint8 array/tensor) to a server string; with
        final=True, out (a host array of one uint32/uint64) receives the hash
        of everything appended so far. Keeps the buffers alive until release."""
        t = ctypes.c_uint64()
        n = len(piece)
        _check(load().pmp_server_submit_piece(self._h, stream_id, _host_ptr(piece) if n else None, n,
                                              1 if final else 0, _host_ptr(out) if final else None,
                                              ctypes.byref(t)), "pmp_server_submit_piece")
        self._live[t.value] = (piece, out)
        return t.value

    def stream_close(self, stream_id: int):
        _check(load().pmp_server_stream_close(self._h, stream_id), "pmp_server_stream_close")

    def times(self, ticket: int):
        """(submit, admit, done) steady-clock nanoseconds of a ticket."""
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().pmp_server_ticket_times(self._h, ticket, ctypes.byref(a), ctypes.byref(b),
                                              ctypes.byref(c)), "pmp_server_ticket_times")
        return a.value, b.value, c.value

    def release(self, ticket: int):
        _check(load().pmp_server_release(self._h, ticket), "pmp_server_release")
        self._live.pop(ticket, None)

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            load().pmp_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _host_ptr(x):
    """Address of a host numpy array or CPU torch tensor."""
    if isinstance(x, np.ndarray):
        return ctypes.c_void_p(x.ctypes.data)
    return ctypes.c_void_p(x.data_ptr())
