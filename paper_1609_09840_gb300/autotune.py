"""Autotuner for the library's tuning knobs.

Times every choice of a knob on the current GPU with CUDA events, keeps the
fastest, and caches the winners in a JSON file keyed by GPU name and SM count
(default ~/.cache/pmplus/autotune.json, or $PMPLUS_AUTOTUNE_CACHE). Knobs only
change speed: every choice computes the same hashes (the GPU tests check each
one against the oracle).
"""
from __future__ import annotations

import json
import os

from . import native, synth

TREE_STAGE_CHOICES = (2, 3, 4, 6)
CHUNK_STAGE_CHOICES = (2, 3)
STREAM_SEGMENT_CHOICES = (1 << 17, 1 << 18, 1 << 19)
BATCH_P1_CHOICES = (6, 8)
# schedules of a batch's one-chunk strings: (name, schedule, range size, pass-1 depth)
BATCH_SCHEDULES = (("sorted-512", "sorted", 512, 6), ("sorted-1024", "sorted", 1024, 6),
                   ("tiles-p1-6", "tiles", 1024, 6), ("tiles-p1-8", "tiles", 1024, 8))
_SCHED_VALUE = {"sorted": "BATCH_SORTED", "tiles": "BATCH_TILES"}


def _cache_path() -> str:
    return os.environ.get("PMPLUS_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "pmplus", "autotune.json"))


def _gpu_key(torch) -> str:
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s/%d" % (p.name, p.multi_processor_count)


def _time(torch, fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune_tree(buf=None, nbytes: int = 1 << 30, reps: int = 5) -> dict:
    """Pick the TMA staging depth of the single-buffer tree kernel per width,
    timing a hash of `buf` (or of `nbytes` stream bytes)."""
    import torch

    if buf is None:
        buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        synth.fill_bytes_torch(buf, synth.derive(99, synth.TAG_BYTES))
    result = {}
    for width, knob in ((32, native.KNOB_TREE_STAGES_32), (64, native.KNOB_TREE_STAGES_64)):
        key = native.Key(seed=99, width=width)
        scratch = torch.empty(max(1, native.hash_scratch_bytes(width, buf.numel())),
                              dtype=torch.uint8, device=buf.device)
        out = torch.empty(1, dtype=torch.int64, device=buf.device)
        times = {}
        for stages in TREE_STAGE_CHOICES:
            native.tune_set(knob, stages)
            times[stages] = _time(torch, lambda: native.hash(key, buf, out=out, scratch=scratch), reps)
        best = min(times, key=times.get)
        native.tune_set(knob, best)
        result["tree_stages_%d" % width] = {"choice": best, "ms": times}
        key.close()
    return result


def set_batch_schedule(name: str):
    """Set the batch knobs of one entry of BATCH_SCHEDULES."""
    for nm, sched, rng, p1 in BATCH_SCHEDULES:
        if nm == name:
            native.tune_set(native.KNOB_BATCH_SCHED, getattr(native, _SCHED_VALUE[sched]))
            native.tune_set(native.KNOB_BATCH_RANGE, rng)
            native.tune_set(native.KNOB_BATCH_P1, p1)
            return
    raise ValueError(name)


def tune_batch(n: int = 1 << 21, reps: int = 5) -> dict:
    """Pick the schedule of a batch's one-chunk strings (sorted ranges of 512
    or 1024 strings, or tiles at either pass-1 depth), timing PM+32 and PM+64
    calls on `n` strings with the 4M-string case's length law."""
    import torch

    b = synth.workload_c3(n=n, seed=98)
    base = b.device_bytes("cuda")
    offsets = torch.from_numpy(b.offsets).cuda()
    keys = {w: native.Key(seed=98, width=w) for w in (32, 64)}
    out = torch.empty(b.n, dtype=torch.int64, device="cuda")
    scr = torch.empty(native.batch_scratch_bytes(64, b.n, base.numel()), dtype=torch.uint8, device="cuda")

    def call():
        for w in (32, 64):
            native.hash_batch(keys[w], base, offsets, out=out, scratch=scr)

    times = {}
    for name, _, _, _ in BATCH_SCHEDULES:
        set_batch_schedule(name)
        times[name] = _time(torch, call, reps)
    best = min(times, key=times.get)
    set_batch_schedule(best)
    for k in keys.values():
        k.close()
    return {"batch_schedule": {"choice": best, "ms": times}}


def tune_chunk(reps: int = 3) -> dict:
    """Pick the staging depth of the chunk kernel (a batch's strings of 32 or
    more level-1 chunks) for each width, timing calls on a reduced skewed
    mix: 20,000 strings, 1% of 1..4 MiB (about 0.5 GB)."""
    import torch

    b = synth.workload_c4(n=20000, seed=97, long_lo=1 << 20, long_hi=4 << 20)
    base = b.device_bytes("cuda")
    offsets = torch.from_numpy(b.offsets).cuda()
    result = {}
    for width, knob in ((32, native.KNOB_CHUNK_STAGES_32), (64, native.KNOB_CHUNK_STAGES_64)):
        key = native.Key(seed=97, width=width)
        out = torch.empty(b.n, dtype=torch.int64, device="cuda")
        scr = torch.empty(native.batch_scratch_bytes(width, b.n, base.numel()), dtype=torch.uint8, device="cuda")
        times = {}
        for st in CHUNK_STAGE_CHOICES:
            native.tune_set(knob, st)
            times[st] = _time(torch, lambda: native.hash_batch(key, base, offsets, out=out, scratch=scr), reps)
        best = min(times, key=times.get)
        native.tune_set(knob, best)
        key.close()
        result["chunk_stages_%d" % width] = {"choice": best, "ms": times}
    return result


def tune_stream(buf=None, nbytes: int = 1 << 30, piece: int = 256 << 20, reps: int = 3) -> dict:
    """Pick the segment size of streaming updates, timing `buf` (or `nbytes`
    stream bytes) appended in `piece`-byte pieces with PM+64 and PM+32."""
    import torch

    if buf is None:
        buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        synth.fill_bytes_torch(buf, synth.derive(96, synth.TAG_BYTES))
    n = buf.numel()
    streams = [native.Stream(native.Key(seed=96, width=w)) for w in (64, 32)]
    out = torch.empty(1, dtype=torch.int64, device=buf.device)

    def call():
        for s in streams:
            s.reset()
            for a in range(0, n, piece):
                s.update(buf[a:a + piece])
            native.load().pmp_stream_final(s._h, out.data_ptr(), None, None)
            s._pieces = []

    times = {}
    for seg in STREAM_SEGMENT_CHOICES:
        native.tune_set(native.KNOB_STREAM_SEGMENT, seg)
        times[seg] = _time(torch, call, reps)
    best = min(times, key=times.get)
    native.tune_set(native.KNOB_STREAM_SEGMENT, best)
    for s in streams:
        s.close()
    return {"stream_segment": {"choice": best, "ms": times}}


def apply(choices: dict):
    if "stream_segment" in choices:
        native.tune_set(native.KNOB_STREAM_SEGMENT, int(choices["stream_segment"]["choice"]))
    if "chunk_stages_32" in choices:
        native.tune_set(native.KNOB_CHUNK_STAGES_32, int(choices["chunk_stages_32"]["choice"]))
    if "chunk_stages_64" in choices:
        native.tune_set(native.KNOB_CHUNK_STAGES_64, int(choices["chunk_stages_64"]["choice"]))
    if "batch_schedule" in choices:
        set_batch_schedule(choices["batch_schedule"]["choice"])
    if "tree_stages_32" in choices:
        native.tune_set(native.KNOB_TREE_STAGES_32, int(choices["tree_stages_32"]["choice"]))
    if "tree_stages_64" in choices:
        native.tune_set(native.KNOB_TREE_STAGES_64, int(choices["tree_stages_64"]["choice"]))


def load_or_tune(buf=None, force: bool = False) -> dict:
    """Apply cached choices for this GPU, tuning (and caching) when absent."""
    import torch

    path = _cache_path()
    key = _gpu_key(torch)
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if not force and key in cache and "batch_schedule" in cache[key] and "chunk_stages_64" in cache[key] \
            and "stream_segment" in cache[key]:
        apply(cache[key])
        return dict(cache[key], cached=True)
    res = tune_tree(buf)
    res.update(tune_batch())
    res.update(tune_chunk())
    res.update(tune_stream(buf))
    cache[key] = res
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return dict(res, cached=False)
