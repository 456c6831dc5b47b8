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


def apply(choices: dict):
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
    if not force and key in cache:
        apply(cache[key])
        return dict(cache[key], cached=True)
    res = tune_tree(buf)
    cache[key] = res
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path, "w") as f:
            json.dump(cache, f, indent=1)
    except OSError:
        pass
    return dict(res, cached=False)
