#!/usr/bin/env python3
"""Benchmark of PM+ hashing on GB300 (one JSON line on stdout, rank 0).

Headline workload: one 1 GiB uniform-random buffer (seed 2) hashed through
all PM+ tree levels with PM+64 and with PM+32 (the 32-bit variant on the same
buffer). One step = both hashes of the buffer; value = bytes hashed per second
over the whole job (GB/s, 1e9 bytes). Inputs are larger than L2 (1 GiB vs
129 MB), so no flush is needed between steps.

Beside it: the batched ragged case (4M log-normal strings) with the batched
path, one launch per string against the batched path (the 10,000-string case
and a 20,000-string prefix of the log-normal batch), the skewed mix (~176 GiB)
at full size, fixed-length keys, the streaming API on the 1 GiB buffer (256
MiB, 16 MiB and 1 MiB + 3 byte pieces), the serving loop (Poisson arrivals,
p50/p99), the oracle on the host cores (cpu_baseline on the buffer,
cpu_baseline_batched on the log-normal batch with one thread and with every
core), the paper's single-core figures as context, and the end-to-end rate
through the public API with the input copied from pinned host memory every
step (e2e).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  N > 1: one rank per GPU, replicas (each rank hashes its own buffer); run
  under torchrun, or started by bench.py itself through torch.distributed.run
  when no torchrun environment is set.
  --dry-run: the launch and timing plumbing alone on CPU (gloo; no GPU).
  --case small|batch|long|stream|fixed: one kernel family alone (ncu captures).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PM+32/PM+64 GB/s hashed and % of roofline; batched vs plain; p50/p99 latency"
C2_LEN = 1 << 30
WORKLOAD = ("one 1 GiB uniform-random buffer (seed 2) hashed through all PM+ tree levels, "
            "PM+64 then PM+32 on the same buffer")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="headline workload only")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-autotune", action="store_true",
                    help="small case: keep the default staging depth (ncu captures)")
    ap.add_argument("--dry-run", action="store_true",
                    help="replica launch, barrier and max-over-ranks timing on CPU (gloo), no GPU work")
    ap.add_argument("--case", default="c2", choices=["c2", "small", "batch", "long", "stream", "fixed"],
                    help="small: a 256 MiB buffer, both widths; batch: the 4M-string "
                         "batched case, both widths; stream: a 1 GiB buffer streamed in "
                         "256 MiB pieces, both widths; fixed: 256 MiB of keys of "
                         "--key-len bytes, both widths (ncu captures)")
    ap.add_argument("--key-len", type=int, default=8, help="fixed case: key length in bytes")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# distributed plumbing (replicas only: no data-path collective)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist

            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch

        t = torch.tensor([x], dtype=torch.float64,
                         device="cuda" if torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def done(self):
        if self.pg:
            self.pg.destroy_process_group()


def whole_job_rate(world: int, bytes_per_rank_step: int, steps: int, slowest_secs: float) -> float:
    """GB/s of the whole job: every rank hashes its own bytes each step; the
    job's time is the slowest rank's (max over ranks)."""
    return world * bytes_per_rank_step * steps / slowest_secs / 1e9


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.3)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        sms, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                maxes.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.f.name)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # median over samples under load (clock above a third of max)
        mx = max(maxes)
        loaded = [s for s in sms if s > mx / 3] or sms
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "samples": len(sms),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------
def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# sources the single-buffer tree kernel is compiled from
TREE_SOURCES = ("pm_async.cuh", "pm_device.cuh", "pm_kernels.cuh", "pm_tree.cuh")
E2E_PIECES = 8  # host-to-device pieces of the end-to-end step


def kernel_source_sha(files=TREE_SOURCES) -> str:
    """Hash of the kernel sources an ncu capture was taken on."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1609_09840_gb300", "csrc")
    for f in files:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch from the committed ncu summary
    (profiles/traffic.json), if it was taken on the current sources of that
    kernel (the entry lists them); else None."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
        e = d[kernel]
        if e.get("src_sha") != kernel_source_sha(tuple(e.get("sources", TREE_SOURCES))):
            return None
        return int(e["dram_bytes_per_launch"])
    except Exception:
        return None


def path_roofline(alg_bytes: int, secs: float, products: int, pk, hbm: float, kernel: str,
                  traffic_key: str = None, traffic_launches: int = 1) -> dict:
    """Roofline of one call of a path: achieved = algorithmic bytes / the
    call's CUDA-event time; bound = the lower of the measured copy bandwidth
    and the integer bound (the call's 32 x 32 -> 64 products of the chunk
    sums at the measured carry-chain multiply-add rate, pk['madc_per_s'],
    expressed as algorithmic bytes per second); frac against that bound."""
    achieved = alg_bytes / secs / 1e9
    int_bound = alg_bytes / (products / pk["madc_per_s"]) / 1e9 if pk and products else None
    bound = min(hbm, int_bound) if int_bound else hbm
    return {"bound": "hbm" if bound == hbm else "int", "achieved": achieved, "peak": bound, "unit": "GB/s",
            "frac": achieved / bound, "hbm_gbs": hbm, "int_bound_gbs": int_bound, "alg_bytes": alg_bytes,
            "products": products, "ms": secs * 1e3, "kernel": kernel,
            "traffic": (lambda t: t * traffic_launches if t is not None else None)(ncu_traffic(traffic_key))
            if traffic_key else None}


def timed_loop(torch, fn, steps, warmup, dist, stream):
    """Warm up, then time exactly `steps` calls with CUDA events on `stream`,
    bracketed by a barrier and a synchronize; returns (seconds, per-call ms)."""
    for _ in range(warmup):
        fn(None)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    ev[0].record(stream)
    for i in range(steps):
        fn(i)
        ev[i + 1].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    per = [ev[i].elapsed_time(ev[i + 1]) for i in range(steps)]
    return sum(per) / 1e3, per


# ---------------------------------------------------------------------------
# reference arm: the oracle on the host cores
# ---------------------------------------------------------------------------
def run_reference(args, dist):
    if dist.rank != 0:
        return
    from oracle import pmo
    from paper_1609_09840_gb300 import synth

    sample = 8 << 20  # bytes per width per step
    seed = synth.workload_c2_bytes(2)
    data = synth.bytes_np(seed, 0, sample)
    keys = {w: pmo.key_expand(pmo.width_params(w), 2) for w in (64, 32)}

    def step():
        for w in (64, 32):
            pmo.hash_bytes(pmo.width_params(w), keys[w], data)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    value = 2 * sample * args.steps / dt / 1e9
    desc = ("oracle (plain C, one thread) hashing the first %d MiB of the 1 GiB buffer "
            "with PM+64 and PM+32 per step" % (sample >> 20))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32+u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_bytes_per_width": sample},
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": desc},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def cpu_baseline(seconds: float):
    """The oracle as it stands, single-threaded, on a bounded prefix sample of
    the headline buffer (PM+64 and PM+32), about `seconds` of CPU work."""
    from oracle import pmo
    from paper_1609_09840_gb300 import synth

    seed = synth.workload_c2_bytes(2)
    probe = synth.bytes_np(seed, 0, 4 << 20)
    keys = {w: pmo.key_expand(pmo.width_params(w), 2) for w in (64, 32)}
    t0 = time.perf_counter()
    for w in (64, 32):
        pmo.hash_bytes(pmo.width_params(w), keys[w], probe)
    rate = 2 * probe.size / (time.perf_counter() - t0)
    nbytes = int(min(C2_LEN, max(4 << 20, rate * seconds / 2)) // (1 << 20) * (1 << 20))
    data = synth.bytes_np(seed, 0, nbytes)
    t0 = time.perf_counter()
    for w in (64, 32):
        pmo.hash_bytes(pmo.width_params(w), keys[w], data)
    dt = time.perf_counter() - t0
    return {"value": 2 * nbytes / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": "first %d MiB of the 1 GiB buffer, hashed with PM+64 and PM+32 as one "
                      "string each (%.1f s)" % (nbytes >> 20, dt)}


def _oracle_batch_part(task):
    """Worker of cpu_baseline_batched: the oracle on strings [a, b) of the
    4M-string log-normal batch (its lengths and bytes regenerated here from
    seed 3); returns (string bytes, seconds spent hashing)."""
    a, b, width = task
    from oracle import pmo
    from paper_1609_09840_gb300 import synth

    lengths = synth.lognormal_lengths(3, b)
    offs = synth.pack_offsets(lengths)
    s0 = int(offs[a]) & ~7
    sub = np.ascontiguousarray(offs[a:] - s0)
    buf = synth.bytes_np(synth.derive(3, synth.TAG_BYTES), s0, (int(sub[-1]) + 31) // 16 * 16)
    P = pmo.width_params(width)
    key = pmo.key_expand(P, 3)
    t0 = time.perf_counter()
    pmo.hash_batch(P, key, buf, sub)
    return int(lengths[a:].sum()), time.perf_counter() - t0


def cpu_baseline_batched(seconds: float):
    """The oracle as it stands on the 4M-string log-normal batch: one thread
    on a prefix of the strings (about seconds / 2 per width), and every host
    core on the whole batch (contiguous string ranges, one spawned process
    per core; rate = all string bytes / the slowest process's hashing time)."""
    import multiprocessing as mp

    n = 4 * 1024 * 1024
    single = {}
    for w in (32, 64):
        nb, dt = _oracle_batch_part((0, 20000, w))
        k = int(min(n, max(20000, 20000 / dt * seconds / 2)))
        nb, dt = _oracle_batch_part((0, k, w))
        single["pm%d" % w] = {"GB/s": nb / dt / 1e9, "strings": k, "seconds": dt}
    cores = os.cpu_count() or 1
    cuts = [n * i // cores for i in range(cores + 1)]
    allc = {}
    with mp.get_context("spawn").Pool(cores) as pool:
        for w in (32, 64):
            res = pool.map(_oracle_batch_part, [(cuts[i], cuts[i + 1], w) for i in range(cores)], chunksize=1)
            nb, slowest = sum(r[0] for r in res), max(r[1] for r in res)
            allc["pm%d" % w] = {"GB/s": nb / slowest / 1e9, "strings": n, "seconds": slowest}
    return {"kind": "oracle", "unit": "GB/s", "workload": "4,194,304 log-normal strings (median 24 B)",
            "single_thread": dict(single, cores=1), "all_cores": dict(allc, cores=cores),
            "sample": "one thread: the first strings of the batch, about %.0f s per width; all cores: "
                      "the whole batch split into %d contiguous ranges" % (seconds / 2, cores)}


def peaks(torch, native_peaks_lib, dev):
    """Read-only stream bandwidth and integer-multiply rates on this GPU."""
    import ctypes

    lib = ctypes.CDLL(native_peaks_lib)
    lib.pmpk_read_gbs.restype = ctypes.c_double
    lib.pmpk_read_gbs.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_int]
    lib.pmpk_imad_wide_per_s.restype = ctypes.c_double
    lib.pmpk_imad_wide_per_s.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.pmpk_mulhi64_per_s.restype = ctypes.c_double
    lib.pmpk_mulhi64_per_s.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.pmpk_madc_per_s.restype = ctypes.c_double
    lib.pmpk_madc_per_s.argtypes = [ctypes.c_void_p, ctypes.c_int]
    buf = torch.empty(2 << 30, dtype=torch.uint8, device=dev)
    buf.fill_(7)
    sink = torch.zeros(64, dtype=torch.uint8, device=dev)
    torch.cuda.synchronize()
    read = lib.pmpk_read_gbs(buf.data_ptr(), buf.numel(), sink.data_ptr(), 5)
    imad = lib.pmpk_imad_wide_per_s(sink.data_ptr(), 5)
    mulhi = lib.pmpk_mulhi64_per_s(sink.data_ptr(), 5)
    madc = lib.pmpk_madc_per_s(sink.data_ptr(), 5)
    del buf
    torch.cuda.synchronize()
    return {"read_gbs": read, "imad_wide_per_s": imad, "mulhi64_per_s": mulhi, "madc_per_s": madc}


def run_ours(args, dist):
    import torch

    from paper_1609_09840_gb300 import build, native, synth

    build.build()
    native.load()
    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    dist.init("nccl")
    stream = torch.cuda.current_stream()

    pk = peaks(torch, build.PEAKS_LIB, dev) if not args.no_extras else None

    # ----- headline: 1 GiB, PM+64 then PM+32 ---------------------------------
    buf = torch.empty(C2_LEN, dtype=torch.uint8, device=dev)
    synth.fill_bytes_torch(buf, synth.workload_c2_bytes(2))
    from paper_1609_09840_gb300 import autotune

    tuned = autotune.load_or_tune(buf)
    keys = {w: native.Key(seed=2, width=w) for w in (64, 32)}
    outs = {w: torch.empty(1, dtype=torch.int64 if w == 64 else torch.int32, device=dev)
            for w in (64, 32)}
    scr = {w: torch.empty(max(1, native.hash_scratch_bytes(w, C2_LEN)), dtype=torch.uint8, device=dev)
           for w in (64, 32)}
    ev = {w: [] for w in (64, 32)}

    def step(i):
        for w in (64, 32):
            if i is not None:
                a = torch.cuda.Event(enable_timing=True)
                a.record(stream)
            native.hash(keys[w], buf, out=outs[w], scratch=scr[w], stream=stream)
            if i is not None:
                b = torch.cuda.Event(enable_timing=True)
                b.record(stream)
                ev[w].append((a, b))

    clk = Clocks(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ
                 else dist.local)
    clk.start()
    secs, per = timed_loop(torch, step, args.steps, args.warmup, dist, stream)
    clocks = clk.stop()
    secs = dist.max(secs)
    per_launch = {w: statistics.mean(a.elapsed_time(b) for a, b in ev[w]) for w in (64, 32)}
    value = whole_job_rate(dist.world, 2 * C2_LEN, args.steps, secs)
    hbm, peak_kind = measured_peaks()

    # dominant kernel: the slower of the two tree launches
    wdom = max((64, 32), key=lambda w: per_launch[w])
    levels = {64: 4, 32: 5}
    alg_bytes = C2_LEN + 16 * ((C2_LEN // (128 * wdom // 8)) // 128 + 1)  # message + level-2 values
    achieved = alg_bytes / (per_launch[wdom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": ncu_traffic("k_tree<%d>" % wdom),
                "kernel": "k_tree<%d> (PM+%d single buffer, all levels)" % (wdom, wdom),
                "peak_kind": "%s copy bandwidth (MEASURED_PEAKS.json hbm_gbs, burst)" % peak_kind,
                "alg_bytes_per_launch": alg_bytes}
    if pk:  # context: against the read-only stream rate measured in this run
        roofline["read_stream_gbs"] = pk["read_gbs"]
        roofline["frac_of_read_stream"] = achieved / pk["read_gbs"]
    widths = {}
    for w in (64, 32):
        gbs = C2_LEN / (per_launch[w] * 1e-3) / 1e9
        widths["pm%d" % w] = {"ms_per_launch": per_launch[w], "GB/s": gbs,
                              "frac_of_hbm": gbs / hbm, "levels": levels[w]}
    if pk:
        # integer bound of the tree kernel's hot loop: full 32 x 32 products
        # on carry chains per byte (PM+32: 1 per 4-byte word; PM+64: 4 per
        # 8-byte word)
        for w, per_byte in ((32, 0.25), (64, 0.5)):
            widths["pm%d" % w]["int_bound_GB/s"] = pk["madc_per_s"] / per_byte / 1e9

    # ----- end to end through the public API with a pinned host input --------
    # The input is copied in E2E_PIECES pieces on a copy stream; each piece is
    # hashed with both widths through the streaming API as soon as it has
    # landed, so that only the last piece's hashing follows the copy.
    host = torch.empty(C2_LEN, dtype=torch.uint8, pin_memory=True)
    host.copy_(buf)
    res_host = {w: torch.empty(1, dtype=outs[w].dtype, pin_memory=True) for w in (64, 32)}
    want = {w: int(outs[w].item()) for w in (64, 32)}
    copy_stream = torch.cuda.Stream()
    strs = {w: native.Stream(keys[w]) for w in (64, 32)}
    piece = C2_LEN // E2E_PIECES
    landed = [torch.cuda.Event() for _ in range(E2E_PIECES)]
    lib = native.load()

    def e2e_step(i):
        start = torch.cuda.Event()
        start.record(stream)
        copy_stream.wait_event(start)  # the previous step is done with buf
        for w in (64, 32):
            strs[w].reset(stream=stream)
        for k in range(E2E_PIECES):
            with torch.cuda.stream(copy_stream):
                buf[k * piece:(k + 1) * piece].copy_(host[k * piece:(k + 1) * piece], non_blocking=True)
            landed[k].record(copy_stream)
            stream.wait_event(landed[k])
            for w in (64, 32):
                strs[w].update(buf[k * piece:(k + 1) * piece], stream=stream)
        for w in (64, 32):
            lib.pmp_stream_final(strs[w]._h, outs[w].data_ptr(), None, stream.cuda_stream)
            strs[w]._pieces = []
            res_host[w].copy_(outs[w], non_blocking=True)

    e2e_steps = max(3, min(args.steps, 10))
    esecs, _ = timed_loop(torch, e2e_step, e2e_steps, 1, dist, stream)
    esecs = dist.max(esecs)
    for w in (64, 32):
        assert int(res_host[w].item()) == want[w], "end-to-end hash differs from the single-buffer hash"
        strs[w].close()
    e2e = {"value": dist.world * 2 * C2_LEN * e2e_steps / esecs / 1e9, "unit": "GB/s",
           "h2d_bytes_per_step": C2_LEN, "d2h_bytes_per_step": 4 + 8,
           "how": "the 1 GiB input copied from pinned host memory in %d pieces on a copy stream, each piece "
                  "hashed with both widths through the streaming API once it has landed; both results read "
                  "back" % E2E_PIECES}
    del host

    line = {
        "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32+u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "bytes_per_step": 2 * C2_LEN, "levels": {"pm64": 4, "pm32": 5},
                   "l2": "inputs larger than L2 (1 GiB per buffer), no flush",
                   "parallelism": "replicas" if dist.world > 1 else "single GPU"},
        "roofline": roofline, "widths": widths, "e2e": e2e,
        "gpu_launches": 2 * args.steps, "clocks": clocks, "autotune": tuned,
    }
    if pk:
        line["peaks"] = pk

    if not args.no_extras:
        line["streaming"] = bench_streaming(torch, native, buf, keys, stream, hbm, pk, dist)
        del buf
        torch.cuda.empty_cache()
        line["batched"] = bench_batched(torch, native, synth, dev, stream, dist, hbm, pk)
        line["fixed_keys"] = bench_fixed(torch, native, synth, dev, stream, hbm, pk, dist)
        line["plain_vs_batched"] = bench_plain(torch, native, synth, dev, stream, dist)
        line["skewed"] = bench_skewed(torch, native, synth, dev, stream, dist, hbm, pk)
        if dist.rank == 0:
            line["serving"] = bench_serving(torch, native, synth)
    # context only (another machine): the paper's single-core Haswell i7-4770
    # figures for long random strings, Sec. 8 (variable-length results)
    line["paper_cpu_context"] = {
        "pm32": {"bytes_per_cycle": 4.7, "GB/s": 4.7 * 3.4},
        "pm64": {"bytes_per_cycle": 3.3, "GB/s": 3.3 * 3.4},
        "machine": "Intel i7-4770 at 3.4 GHz, one core, strings of 4 kB or more"}
    if dist.rank == 0 and not args.no_extras:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        line["cpu_baseline_batched"] = cpu_baseline_batched(args.cpu_seconds / 2)
    for k in keys.values():
        k.close()
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    dist.done()


def bench_streaming(torch, native, buf, keys, stream, hbm, pk, dist):
    """The 1 GiB buffer hashed through the streaming API (pmp_stream_*), fed
    in pieces of 256 MiB, 16 MiB and 1 MiB + 3 bytes (pieces at odd
    addresses), each width; the result is checked against the single-buffer
    hash. Whole strings (reset, every update, the result) run back to back,
    as the batched calls do, so that the host issues one while the device
    runs the one before; the best single synchronised string is reported
    beside it."""
    res = {"workload": "the 1 GiB buffer of the headline, appended in pieces, then one final()"}
    n = buf.numel()
    for w in (64, 32):
        ref = native.hash(keys[w], buf)
        s = native.Stream(keys[w])
        out = torch.empty(1, dtype=ref.dtype, device=buf.device)
        for piece in (256 << 20, 16 << 20, (1 << 20) + 3):
            def run():
                s.reset(stream=stream)
                for a in range(0, n, piece):
                    s.update(buf[a: a + piece], stream=stream)
                native.load().pmp_stream_final(s._h, out.data_ptr(), None, stream.cuda_stream)
                s._pieces = []
            run()
            torch.cuda.synchronize()
            assert int(out.item()) == int(ref.item()), "streamed hash differs from the single-buffer hash"
            ts = []
            for _ in range(3):
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                run()
                b.record(stream)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
            steps = 5 if piece >= 16 << 20 else 2
            secs, _ = timed_loop(torch, lambda i: run(), steps, 1, dist, stream)
            t = dist.max(secs) / steps
            assert int(out.item()) == int(ref.item()), "streamed hash differs from the single-buffer hash"
            res["pm%d_piece_%d" % (w, piece)] = {
                "ms": t * 1e3, "GB/s": n / t / 1e9, "frac_of_hbm": n / t / 1e9 / hbm,
                "single_string_ms": min(ts),
                "pieces": (n + piece - 1) // piece,
                # products: one per 4-byte word (PM+32), four per 8-byte word (PM+64)
                "roofline": path_roofline(n, t, n // 4 if w == 32 else n // 2, pk, hbm,
                                          "k_tree<%d> in the streaming modes + folds + final (every launch "
                                          "of the updates and the result)" % w,
                                          "k_tree_l2mode<%d>" % w if piece == 256 << 20 else None,
                                          (n + piece - 1) // piece)}
        s.close()
    return res


def bench_fixed(torch, native, synth, dev, stream, hbm, pk, dist):
    """Fixed-length keys (hash-table keys): 1 GiB of keys of 8, 16, 32 and 64
    bytes packed back to back, both widths, one call each; calls timed back
    to back (CUDA events between them), as the batched calls are."""
    buf = torch.empty(1 << 30, dtype=torch.uint8, device=dev)
    synth.fill_bytes_torch(buf, synth.derive(7, synth.TAG_BYTES))
    res = {"workload": "1 GiB of uniform-random keys per length, stride = length, one pmp_hash_fixed call"}
    for w in (32, 64):
        key = native.Key(seed=7, width=w)
        for L in (8, 16, 32, 64):
            n = buf.numel() // L
            out = torch.empty(n, dtype=torch.int32 if w == 32 else torch.int64, device=dev)
            steps = 8
            secs, _ = timed_loop(torch, lambda i: native.hash_fixed(key, buf, n, L, L, out=out, stream=stream),
                                 steps, 3, dist, stream)
            t = dist.max(secs) / steps
            alg = n * L + n * (w // 8)
            # products: the key's whole 8-byte units and its tail unit, 2 or 4 per
            # unit (when L % 8 == 0 the pad word's key word is one more product
            # in k_fixed_few, folded into a constant in k_fixed_one and added
            # without a multiply in k_fixed: not counted)
            prods = n * (L // 8 + (1 if L % 8 else 0)) * (2 if w == 32 else 4)
            kern = ("k_fixed_one<%d>" if L <= 8 else "k_fixed_few<%d>" if L <= 72 else "k_fixed<%d>") % w
            res["pm%d_len%d" % (w, L)] = {"ms": t * 1e3, "keys_per_s": n / t, "GB/s": n * L / t / 1e9,
                                         "frac_of_hbm": alg / t / 1e9 / hbm,
                                         "roofline": path_roofline(alg, t, prods, pk, hbm, kern,
                                                                   kern if L == 8 else "%s/%d" % (kern, L))}
        key.close()
    del buf
    torch.cuda.empty_cache()
    return res


def bench_batched(torch, native, synth, dev, stream, dist, hbm, pk):
    """4M log-normal strings (median 24 B, 1 B..64 KiB), one batched call per width."""
    b = synth.workload_c3()
    base = b.device_bytes(dev)
    offsets = torch.from_numpy(b.offsets).to(dev)
    res = {"workload": "4,194,304 strings, log-normal lengths (median 24 B, sigma_ln 1, "
                       "1 B..64 KiB), 8-byte-aligned packing, int64 offsets",
           "data_bytes": b.data_bytes, "strings": b.n}
    units = (b.lengths // 8 + 1) * 8  # bytes of 8-byte words read per string (incl. pad word)
    for w in (32, 64):
        key = native.Key(seed=3, width=w)
        out = torch.empty(b.n, dtype=torch.int32 if w == 32 else torch.int64, device=dev)
        scr = torch.empty(native.batch_scratch_bytes(w, b.n, b.buffer_bytes), dtype=torch.uint8, device=dev)
        steps = 20
        secs, per = timed_loop(torch, lambda i: native.hash_batch(key, base, offsets, out=out,
                                                                  scratch=scr, stream=stream),
                               steps, 3, dist, stream)
        secs = dist.max(secs)
        t = secs / steps
        alg = int(np.minimum(units, b.lengths + 8).sum()) + 8 * (b.n + 1) + b.n * (w // 8)
        g = native.graph_batch(key, base, offsets, out, scratch=scr)
        gsecs, _ = timed_loop(torch, lambda i: g.launch(stream), steps, 3, dist, stream)
        tg = dist.max(gsecs) / steps
        g.close()
        # products: every string's 8-byte units including the tail/pad unit, 2 or 4 per unit
        prods = int((b.lengths // 8 + 1).sum()) * (2 if w == 32 else 4)
        res["pm%d" % w] = {"GB/s": b.data_bytes / t / 1e9, "ms": t * 1e3,
                           "strings_per_s": b.n / t,
                           "alg_bytes": alg, "frac_of_hbm": alg / t / 1e9 / hbm,
                           "cuda_graph_ms": tg * 1e3, "cuda_graph_GB/s": b.data_bytes / tg / 1e9,
                           "roofline": path_roofline(alg, t, prods, pk, hbm,
                                                     "k_batch_range<%d> (one call: a 64-byte memset, the "
                                                     "range kernel, the chunk kernel's empty launch)" % w,
                                                     "k_batch_range<%d>" % w)}
        key.close()
    return res


def bench_skewed(torch, native, synth, dev, stream, dist, hbm, pk):
    """The skewed mix at full size: 2,097,152 strings, 1% of 1..16 MiB, the
    rest 8..64 B, with zero and repeated-byte content (~176 GiB), PM+64."""
    b = synth.workload_c4()
    torch.cuda.empty_cache()
    free, _ = torch.cuda.mem_get_info()
    if free < b.buffer_bytes + (8 << 30):
        return {"skipped": "needs %.0f GiB free" % (b.buffer_bytes / 2 ** 30)}
    base = b.device_bytes(dev)
    offsets = torch.from_numpy(b.offsets).to(dev)
    key = native.Key(seed=4, width=64)
    out = torch.empty(b.n, dtype=torch.int64, device=dev)
    scr = torch.empty(native.batch_scratch_bytes(64, b.n, b.buffer_bytes), dtype=torch.uint8, device=dev)
    secs, _ = timed_loop(torch, lambda i: native.hash_batch(key, base, offsets, out=out, scratch=scr,
                                                            stream=stream), 3, 1, dist, stream)
    t = dist.max(secs) / 3
    key.close()
    del base
    torch.cuda.empty_cache()
    alg = b.data_bytes + 8 * (b.n + 1) + 8 * b.n
    prods = int((b.lengths // 8 + 1).sum()) * 4
    return {"workload": "2,097,152 strings: 1% uniform 1..16 MiB, 99% uniform 8..64 B; 80% random, "
                        "10% zero, 10% repeated-byte content; PM+64",
            "data_bytes": b.data_bytes, "ms": t * 1e3, "GB/s": b.data_bytes / t / 1e9,
            "frac_of_hbm": alg / t / 1e9 / hbm,
            "roofline": path_roofline(alg, t, prods, pk, hbm, "k_long_chunk<64> (dominant) + k_batch_range<64>",
                                      "k_long_chunk<64>")}


def bench_serving(torch, native, synth, n_requests=2000):
    """Serving loop: Poisson arrivals of requests of 1..100,000 strings with the
    batched case's length law, each PM+32 or PM+64 with probability 1/2, under
    a 16 GiB device budget. Request payloads come from a pool of 48 seeded
    requests (seed 5) reused in arrival order. Capacity is measured closed
    loop first; the open-loop runs use 0.5x and 0.9x of it. Latency = arrival
    (submission) to results visible in host memory."""
    pool_reqs = synth.serving_requests(48, rate_per_s=1.0, seed=5)
    pool = []
    for r in pool_reqs:
        host = torch.from_numpy(r.batch.host_bytes()).pin_memory()
        offs = torch.from_numpy(r.batch.offsets).pin_memory()
        out = torch.empty(r.batch.n, dtype=torch.int32 if r.width == 32 else torch.int64).pin_memory()
        pool.append((r.width, host, offs, out, r.batch.data_bytes, r.batch.n))
    k32, k64 = native.Key(seed=5, width=32), native.Key(seed=5, width=64)
    server = native.Server(k32, k64, budget_bytes=16 << 30, slots=4)

    def run(arrivals):
        t0 = time.perf_counter()
        tickets = []
        for i, a in enumerate(arrivals):
            while time.perf_counter() - t0 < a:
                pass
            w, host, offs, out, _, _ = pool[i % len(pool)]
            tickets.append(server.submit(w, host, offs, out))
        for t in tickets:
            server.wait(t, timeout_s=120.0)
        times = [server.times(t) for t in tickets]
        for t in tickets:
            server.release(t)
        lat = np.array([(d - s_) / 1e6 for s_, _, d in times])  # ms
        span = (max(d for _, _, d in times) - min(s_ for s_, _, _ in times)) / 1e9
        nbytes = sum(pool[i % len(pool)][4] for i in range(len(arrivals)))
        nstr = sum(pool[i % len(pool)][5] for i in range(len(arrivals)))
        return lat, span, nbytes, nstr

    run([0.0] * 16)  # warm-up
    lat, span, nbytes, _ = run([0.0] * 200)
    capacity = 200 / span
    res = {"workload": "Poisson arrivals; requests of 1..100,000 strings (log-normal lengths, median "
                       "24 B), PM+32 or PM+64 with p = 1/2; 16 GiB device budget; 4 stream slots",
           "closed_loop": {"requests": 200, "requests_per_s": capacity, "GB/s": nbytes / span / 1e9,
                           "p50_ms": float(np.percentile(lat, 50)),
                           "p99_ms": float(np.percentile(lat, 99))}}
    for frac in (0.5, 0.9):
        gaps = -np.log(synth.uniform01_np(synth.derive(5, synth.TAG_ARRIVALS), 0, n_requests)) / (
            frac * capacity)
        arrivals = np.cumsum(gaps) - gaps[0]
        lat, span, nbytes, nstr = run(list(arrivals))
        res["load_%.1f" % frac] = {"requests": n_requests, "offered_requests_per_s": frac * capacity,
                                   "GB/s": nbytes / span / 1e9, "strings_per_s": nstr / span,
                                   "p50_ms": float(np.percentile(lat, 50)),
                                   "p99_ms": float(np.percentile(lat, 99))}
    server.close()
    k32.close()
    k64.close()
    return res


def bench_plain(torch, native, synth, dev, stream, dist):
    """One launch per string vs one batched call: the 10,000-string case
    (1..256 B, PM+32) and a 20,000-string prefix of the log-normal batch
    (both widths)."""
    b = synth.workload_c1()
    base = torch.from_numpy(b.host_bytes()).to(dev)
    offsets = torch.from_numpy(b.offsets).to(dev)
    key = native.Key(seed=1, width=32)
    out = torch.empty(b.n, dtype=torch.int32, device=dev)
    scr = torch.empty(native.batch_scratch_bytes(32, b.n, b.buffer_bytes), dtype=torch.uint8, device=dev)
    res = {"workload": "10,000 strings, lengths uniform 1..256 B, PM+32", "data_bytes": b.data_bytes}
    secs, _ = timed_loop(torch, lambda i: native.hash_batch_plain(key, base, offsets, out=out,
                                                                  stream=stream), 3, 1, dist, stream)
    t = dist.max(secs) / 3
    res["plain"] = {"ms": t * 1e3, "us_per_string": t / b.n * 1e6, "GB/s": b.data_bytes / t / 1e9}
    secs, _ = timed_loop(torch, lambda i: native.hash_batch(key, base, offsets, out=out, scratch=scr,
                                                            stream=stream), 20, 3, dist, stream)
    t = dist.max(secs) / 20
    res["batched"] = {"ms": t * 1e3, "us_per_string": t / b.n * 1e6, "GB/s": b.data_bytes / t / 1e9}
    key.close()
    # the log-normal batch's first 20,000 strings, both widths: one launch per
    # string (the whole 4M-string batch would take tens of seconds this way)
    # against the tile kernel on the same strings
    c3 = synth.workload_c3(n=20_000)
    base = torch.from_numpy(c3.host_bytes()).to(dev)
    offsets = torch.from_numpy(c3.offsets).to(dev)
    res["lognormal_sample"] = {"workload": "first 20,000 strings of the 4M log-normal batch",
                               "data_bytes": c3.data_bytes}
    for w in (32, 64):
        key = native.Key(seed=3, width=w)
        out = torch.empty(c3.n, dtype=torch.int32 if w == 32 else torch.int64, device=dev)
        scr = torch.empty(native.batch_scratch_bytes(w, c3.n, c3.buffer_bytes), dtype=torch.uint8, device=dev)
        secs, _ = timed_loop(torch, lambda i: native.hash_batch_plain(key, base, offsets, out=out, stream=stream),
                             3, 1, dist, stream)
        tp = dist.max(secs) / 3
        secs, _ = timed_loop(torch, lambda i: native.hash_batch(key, base, offsets, out=out, scratch=scr,
                                                                stream=stream), 20, 3, dist, stream)
        tb = dist.max(secs) / 20
        res["lognormal_sample"]["pm%d" % w] = {
            "plain_us_per_string": tp / c3.n * 1e6, "batched_us_per_string": tb / c3.n * 1e6,
            "speedup": tp / tb}
        key.close()
    return res


def run_small(args, dist):
    """A 256 MiB buffer (larger than L2, a few hundred MB on the device) hashed
    with PM+64 and PM+32: the case the ncu captures of the tree kernel use."""
    import torch

    from paper_1609_09840_gb300 import build, native, synth

    build.build()
    native.load()
    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    n = 256 << 20
    buf = torch.empty(n, dtype=torch.uint8, device=dev)
    synth.fill_bytes_torch(buf, synth.workload_c2_bytes(2))
    if not args.no_autotune:
        from paper_1609_09840_gb300 import autotune

        autotune.load_or_tune()
    keys = {w: native.Key(seed=2, width=w) for w in (64, 32)}
    scr = {w: torch.empty(max(1, native.hash_scratch_bytes(w, n)), dtype=torch.uint8, device=dev)
           for w in (64, 32)}
    stream = torch.cuda.current_stream()

    def step(i):
        for w in (64, 32):
            native.hash(keys[w], buf, scratch=scr[w], stream=stream)

    secs, _ = timed_loop(torch, step, args.steps, args.warmup, dist, stream)
    print(json.dumps({"case": "small", "bytes": n, "GB/s": 2 * n * args.steps / secs / 1e9}))


def run_long_case(args, dist):
    """The skewed mix at reduced size (100,000 strings, 1% of 1..4 MiB, ~2.6 GB),
    PM+64: the case the ncu captures of the long-string kernels use."""
    import torch

    from paper_1609_09840_gb300 import build, native, synth

    build.build()
    native.load()
    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    b = synth.workload_c4(n=100_000, seed=4, long_lo=1 << 20, long_hi=4 << 20)
    base = b.device_bytes(dev)
    offsets = torch.from_numpy(b.offsets).to(dev)
    stream = torch.cuda.current_stream()
    key = native.Key(seed=4, width=64)
    out = torch.empty(b.n, dtype=torch.int64, device=dev)
    scr = torch.empty(native.batch_scratch_bytes(64, b.n, b.buffer_bytes), dtype=torch.uint8, device=dev)

    def step(i):
        native.hash_batch(key, base, offsets, out=out, scratch=scr, stream=stream)

    secs, _ = timed_loop(torch, step, args.steps, args.warmup, dist, stream)
    print(json.dumps({"case": "long", "strings": b.n, "data_bytes": b.data_bytes,
                      "GB/s": b.data_bytes * args.steps / secs / 1e9}))


def run_batch_case(args, dist):
    """The 4M-string batched case with PM+32 and PM+64 (ncu captures)."""
    import torch

    from paper_1609_09840_gb300 import build, native, synth

    build.build()
    native.load()
    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    b = synth.workload_c3()
    base = b.device_bytes(dev)
    offsets = torch.from_numpy(b.offsets).to(dev)
    stream = torch.cuda.current_stream()
    keys = {w: native.Key(seed=3, width=w) for w in (32, 64)}
    outs = {w: torch.empty(b.n, dtype=torch.int64, device=dev) for w in (32, 64)}
    scr = torch.empty(native.batch_scratch_bytes(64, b.n, b.buffer_bytes), dtype=torch.uint8, device=dev)

    def step(i):
        for w in (32, 64):
            native.hash_batch(keys[w], base, offsets, out=outs[w], scratch=scr, stream=stream)

    secs, _ = timed_loop(torch, step, args.steps, args.warmup, dist, stream)
    print(json.dumps({"case": "batch", "strings": b.n,
                      "GB/s": 2 * b.data_bytes * args.steps / secs / 1e9}))


def run_stream_case(args, dist):
    """A 1 GiB buffer hashed through the streaming API in 256 MiB pieces,
    PM+64 then PM+32 (ncu captures of the streaming kernels)."""
    import torch

    from paper_1609_09840_gb300 import build, native, synth

    build.build()
    native.load()
    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    n, piece = 1 << 30, 256 << 20
    buf = torch.empty(n, dtype=torch.uint8, device=dev)
    synth.fill_bytes_torch(buf, synth.workload_c2_bytes(2))
    stream = torch.cuda.current_stream()
    streams = {w: native.Stream(native.Key(seed=2, width=w)) for w in (64, 32)}
    outs = {w: torch.empty(1, dtype=torch.int64, device=dev) for w in (64, 32)}

    def step(i):
        for w in (64, 32):
            s = streams[w]
            s.reset(stream=stream)
            for a in range(0, n, piece):
                s.update(buf[a:a + piece], stream=stream)
            native.load().pmp_stream_final(s._h, outs[w].data_ptr(), None, stream.cuda_stream)
            s._pieces = []

    secs, _ = timed_loop(torch, step, args.steps, args.warmup, dist, stream)
    print(json.dumps({"case": "stream", "piece_bytes": piece, "GB/s": 2 * n * args.steps / secs / 1e9}))


def run_fixed_case(args, dist):
    """256 MiB of keys of --key-len bytes (stride = length), PM+32 then PM+64
    (ncu captures of the fixed-length key kernels)."""
    import torch

    from paper_1609_09840_gb300 import build, native, synth

    build.build()
    native.load()
    dev = torch.device("cuda", dist.local)
    torch.cuda.set_device(dev)
    buf = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    synth.fill_bytes_torch(buf, synth.derive(7, synth.TAG_BYTES))
    L = args.key_len
    n = buf.numel() // L
    stream = torch.cuda.current_stream()
    keys = {w: native.Key(seed=7, width=w) for w in (32, 64)}
    outs = {32: torch.empty(n, dtype=torch.int32, device=dev), 64: torch.empty(n, dtype=torch.int64, device=dev)}

    def step(i):
        for w in (32, 64):
            native.hash_fixed(keys[w], buf, n, L, L, out=outs[w], stream=stream)

    secs, _ = timed_loop(torch, step, args.steps, args.warmup, dist, stream)
    print(json.dumps({"case": "fixed", "keys": n, "key_len": L, "GB/s": 2 * buf.numel() * args.steps / secs / 1e9}))


def launch_replicas(args) -> int:
    """bench.py --gpus N (N > 1) without a torchrun environment: one process
    per GPU through torch.distributed.run on this node (127.0.0.1), the same
    arguments; rank 0 prints the line. Returns the launcher's exit code."""
    import socket

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", str(args.gpus),
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def run_dry(args, dist):
    """The replica plumbing without GPU work: process group (gloo), barrier,
    each rank's own timed region (a fixed pause of 20 ms x (rank + 1)), max
    over ranks and the whole-job rate, as the real arm computes them."""
    dist.init("gloo")
    dist.barrier()
    t0 = time.perf_counter()
    time.sleep(0.02 * (dist.rank + 1))
    secs = time.perf_counter() - t0
    dist.barrier()
    slowest = dist.max(secs)
    if dist.rank == 0:
        print(json.dumps({"dry_run": True, "metric": METRIC, "n_gpus": dist.world, "slowest_s": slowest,
                          "value": whole_job_rate(dist.world, 1 << 20, 1, slowest), "unit": "GB/s"}),
              flush=True)
    dist.done()


def main():
    args = parse()
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        sys.exit(launch_replicas(args))
    dist = Dist()
    if args.dry_run:
        run_dry(args, dist)
        return
    if args.impl == "reference":
        run_reference(args, dist)
        return
    if args.case == "small":
        run_small(args, dist)
        return
    if args.case == "long":
        run_long_case(args, dist)
        return
    if args.case == "batch":
        run_batch_case(args, dist)
        return
    if args.case == "stream":
        run_stream_case(args, dist)
        return
    if args.case == "fixed":
        run_fixed_case(args, dist)
        return
    run_ours(args, dist)


if __name__ == "__main__":
    main()
