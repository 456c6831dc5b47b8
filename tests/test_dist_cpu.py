"""The multi-GPU launch of bench.py (replicas, no data-path collective) on
CPU: two gloo ranks run the benchmark's distributed plumbing (process group
from the torchrun environment, barrier, max over ranks of the timed
seconds, whole-job rate = ranks x bytes / slowest rank's time)."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench

    d = bench.Dist()
    d.init("gloo")
    d.barrier()
    secs = 0.5 + rank  # the ranks' own timed seconds
    slowest = d.max(secs)
    rate = bench.whole_job_rate(d.world, 1 << 30, 3, slowest)
    d.barrier()
    q.put((rank, d.world, slowest, rate))
    d.done()


def test_two_gloo_ranks_take_the_slowest_rank():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=10) for _ in procs)
    for rank, world, slowest, rate in res:
        assert world == 2
        assert slowest == pytest.approx(1.5)
        assert rate == pytest.approx(2 * (1 << 30) * 3 / 1.5 / 1e9)


def test_single_rank_plumbing_needs_no_process_group():
    import sys

    sys.path.insert(0, ROOT)
    import bench

    d = bench.Dist()
    assert d.world == int(os.environ.get("WORLD_SIZE", "1"))
    d.init("gloo")  # no-op for one rank
    d.barrier()
    assert d.max(2.5) == 2.5
    assert bench.whole_job_rate(1, 100, 2, 4.0) == pytest.approx(100 * 2 / 4.0 / 1e9)


def test_bench_gpus_n_launches_n_replicas():
    """python bench.py --gpus 2 with no torchrun environment starts the two
    ranks itself; the line reports n_gpus = 2 and the slowest rank's time."""
    import json
    import subprocess
    import sys

    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--dry-run"],
                       capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(x) for x in p.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["n_gpus"] == 2 and line["dry_run"]
    assert line["slowest_s"] >= 0.04  # rank 1's pause
