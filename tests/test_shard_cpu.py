"""The multi-rank path on CPU: frames dealt to ranks by pixel count, and the slowest rank's time, over a
world_size-2 gloo process group (no GPU, no data-path collective)."""
import os
import socket

import pytest

from paper_2408_14050_gb300 import shard


def test_assign_frames_covers_each_frame_once_and_balances():
    sizes = [640 * 480, 1280 * 720, 1920 * 1080, 4096 * 2160] * 16
    for world in (1, 2, 3, 4, 8):
        parts = shard.assign_frames(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    assert shard.assign_frames([5, 5, 5], 1) == [[0, 1, 2]]
    with pytest.raises(ValueError):
        shard.assign_frames([1], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, sizes, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = shard.assign_frames(sizes, world)[rank]
        t = shard.max_over_ranks(1.0 + rank)
        units = shard.sum_over_ranks(float(sum(sizes[i] for i in mine)))
        q.put((rank, mine, t, units))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_group():
    import torch.multiprocessing as mp
    sizes = [100, 300, 200, 50, 400, 250]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert sorted(res[0][1] + res[1][1]) == list(range(len(sizes)))
    assert not set(res[0][1]) & set(res[1][1])
    assert res[0][2] == res[1][2] == 2.0                 # the slowest rank's time
    assert res[0][3] == res[1][3] == float(sum(sizes))   # all units counted once


def test_bench_gpus_2_starts_two_ranks_and_reports_the_slowest():
    """bench.py --gpus 2, started as a plain process, starts two ranks under torch.distributed.run; in a dry run each
    rank waits (1 + rank) ms per step on the host and the line reports both ranks' units over the slower rank's time
    (max over a gloo group).  No GPU is touched."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_ADDR",
                                                            "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--dry-run", "--steps", "20",
                        "--warmup", "3"], capture_output=True, text=True, timeout=300, env=env, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = lines[0]
    assert line["n_gpus"] == 2 and line["dry_run"] and line["scaling"] == "weak"
    assert line["ms_per_step"] >= 2.0                     # rank 1's wait: the slowest rank sets the time
    assert abs(line["value"] - 2 * 1920 * 1080 * 8 / (line["ms_per_step"] / 1e3) / 1e6) / line["value"] < 1e-3
