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
