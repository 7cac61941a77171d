"""The multi-GPU host logic of the benchmark on two CPU ranks (gloo): every
rank takes its own disks per step (disjoint, consecutive blocks) and only the
timings cross ranks (max and sum reductions)."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ids = [bench.disk_ids(k, rank, world, 19, 768, 300) for k in range(-3, 6)]
    mx = bench.max_over_ranks(float(rank + 1), world)
    sm = bench.sum_over_ranks(float(10 * (rank + 1)), world)
    q.put((rank, ids, mx, sm))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(180)
def test_two_ranks_shard_disks_and_reduce_timings():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r, (ids, mx, sm)) for r, ids, mx, sm in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for k in range(9):
        a, b = set(out[0][0][k]), set(out[1][0][k])
        assert len(a) == len(b) == 19 and not (a & b)
        both = sorted(out[0][0][k] + out[1][0][k])
        assert both == sorted((300 + (k - 3) * 38 + i) % 768 for i in range(38))
    assert out[0][1] == out[1][1] == 2.0
    assert out[0][2] == out[1][2] == 30.0
