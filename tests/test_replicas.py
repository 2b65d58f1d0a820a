"""The multi-process path of bench.py (replicas, one per GPU) on CPU with gloo: the step
time is the maximum over ranks and the value counts all ranks' units."""
import os
import socket
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [2.0, 5.0][rank]
    out.put((rank, bench.aggregate_replicas(local_ms, 1000, dist, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_count_all_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        ms, value = res[r]
        assert ms == 5.0
        assert abs(value - 2 * 1000 / 5e-3) < 1e-6


def test_single_process_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_replicas(4.0, 100) == (4.0, 100 / 4e-3)
