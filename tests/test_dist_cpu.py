"""Host logic of the multi-GPU bench on CPU: world_size-2 gloo ranks.

Frames are independent, so N GPUs run N replicas on disjoint frames with no
collective on the data path; ranks meet only at a barrier and a max-reduce
of the timed region. This exercises that logic with gloo on CPU.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    frames = bench.rank_frame_indices(rank, 4)
    t = bench.reduce_max(float(10 + rank), world)
    bench.barrier(world)
    gathered = [None] * world
    dist.all_gather_object(gathered, frames)
    out[rank] = (t, gathered)
    dist.destroy_process_group()


def test_two_rank_replicas_and_max_reduce():
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, gathered = out[r]
        assert t == 11.0  # max over ranks
        assert gathered[0] == [0, 1, 2, 3] and gathered[1] == [4, 5, 6, 7]  # disjoint frames


def test_single_rank_helpers():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.rank_frame_indices(2, 3) == [6, 7, 8]
    bench.barrier(1)
