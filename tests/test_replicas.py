"""Multi-GPU is replicas only (frames are independent): the bench's aggregation
over ranks -- max time over ranks, whole-job frames/s -- on two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = [1500.0, 2500.0][rank]           # rank 1 is the slow replica
    ms, value = bench.aggregate(local_ms, 1000, dist, torch.device("cpu"))
    out.put((rank, ms, value))
    dist.destroy_process_group()


def test_two_replicas_report_max_time_and_total_frames():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 2500.0
        assert value == pytest.approx(2 * 1000 / 2.5)
