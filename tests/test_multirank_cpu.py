"""The multi-GPU path shards independent lines/instances over ranks with no
data-path collective; only the timing is reduced (max over ranks).  This
covers that host logic with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    def reduce_max(x):
        t = torch.tensor([x], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    local = 1.0 + rank            # rank 1 is the slow one
    value, t = bench.aggregate(ws, 1000, local, reduce_max)
    out[rank] = (value, t)
    # ranks run independent instances: seeds differ, no data exchanged
    assert bench.dist_env() == (ws, rank, 0)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ws = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    os.environ.pop("LOCAL_RANK", None)
    mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
    for r in range(ws):
        value, t = out[r]
        assert t == 2.0
        assert value == pytest.approx(ws * 1000 / 2.0)


def test_single_rank_aggregation():
    import bench
    assert bench.aggregate(1, 500, 2.0) == (250.0, 2.0)
