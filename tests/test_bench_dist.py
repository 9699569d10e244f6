"""The multi-rank path of bench.py on CPU: two gloo ranks with different
timings agree on the slowest rank's time and on the whole-job MLUPS (all
ranks' cell updates over that time)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    local_ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    out[rank] = bench.aggregate(local_ms, 1000, 10, dist)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(ws, port, out), nprocs=ws, start_method="spawn", join=True)
    assert out[0] == out[1]
    ms, mlups = out[0]
    assert ms == pytest.approx(150.0)
    assert mlups == pytest.approx(ws * 1000 * 10 / 0.150 / 1e6)


def test_single_rank_without_process_group():
    import bench
    ms, mlups = bench.aggregate(20.0, 500, 4, None)
    assert ms == 20.0 and mlups == pytest.approx(500 * 4 / 0.020 / 1e6)
