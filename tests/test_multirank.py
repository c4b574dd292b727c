"""bench.py's multi-rank aggregation, on CPU with the gloo backend (world size 2).

With N GPUs the benchmark runs N independent replicas (the path is not
sharded); each rank times its own steps, the reported time is the maximum over
ranks and the value counts every rank's particles.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


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
    ms = [12.5, 20.0][rank]
    mx = bench._barrier_max(torch, ms, ws)
    out[rank] = (mx, bench.weak_value(1000, ws, 10, mx))
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_value():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(ws, _free_port(), out), nprocs=ws, start_method="spawn", join=True)
    for r in range(ws):
        mx, val = out[r]
        assert mx == 20.0
        assert val == pytest.approx(1000 * 2 * 10 / 0.020)
