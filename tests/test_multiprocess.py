"""The N > 1 path of bench.py (independent replicas) on CPU: two gloo ranks, max over ranks of the
timed region and the whole-job value = all ranks' node updates / the slowest rank's time."""
import os
import socket
import sys
from pathlib import Path

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parent.parent


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out):
    sys.path.insert(0, str(ROOT))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    assert bench.dist_env() == (ws, rank, rank)
    local_ms = 100.0 + 50.0 * rank             # rank 1 is the slow one
    ms, glups = bench.replica_aggregate(local_ms, nodes_per_rank=1_000_000, steps=10, ws=ws)
    out[rank] = (ms, glups)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_aggregate_like_the_benchmark():
    ws = 2
    port = _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_worker, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for rank in range(ws):
        ms, glups = res[rank]
        assert ms == 150.0
        assert abs(glups - 2 * 1_000_000 * 10 / 0.150 / 1e9) < 1e-12
