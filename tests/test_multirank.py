"""The N > 1 bench path on CPU with gloo, world size 2: each rank takes its
own slice of the counter-based input stream (no data-path collective), the
slices tile the single-process stream exactly, and the step time reported is
the maximum over ranks."""
import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_0901_0638_gb300 import workloads as W


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    u = W.mixture_f64(2, n, first=bench.shard_first(rank, n))
    ms = 10.0 + rank                     # the slower rank sets the step time
    worst = bench.max_over_ranks(ms, dist)
    dist.barrier()
    out[rank] = (u, worst)
    dist.destroy_process_group()


def test_two_ranks_shard_stream_and_take_max_time():
    n, world = 4096, 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, n, out), nprocs=world, join=True)
        res = dict(out)
    full = W.mixture_f64(2, world * n)
    assert torch.equal(torch.cat([res[0][0], res[1][0]]), full)
    assert res[0][1] == res[1][1] == 11.0
