"""Multi-process path of bench.py on CPU: two gloo ranks (replicas) on 127.0.0.1."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, loc = bench.dist_setup()
    elapsed = 1.0 + rank            # rank 1 is the slow one
    m = bench.reduce_max(elapsed, w, device="cpu")
    out[rank] = (w, r, m, bench.rank_seed(r))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_max_and_distinct_seeds():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0][0] == out[1][0] == 2
    assert out[0][2] == out[1][2] == 2.0          # max over ranks
    assert out[0][3] != out[1][3]                 # replicas draw different inputs


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
