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


def _seed_worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench
    from paper_2605_24514_gb300 import streams
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    S = 4096
    # the panel seeds the batched workload gives its streams on this rank, and a digest of a few panels
    seeds = [bench.rank_seed(rank) * 1_000_003 + s + 1 for s in range(S)]
    digest = [float(streams.make_panel(20, 10, 5, seed=sd)[0].sum()) for sd in seeds[:4]]
    t = torch.tensor([min(seeds), max(seeds)] + digest, dtype=torch.float64)
    got = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(got, t)
    out[rank] = [g.tolist() for g in got]
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_draw_disjoint_stream_sets():
    """Replicas shard the batched workload by rank: the streams' panel seeds of two ranks do not
    overlap, so no stream is served twice and each rank's pool admits only its own streams."""
    pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_seed_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    (lo0, hi0, *d0), (lo1, hi1, *d1) = out[0]
    assert out[0] == out[1]                       # both ranks saw the same gathered view
    assert hi0 < lo1 or hi1 < lo0                 # disjoint seed ranges
    assert all(a != b for a, b in zip(d0, d1))    # and different panels
