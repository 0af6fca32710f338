"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

Each rank runs an independent replica (no data-path collective); the only
collectives are the timing reduction (max of times, sum of bytes) and the
barrier around the timed region."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, lr = bench.dist_env()
    assert (r, w, lr) == (rank, world, rank)
    ms = 10.0 + 5.0 * rank
    nbytes = 1e9 * (rank + 1)
    t, b = bench.reduce_max_sum(torch, ms, nbytes, torch.device("cpu"))
    bench.barrier_sync(torch)
    # replicas differ by seed but share the shape
    H, x = bench.make_matrix(dict(kind="stencil27", N=6, seed_a=1, seed_x=2), rank)
    out[rank] = (t, b, float(H.val[0]), int(H.nnz), float(x[0]))
    dist.destroy_process_group()


def test_two_rank_timing_reduction_and_replicas():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()  # no fork of a multi-threaded process
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    t0, b0, v0, n0, x0 = out[0]
    t1, b1, v1, n1, x1 = out[1]
    assert t0 == t1 == 15.0  # max over ranks
    assert b0 == b1 == 3e9  # bytes of all ranks
    assert n0 == n1 and v0 != v1 and x0 != x1


def test_single_process_is_identity():
    import bench
    assert not dist.is_initialized()
    assert bench.reduce_max_sum(torch, 3.0, 7.0, torch.device("cpu")) == (3.0, 7.0)
