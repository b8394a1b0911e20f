"""Multi-rank replica path of bench.py on CPU (gloo, world size 2): each rank
solves its own seeded indentation, and the timed region is the MAX over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    m = W.fingertip_mesh(h=2.5)
    ind = W.indenters.fingertip_sphere_indentation(m, seed=bench.replica_seed(rank))
    t = bench.max_over_ranks(1.0 + rank, world)
    out[rank] = (t, tuple(ind.origin))
    dist.destroy_process_group()


def test_two_replicas_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 2.0          # max over ranks on every rank
    assert out[0][1] != out[1][1]                  # each replica has its own draw


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
