"""The multi-GPU measurement protocol (independent replicas, barrier and
max over ranks) on CPU: two gloo ranks, no GPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2411_14968_gb300.replicas import Replicas, throughput
    r = Replicas(world)
    r.barrier()
    secs = 1.0 + rank  # rank 1 is the slow one
    m = r.max_over_ranks(secs)
    total = r.sum_over_ranks(10.0)
    out[rank] = (m, total, throughput(4e6, world, m))
    r.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    for rank in range(world):
        m, total, thr = res[rank]
        assert m == 2.0 and total == 20.0
        assert thr == pytest.approx(4e6 * 2 / 2.0)


def test_single_replica_needs_no_process_group():
    from paper_2411_14968_gb300.replicas import Replicas, dist_env, throughput
    r = Replicas(1)
    r.barrier()
    assert r.max_over_ranks(3.5) == 3.5
    assert throughput(10.0, 1, 2.0) == 5.0
    assert dist_env()[1] >= 1
