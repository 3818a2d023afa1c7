"""The multi-GPU path is independent replicas (the phi product of one workload
fits one GPU): every rank times its own calls, the job time is the maximum over
ranks and the value counts all ranks' calls.  Checked with two gloo ranks on
the CPU."""
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

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    local_ms = [40.0, 55.0][rank]            # rank 1 is the slow replica
    t, value = bench.aggregate_replicas(local_ms, steps=10, world=world, device="cpu")
    out[rank] = (t, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        t, value = out[r]
        assert t == pytest.approx(55.0)
        assert value == pytest.approx(2 * 10 / 0.055)


def test_single_process_aggregation():
    import bench

    t, value = bench.aggregate_replicas(20.0, steps=4, world=1)
    assert t == 20.0 and value == pytest.approx(200.0)
