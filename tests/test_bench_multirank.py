"""The N > 1 path of bench.py on CPU: world_size-2 gloo ranks.

Every rank runs an independent replica (replicas only: the workload has no data-path
exchange across GPUs in this build), the job time is the maximum over ranks, and the
reported value is the whole-job throughput."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]                  # the second replica is slower
    ms_max = bench.max_over_ranks(ms, world, device="cpu")
    out[rank] = (ms_max, bench.job_throughput(world, 64, 10, ms_max))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert out[0] == out[1]
    ms_max, value = out[0]
    assert ms_max == 150.0
    assert value == pytest.approx(2 * 64 * 10 / 0.150)
