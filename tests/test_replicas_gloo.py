"""The multi-GPU path of the benchmark runs independent replicas: the only
exchange is the timing reduction (max of the step time, sum of the units).
Covered here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(('127.0.0.1', 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    dist.init_process_group('gloo', rank=rank, world_size=world)
    import bench
    ms_local = [12.5, 13.75][rank]
    units_local = [1000.0, 1000.0][rank]
    ms, units = bench.reduce_timing(ms_local, units_local, True)
    out[rank] = (ms, units)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_reduction_two_ranks():
    port = _free_port()
    ctx = mp.get_context('spawn')
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ms, units = out[r]
        assert ms == 13.75 and units == 2000.0


def test_replica_timing_single_rank():
    import bench
    assert bench.reduce_timing(5.0, 7.0, False) == (5.0, 7.0)
