"""Multi-GPU form of the bench: independent replicas, no data-path collective;
only the step time is reduced (MAX over ranks).  Checked with two gloo ranks
on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms_local = [120.0, 200.0][rank]
    value, ms = bench.replica_value(1_000_000, ms_local, ws, device="cpu")
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_value_two_ranks():
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
    # both ranks see the slowest rank's time; the value counts both replicas
    assert out[0] == out[1]
    value, ms = out[0]
    assert ms == 200.0
    assert value == pytest.approx(2 * 1_000_000 / 0.2 / 1e6)


def test_replica_value_single_rank():
    import bench
    assert bench.replica_value(4096, 2.0, 1) == (4096 / 2e-3 / 1e6, 2.0)
