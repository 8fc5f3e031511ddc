"""The benchmark's multi-rank aggregation over 2 gloo ranks on CPU: whole-job
throughput is all ranks' DOFs over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [100.0, 250.0][rank]
    dofs_local = [1000.0, 3000.0][rank]
    value, ms = bench.job_throughput(ms_local, dofs_local, "cpu", world)
    out[rank] = (value, ms)
    dist.barrier()
    dist.destroy_process_group()


def test_job_throughput_two_gloo_ranks():
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
    for r in range(2):
        value, ms = out[r]
        assert ms == 250.0 and abs(value - 4000.0 / 0.25) < 1e-9
