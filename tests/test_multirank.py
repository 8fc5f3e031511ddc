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


def _replica_worker(rank, world, port, out):
    """One replica per rank, as bench.py --gpus N runs them: the rank's own
    seeded instance (J0 drawn from seed = rank), solved to tolerance (here by
    the oracle on a small grid, on CPU), then the whole-job aggregation."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import time

    import numpy as np

    import bench
    import workloads as W
    from oracle import periodic as P
    prob = W.config_mixed(seed=rank, n=9, N=8)
    t = time.perf_counter()
    d = P.assemble(prob)
    r = P.fixed_point(prob, d, tol=1e-8, max_it=20000)
    ms = (time.perf_counter() - t) * 1e3
    res = float(np.linalg.norm(P.residual(prob, d, r.U)) / np.linalg.norm(P.source(prob, d)))
    value, ms_max = bench.job_throughput(ms, d.n * d.N, "cpu", world)
    out[rank] = (float(prob.amp[0]), r.converged, res, d.n * d.N, ms, value, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_two_gloo_ranks_solve_their_own_instances():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_replica_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(300)
        assert p.exitcode == 0
    amps = [out[r][0] for r in range(2)]
    assert amps[0] != amps[1]                      # each rank its own seeded source
    for r in range(2):
        _, conv, res, dofs, ms, value, ms_max = out[r]
        assert conv and res <= 1e-8
        assert dofs == out[0][3]                   # weak scaling: the same work per rank
        assert ms_max == max(out[0][4], out[1][4])
        assert abs(value - 2 * dofs / (ms_max / 1e3)) <= 1e-9 * value
