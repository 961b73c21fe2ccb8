"""The N-GPU benchmark runs independent replicas (one chain per rank, no
data-path exchange); its host logic, run here as two gloo ranks on the CPU:
the job time is the slowest rank's, the job rate sums the ranks' units over
it, and the replicas draw independent data."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    from paper_1603_08114_gb300 import synth
    t = bench._barrier_max(ws, 1.0 + 2.0 * rank)  # rank 1 is the slowest
    bench._barrier(ws)
    s = synth.rsv_series(64, synth.THETA_STD, seed=bench.replica_data_seed(rank))
    ys = [torch.zeros(64, dtype=torch.float64) for _ in range(ws)]
    dist.all_gather(ys, torch.tensor(s.y))
    rate = bench.job_rate(ws, 1000.0, t)
    if rank == 0:
        out.put((t, rate, [y.numpy() for y in ys]))
    dist.destroy_process_group()


def test_two_gloo_replicas():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    t, rate, ys = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert t == pytest.approx(3.0)            # the maximum over the ranks
    assert rate == pytest.approx(2 * 1000.0 / 3.0)
    assert not np.array_equal(ys[0], ys[1])  # independent replica data
