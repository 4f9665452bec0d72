"""The N > 1 host logic of bench.py on CPU with gloo (world size 2): each rank draws its own
particles, the job time is the slowest rank's, and the job value counts every rank's points."""
import os
import socket

import numpy as np
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench.make_workload("tiny", 1.0, rank)
    local_ms = 10.0 + 5.0 * rank
    m = bench.max_over_ranks(local_ms, dist, torch.device("cpu"))
    out[rank] = (m, float(w.particles[0, 0]), bench.job_value(w.n_points, world, m))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] != res[1][1]  # independent particles per rank
    n_points = 11000
    assert res[0][2] == pytest.approx(world * n_points / 0.015)
    assert np.isfinite(res[1][2])
