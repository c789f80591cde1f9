"""The multi-rank path of bench.py on CPU with the gloo backend (world size 2):
each rank advances its own seeded ensemble with no data-path collective, the
job's time is the slowest rank's, and the job's rate counts every rank's cells."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    cases, desc = bench.workload("batch", 1802 + r)
    seconds = 1.0 + r                      # rank 1 is the slow one
    slowest = bench.max_over_ranks(seconds, dist, "cpu")
    cells = sum(c.mesh.ncells for c in cases)
    out[r] = (ws, r, cells, float(cases[0].phi0.sum()), slowest, bench.job_rate(cells, ws, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    (ws0, r0, c0, s0, slow0, rate0), (ws1, r1, c1, s1, slow1, rate1) = res[0], res[1]
    assert (ws0, r0, ws1, r1) == (2, 0, 2, 1)
    assert s0 != s1                        # different seeded ensembles per rank
    assert slow0 == slow1 == 2.0           # max over ranks
    assert rate0 == pytest.approx(2 * c0 / 2.0)
    assert rate1 == pytest.approx(2 * c1 / 2.0)
