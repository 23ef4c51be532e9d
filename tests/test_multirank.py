"""The multi-rank form of the benchmark on CPU: two gloo ranks, each propagating its own replica
(the oracle stands in for the device work), then the whole-job totals of bench.py: the units of
all ranks over the slowest rank's time.  No collective touches the propagation itself."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    import bench
    import oracle
    from paper_2510_20499_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = synth.binary_knapsack()
    l, u, r, _ = oracle.Problem(p).bp(p.lb, p.ub)
    ms = 10.0 + 5.0 * rank                       # a stand-in time per rank
    units, t = bench.whole_job(r["nnz_updates"], ms, torch.device("cpu"))
    # every replica reached the same fixpoint
    digest = torch.tensor([float(np.sum(l * 3.0 + u)), float(r["rounds"])], dtype=torch.float64)
    gathered = [torch.zeros_like(digest) for _ in range(world)]
    dist.all_gather(gathered, digest)
    out[rank] = (units, t, r["nnz_updates"], [g.tolist() for g in gathered])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_whole_job():
    import torch.multiprocessing as mp
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    nnz = res[0][2]
    for rank in range(world):
        units, t, mine, digests = res[rank]
        assert mine == nnz
        assert units == world * nnz                  # units of all ranks
        assert t == pytest.approx(10.0 + 5.0 * (world - 1))   # the slowest rank's time
        assert all(d == digests[0] for d in digests)


def test_single_process_is_local():
    sys.path.insert(0, ROOT)
    import torch

    import bench
    assert bench.whole_job(123, 4.5, torch.device("cpu")) == (123, 4.5)
