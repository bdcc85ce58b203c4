"""The multi-GPU path of the benchmark on CPU: two gloo ranks, each with its own
seeded shard (independent matrices, no data-path collective); the job's time is
the slowest rank's and the throughput counts every rank's units."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    import oracle
    from paper_2104_07638_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank: its own shard (seed 2 + rank), computed by the CPU oracle here
    A = inputs.hubbard_batch(4, 6, seed=2 + rank)
    m = oracle.minors_lu(A)
    c = oracle.cdet_recursion(m * m)
    t_rank = 1.0 + rank                       # pretend rank r took 1 + r seconds
    t_job = bench.max_over_ranks(t_rank, world)
    value = bench.job_throughput(4, world, 3, t_job)
    out[rank] = (t_job, value, float(c[:, -1].sum()), float(A.sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_slowest_time_and_count_all_units():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as man:  # no fork of a process that holds threads
        out = man.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.0                     # max over ranks
    assert res[0][1] == res[1][1] == 2 * 4 * 3 / 2.0         # all ranks' units / job time
    assert res[0][3] != res[1][3]                            # different shards per rank
