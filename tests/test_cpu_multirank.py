"""The data-parallel path on CPU: two gloo ranks.

Each rank takes a contiguous slice of one seeded batch (dist.shard_bounds,
inputs.hubbard_batch_slice); the one exchange of the path is the per-order sum
table of the connected sums of whole vertex sets (dist.combine_order_sums) and,
for data-parallel training of the surrogate, the averaged gradient
(dist.average_gradient_). The combined results must equal those of a single
rank over the concatenated slices. The per-rank tables and gradients come from
the oracle here (the device reduction apm_order_sums is checked against the
same definition in tests/test_gpu_order_sums.py); the benchmark's timing
helpers are checked as well: the job's time is the slowest rank's and the
throughput counts every rank's units."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2104_07638_gb300 import dist as D  # noqa: E402

TOTAL, ORDER, SEED = 10, 6, 21


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def order_table(c_full, n, n_max):
    """(count, sum c, sum |c|, sum c^2) per order, the definition apm_order_sums computes."""
    t = np.zeros((n_max + 1, 4))
    v = np.asarray(c_full, dtype=np.float64)
    t[n] = [v.size, v.sum(), np.abs(v).sum(), (v * v).sum()]
    return t


def connected_full_sets(A):
    import oracle
    m = oracle.minors_lu(A)
    return oracle.cdet_recursion(m * m)[:, -1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    import oracle.mlp as om
    from paper_2104_07638_gb300 import dist as Dr
    from paper_2104_07638_gb300 import inputs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    assert Dr.world() == (rank, world)
    # estimator sums: this rank's slice of one seeded batch
    lo, hi = Dr.shard_bounds(TOTAL, rank, world)
    A = inputs.hubbard_batch_slice(TOTAL, ORDER, SEED, lo, hi)
    local = torch.tensor(order_table(connected_full_sets(A), ORDER, ORDER + 2))
    total = Dr.combine_order_sums(local)
    # surrogate gradient over this rank's rows, averaged with the row count as weight
    rng = np.random.default_rng(7)
    flat = rng.standard_normal(om.NPARAM).astype(np.float32) * 0.05
    X = rng.standard_normal((9, 64))
    t = rng.standard_normal(9)
    rows = slice(*Dr.shard_bounds(9, rank, world))
    _, g = om.loss_and_grad(om.unpack(flat), X[rows], t[rows])
    grad = torch.tensor(om.pack(g), dtype=torch.float32)
    Dr.average_gradient_(grad, float(X[rows].shape[0]))
    # timing helpers of the benchmark
    t_job = bench.max_over_ranks(1.0 + rank, world)
    value = bench.job_throughput(4, world, 3, t_job)
    out[rank] = (total.numpy(), grad.numpy(), t_job, value, (lo, hi))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_bounds_partition():
    for total in (0, 1, 7, 64, 65537):
        for w in (1, 2, 3, 8):
            b = [D.shard_bounds(total, r, w) for r in range(w)]
            assert b[0][0] == 0 and b[-1][1] == total
            assert all(b[i][1] == b[i + 1][0] for i in range(w - 1))
            assert max(h - l for l, h in b) - min(h - l for l, h in b) <= 1
    with pytest.raises(ValueError):
        D.shard_bounds(4, 2, 2)


def test_single_process_exchange_is_identity():
    t = torch.arange(12, dtype=torch.float64).reshape(3, 4)
    assert torch.equal(D.combine_order_sums(t), t)
    g = torch.ones(5)
    assert torch.equal(D.average_gradient_(g, 3.0), torch.ones(5))
    est = D.estimator(torch.tensor([[0, 0, 0, 0], [4, 2.0, 6.0, 14.0]], dtype=torch.float64))
    assert list(est) == [1] and est[1]["count"] == 4 and est[1]["mean"] == 0.5
    assert est[1]["sign"] == pytest.approx(1 / 3) and est[1]["mean_abs"] == 1.5
    assert est[1]["stderr"] == pytest.approx(np.sqrt((14 / 4 - 0.25) / 3))


def test_two_gloo_ranks_exchange_equals_one_rank_over_the_union():
    import oracle.mlp as om
    from paper_2104_07638_gb300 import inputs
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as man:  # no fork of a process that holds threads
        out = man.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    # the slices cover the batch, and the combined table is the whole batch's
    assert res[0][4] == (0, 5) and res[1][4] == (5, 10)
    whole = order_table(connected_full_sets(inputs.hubbard_batch(TOTAL, ORDER, seed=SEED)), ORDER, ORDER + 2)
    for r in range(world):
        assert res[r][0][ORDER][0] == TOTAL
        np.testing.assert_allclose(res[r][0], whole, rtol=1e-13, atol=0)
    e = D.estimator(torch.tensor(res[0][0]))
    ew = D.estimator(torch.tensor(whole))
    assert e.keys() == ew.keys() == {ORDER}
    assert e[ORDER]["mean"] == pytest.approx(ew[ORDER]["mean"], rel=1e-13)
    # the averaged gradient is the gradient over the union of the rows
    rng = np.random.default_rng(7)
    flat = rng.standard_normal(om.NPARAM).astype(np.float32) * 0.05
    X = rng.standard_normal((9, 64))
    t = rng.standard_normal(9)
    _, g = om.loss_and_grad(om.unpack(flat), X, t)
    ref = om.pack(g)
    for r in range(world):
        np.testing.assert_allclose(res[r][1], ref, rtol=2e-6, atol=1e-7 * np.abs(ref).max())
    assert np.array_equal(res[0][1], res[1][1])
    # benchmark timing: the slowest rank's time, all ranks' units
    assert res[0][2] == res[1][2] == 2.0
    assert res[0][3] == res[1][3] == 2 * 4 * 3 / 2.0
