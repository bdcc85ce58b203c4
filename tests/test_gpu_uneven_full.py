"""The uneven batches at the benchmark's size and in its launch configuration
(131072 walkers, orders uniform in 4..16, one captured CUDA graph each): one
sampled walker of every order against the oracle, and a second replay bit for
bit equal on the samples. Tolerances as in the per-path parity tests."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_07638_gb300 import inputs as I

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def apm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_07638_gb300 import apm as m
    m.lib()
    m.tune_set(None)
    return m


def one_of_each_order(orders):
    return [int(np.nonzero(orders == k)[0][0]) for k in range(4, 17)]


def test_cdet_uneven_bench_size_sampled(apm):
    from paper_2104_07638_gb300.batch import CdetVarlenGraph
    orders = I.varlen_orders(131072, 4, 16, seed=3)
    flat, off = I.hubbard_varlen(orders, seed=3)
    g = CdetVarlenGraph(torch.as_tensor(flat).cuda(), torch.as_tensor(off).cuda(), torch.as_tensor(orders).cuda())
    c = g.replay()
    c_off = g.c_off.cpu().numpy()
    picks = one_of_each_order(orders)
    rows = {}
    for b in picks:
        nb = int(orders[b])
        got = c[c_off[b]:c_off[b] + (1 << nb)].cpu().numpy()
        rows[b] = got
        M = flat[off[b]:off[b] + nb * nb].reshape(1, nb, nb)
        mref = oracle.minors_lu(M)
        ahat = (oracle.minors_scale(M) if nb <= 10 else oracle.minors_rowsum_bound(M)) ** 2
        cref = oracle.cdet_recursion(mref * mref)[0]
        scale = np.maximum(oracle.cdet_scale(ahat)[0], 1e-300)
        assert np.all(np.abs(got - cref) <= TOL * scale), nb
    c = g.replay()
    for b in picks:
        nb = int(orders[b])
        assert np.array_equal(c[c_off[b]:c_off[b] + (1 << nb)].cpu().numpy(), rows[b])


def test_keldysh_uneven_bench_size_sampled(apm):
    from paper_2104_07638_gb300.batch import KeldyshVarlenGraph
    orders = I.varlen_orders(131072, 4, 16, seed=3)
    flat, off = I.keldysh_varlen(orders, seed=3)
    g = KeldyshVarlenGraph(torch.as_tensor(flat).cuda(), torch.as_tensor(off).cuda(),
                           torch.as_tensor(orders).cuda())
    s1 = g.replay().cpu().numpy()
    picks = [b for b in one_of_each_order(orders) if orders[b] in (4, 7, 10, 12, 16)]
    for b in picks:
        nb = int(orders[b])
        M = flat[off[b]:off[b] + 4 * nb * nb].reshape(1, 2 * nb, 2 * nb)
        ref = oracle.keldysh(M)[0]
        scale = oracle.keldysh_scale(M, use_perm=nb <= 10)[0]
        assert abs(s1[b] - ref) <= TOL * scale, nb
    s2 = g.replay().cpu().numpy()
    assert np.array_equal(s1, s2)
