"""The uneven batches at the benchmark's size and in its launch configuration
(131072 walkers, orders uniform in 4..16, one captured CUDA graph each): for the
connected sums 1024 seeded sampled walkers plus one of every order against the
oracle (minors scale perm(|A[S]|) up to order 13, the row-sum bound above,
where the permanents of every subset take minutes on the host), for the
Keldysh sums eight walkers of every order up to 12 and one of every order
above; a second replay bit for bit equal on the samples. Tolerances as in the per-path parity tests."""
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
    rng = np.random.default_rng(8)
    picks = sorted(set(one_of_each_order(orders)) | set(int(b) for b in rng.choice(131072, 1024, replace=False)))
    rows = {}
    for k in range(4, 17):
        bs = [b for b in picks if orders[b] == k]
        M = np.stack([flat[off[b]:off[b] + k * k].reshape(k, k) for b in bs])
        mref = oracle.minors_lu(M)
        ahat = (oracle.minors_scale(M) if k <= 13 else oracle.minors_rowsum_bound(M)) ** 2
        cref = oracle.cdet_recursion(mref * mref)
        scale = np.maximum(oracle.cdet_scale(ahat), 1e-300)
        for i, b in enumerate(bs):
            got = c[c_off[b]:c_off[b] + (1 << k)].cpu().numpy()
            rows[b] = got
            assert np.all(np.abs(got - cref[i]) <= TOL * scale[i]), (k, b)
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
    # eight walkers of each order up to 12, one of each order above
    picks = [int(b) for k in range(4, 17) for b in np.nonzero(orders == k)[0][:8 if k <= 12 else 1]]
    for b in picks:
        nb = int(orders[b])
        M = flat[off[b]:off[b] + 4 * nb * nb].reshape(1, 2 * nb, 2 * nb)
        ref = oracle.keldysh(M)[0]
        scale = oracle.keldysh_scale(M, use_perm=nb <= 10)[0]
        assert abs(s1[b] - ref) <= TOL * scale, nb
    s2 = g.replay().cpu().numpy()
    assert np.array_equal(s1, s2)
