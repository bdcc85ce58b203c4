"""Uneven batches (one persistent longest-first launch, CUDA-graph capture,
tuned lane mappings): outputs must be bit-identical to the fixed-order
launches of the same matrices (same per-matrix code path) and within the
parity tolerance of the oracle."""
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


def packed_hubbard(orders, seed):
    flat, off = I.hubbard_varlen(orders, seed=seed)
    return (torch.as_tensor(flat).cuda(), torch.as_tensor(off).cuda(),
            torch.as_tensor(np.asarray(orders, dtype=np.int32)).cuda(), flat, off)


def fixed_reference(apm, flat, off, orders, minors=False):
    """Per-order fixed launches of the same matrices, scattered back to packed rows."""
    orders = np.asarray(orders)
    out_c, out_m = {}, {}
    for n in np.unique(orders):
        idx = np.nonzero(orders == n)[0]
        A = np.stack([flat[off[b]:off[b] + n * n].reshape(n, n) for b in idx])
        c, m = apm.cdet_connected(torch.as_tensor(A).cuda(), return_minors=True)
        for k, b in enumerate(idx):
            out_c[b] = c[k].cpu().numpy()
            out_m[b] = m[k].cpu().numpy()
    return out_c, out_m


def test_varlen_bitwise_equals_fixed_and_oracle(apm):
    rng = np.random.default_rng(1300)
    orders = np.concatenate([np.arange(1, 17), rng.integers(4, 17, 200)]).astype(np.int32)
    rng.shuffle(orders)
    A, a_off, n, flat, off = packed_hubbard(orders, seed=1301)
    c, mo, st = apm.cdet_connected_varlen(A, a_off, n, return_minors=True, return_status=True)
    c_off = apm.varlen_out_offsets(n).cpu().numpy()
    c, mo = c.cpu().numpy(), mo.cpu().numpy()
    assert int(st.cpu().numpy().max() & ~apm.ST_PIVOT_CORRECTED) == 0
    ref_c, ref_m = fixed_reference(apm, flat, off, orders)
    for b, nb in enumerate(orders):
        N = 1 << int(nb)
        assert np.array_equal(c[c_off[b]:c_off[b] + N], ref_c[b]), (b, nb)
        assert np.array_equal(mo[c_off[b]:c_off[b] + N], ref_m[b]), (b, nb)
    # oracle on a sample of the small and mid orders
    for b in [i for i, nb in enumerate(orders) if nb <= 12][:12]:
        nb = int(orders[b])
        Ab = flat[off[b]:off[b] + nb * nb].reshape(nb, nb)
        mref = oracle.minors_lu(Ab)
        ms = oracle.minors_scale(Ab)
        cref = oracle.cdet_recursion(mref * mref)
        cs = oracle.cdet_scale(ms * ms)
        N = 1 << nb
        assert np.all(np.abs(mo[c_off[b]:c_off[b] + N] - mref) <= TOL * ms)
        assert np.all(np.abs(c[c_off[b]:c_off[b] + N] - cref) <= TOL * np.maximum(cs, 1e-300))


def test_bad_order_is_flagged_not_faulting(apm):
    orders = np.array([5, 6, 7], dtype=np.int32)
    A, a_off, n, flat, off = packed_hubbard(orders, seed=1302)
    n_bad = n.clone()
    n_bad[1] = 9                      # larger than the n_max passed below
    c_off = apm.varlen_out_offsets(n)
    c, st = apm.cdet_connected_varlen(A, a_off, n_bad, n_max=7, c_off=c_off, return_status=True)
    st = st.cpu().numpy()
    assert st[1] & apm.ST_BAD_ORDER and not (st[0] & apm.ST_BAD_ORDER) and not (st[2] & apm.ST_BAD_ORDER)


def test_graph_replay_matches_direct_call(apm):
    from paper_2104_07638_gb300.batch import CdetVarlenGraph
    orders = I.varlen_orders(600, 4, 13, seed=1303)
    A, a_off, n, flat, off = packed_hubbard(orders, seed=1304)
    g = CdetVarlenGraph(A, a_off, n)
    direct = apm.cdet_connected_varlen(A, a_off, n)
    c1 = g.replay().clone()
    assert torch.equal(c1, direct)
    A2, _, _, _, _ = packed_hubbard(orders, seed=1305)
    A.copy_(A2)                       # new inputs in place, same shapes
    c2 = g.replay().clone()
    assert torch.equal(c2, apm.cdet_connected_varlen(A, a_off, n))
    assert not torch.equal(c1, c2)


def test_graph_replay_with_order_16(apm):
    """Orders up to 16: the captured graph holds the sort, the persistent kernel
    and the fast subset convolution of the order-16 rows."""
    from paper_2104_07638_gb300.batch import CdetVarlenGraph
    orders = np.concatenate([[16, 16, 16], I.varlen_orders(200, 4, 15, seed=1306)]).astype(np.int32)
    A, a_off, n, flat, off = packed_hubbard(orders, seed=1307)
    g = CdetVarlenGraph(A, a_off, n)
    direct = apm.cdet_connected_varlen(A, a_off, n)
    assert torch.equal(g.replay().clone(), direct)
    c_off = apm.varlen_out_offsets(n).cpu().numpy()
    c = direct.cpu().numpy()
    for b in range(3):                # the order-16 rows against the oracle
        M = flat[off[b]:off[b] + 256].reshape(1, 16, 16)
        mref = oracle.minors_lu(M)
        bound = oracle.minors_rowsum_bound(M) ** 2
        cref = oracle.cdet_recursion(mref * mref)[0]
        scale = np.maximum(oracle.cdet_scale(bound)[0], 1e-300)
        assert np.all(np.abs(c[c_off[b]:c_off[b] + (1 << 16)] - cref) <= TOL * scale)


def test_tuned_tables_keep_bitwise_agreement(apm):
    from paper_2104_07638_gb300.batch import _shift_table
    table = [_shift_table(apm.tune_get(m), m, -1) for m in range(17)]
    apm.tune_set(table)
    try:
        orders = np.array([6, 9, 12, 12, 10, 11], dtype=np.int32)
        A, a_off, n, flat, off = packed_hubbard(orders, seed=1306)
        c = apm.cdet_connected_varlen(A, a_off, n).cpu().numpy()
        c_off = apm.varlen_out_offsets(n).cpu().numpy()
        ref_c, _ = fixed_reference(apm, flat, off, orders)
        for b, nb in enumerate(orders):
            assert np.array_equal(c[c_off[b]:c_off[b] + (1 << int(nb))], ref_c[b])
        nb = 12
        b = 2
        Ab = flat[off[b]:off[b] + nb * nb].reshape(nb, nb)
        mref = oracle.minors_lu(Ab)
        cs = oracle.cdet_scale(oracle.minors_scale(Ab) ** 2)
        assert np.all(np.abs(c[c_off[b]:c_off[b] + 4096] - oracle.cdet_recursion(mref * mref))
                      <= TOL * np.maximum(cs, 1e-300))
    finally:
        apm.tune_set(None)


def test_keldysh_varlen_bitwise_equals_fixed(apm):
    """The uneven-batch kernel walks each matrix like a fixed-order launch of
    whole matrices: bit-identical results. A fixed-order launch of one matrix of
    order >= 10 splits it over warps (chunks added in a fixed order), which only
    changes rounding: those are compared within the parity tolerance."""
    orders = np.array([1, 2, 5, 6, 7, 9, 12, 14, 16, 3, 8, 11], dtype=np.int32)
    flat, off = I.keldysh_varlen(orders, seed=1307)
    Mt = torch.as_tensor(flat).cuda()
    m_off = torch.as_tensor(off).cuda()
    n = torch.as_tensor(orders).cuda()
    s, p = apm.keldysh_sum_varlen(Mt, m_off, n, partial=True)
    s, p = s.cpu().numpy(), p.cpu().numpy()
    for b, nb in enumerate(orders):
        nb = int(nb)
        M = flat[off[b]:off[b] + 4 * nb * nb].reshape(1, 2 * nb, 2 * nb)
        sf, pf = apm.keldysh_sum(torch.as_tensor(M).cuda(), partial=True)
        if nb <= 9:
            assert s[b] == sf.cpu().numpy()[0]
            assert np.array_equal(p[b, :nb + 1], pf.cpu().numpy()[0])
        else:
            scale = oracle.keldysh_scale(M, use_perm=False)[0]
            assert abs(s[b] - sf.cpu().numpy()[0]) <= TOL * scale
            assert np.all(np.abs(p[b, :nb + 1] - pf.cpu().numpy()[0]) <= TOL * scale)
        if nb <= 9:
            assert abs(s[b] - oracle.keldysh(M)[0]) <= TOL * oracle.keldysh_scale(M)[0]


def test_keldysh_graph(apm):
    from paper_2104_07638_gb300.batch import KeldyshVarlenGraph
    orders = I.varlen_orders(300, 4, 12, seed=1308)
    flat, off = I.keldysh_varlen(orders, seed=1309)
    Mt = torch.as_tensor(flat).cuda()
    m_off = torch.as_tensor(off).cuda()
    n = torch.as_tensor(orders).cuda()
    g = KeldyshVarlenGraph(Mt, m_off, n)
    assert torch.equal(g.replay(), apm.keldysh_sum_varlen(Mt, m_off, n))
