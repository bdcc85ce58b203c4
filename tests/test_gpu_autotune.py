"""The autotuner of the uneven batches (no counterpart in the paper): run on
two orders of the recursion and on the hand-off to the fast subset
convolution, it must choose mappings no slower than the defaults, and under
whatever it installs the uneven batch must stay bit for bit equal to
fixed-order launches of the same matrices and within the parity tolerance of
the oracle. Other hand-off orders and launch shapes keep the same agreement."""
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
    yield m
    m.tune_set(None)
    m.tune_options_set(0, 0, 0)


def packed(orders, seed):
    flat, off = I.hubbard_varlen(orders, seed=seed)
    return (torch.as_tensor(flat).cuda(), torch.as_tensor(off).cuda(),
            torch.as_tensor(np.asarray(orders, dtype=np.int32)).cuda(), flat, off)


def check_against_fixed(apm, orders, seed):
    A, a_off, n, flat, off = packed(orders, seed)
    c, st = apm.cdet_connected_varlen(A, a_off, n, return_status=True)
    c_off = apm.varlen_out_offsets(n).cpu().numpy()
    c = c.cpu().numpy()
    assert int(st.cpu().numpy().max() & ~apm.ST_PIVOT_CORRECTED) == 0
    for m in np.unique(orders):
        idx = np.nonzero(orders == m)[0]
        Am = np.stack([flat[off[b]:off[b] + m * m].reshape(m, m) for b in idx])
        ref = apm.cdet_connected(torch.as_tensor(Am).cuda()).cpu().numpy()
        for k, b in enumerate(idx):
            assert np.array_equal(c[c_off[b]:c_off[b] + (1 << int(m))], ref[k]), (b, m)
    return c, c_off, flat, off


def test_autotune_no_slower_and_bitwise_agreement(apm):
    from paper_2104_07638_gb300 import batch
    tuned = batch.autotune(orders=(9, 12), fsc_orders=(15, 16), reps=3, use_cache=False, tune_launch=True)
    for n in (9, 12):
        t = tuned["timings"][f"lane_groups_n{n}"]
        assert t["tuned_ms"] <= t["default_ms"]           # kept only when faster
    for n in (15, 16):
        t = tuned["timings"][f"fsc_n{n}"]
        chose_fsc = tuned["fsc_from_n"] <= n
        assert (t["fsc_ms"] <= t["recursion_ms"]) if chose_fsc else True
    assert tuned["fsc_from_n"] in (15, 16, 17)
    assert tuned["cdet_ctas_per_sm"] in (2, 3) and tuned["keldysh_warps"] in (4, 6, 8, 10, 12)
    assert apm.tune_options_get() == (tuned["fsc_from_n"], tuned["cdet_ctas_per_sm"], tuned["keldysh_warps"])
    orders = np.array([9, 12, 12, 15, 16, 9, 14, 12], dtype=np.int32)
    c, c_off, flat, off = check_against_fixed(apm, orders, seed=1500)
    b, m = 1, 12
    Ab = flat[off[b]:off[b] + m * m].reshape(m, m)
    mref = oracle.minors_lu(Ab)
    cs = oracle.cdet_scale(oracle.minors_scale(Ab) ** 2)
    assert np.all(np.abs(c[c_off[b]:c_off[b] + 4096] - oracle.cdet_recursion(mref * mref))
                  <= TOL * np.maximum(cs, 1e-300))


@pytest.mark.parametrize("fsc_from,ctas", [(13, 2), (15, 3), (17, 1)])
def test_hand_off_orders_and_launch_shapes(apm, fsc_from, ctas):
    """Every hand-off order: fixed-order and uneven launches agree bit for bit,
    and the order-13..16 rows match the oracle within tolerance."""
    apm.tune_options_set(fsc_from, ctas, 6)
    try:
        orders = np.array([13, 16, 14, 15, 13, 12, 7], dtype=np.int32)
        c, c_off, flat, off = check_against_fixed(apm, orders, seed=1510 + fsc_from)
        for b in (0, 1):
            m = int(orders[b])
            M = flat[off[b]:off[b] + m * m].reshape(1, m, m)
            mref = oracle.minors_lu(M)
            cref = oracle.cdet_recursion(mref * mref)[0]
            cs = oracle.cdet_scale(oracle.minors_rowsum_bound(M) ** 2)[0]
            assert np.all(np.abs(c[c_off[b]:c_off[b] + (1 << m)] - cref) <= TOL * np.maximum(cs, 1e-300))
        # the Keldysh uneven batch with 6 warps per CTA against its default launch
        korders = np.array([4, 9, 12, 14, 16, 10], dtype=np.int32)
        kflat, koff = I.keldysh_varlen(korders, seed=1520)
        Mt = torch.as_tensor(kflat).cuda()
        m_off = torch.as_tensor(koff).cuda()
        nk = torch.as_tensor(korders).cuda()
        s6 = apm.keldysh_sum_varlen(Mt, m_off, nk).cpu().numpy()
        apm.tune_options_set(fsc_from, ctas, 0)
        s12 = apm.keldysh_sum_varlen(Mt, m_off, nk).cpu().numpy()
        assert np.array_equal(s6, s12)
    finally:
        apm.tune_options_set(0, 0, 0)


def test_options_out_of_range_are_rejected(apm):
    before = apm.tune_options_get()
    for args in ((12, 0, 0), (18, 0, 0), (16, 4, 0), (16, 0, 3), (16, 0, 13), (16, -1, 0)):
        with pytest.raises(apm.ApmError):
            apm.tune_options_set(*args)
    assert apm.tune_options_get() == before
