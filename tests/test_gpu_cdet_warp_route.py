"""Connected sums at orders 13..16 of one matrix per item: the minors come from
the warp-per-matrix tree, the fused kernel forms the weights from them and
computes the tree itself (with the pivot correction of Section II) only for the
matrices that tree flagged. Checked against the CPU oracle within 1e-10 of the
sum of absolute terms, on batches that mix plain matrices with flagged ones
(zero diagonal: every leading pivot vanishes; a non-finite entry), for the fixed
and the uneven-batch launches, with and without the minors requested.
"""
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


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def scaled_err(got, ref, scale):
    return float(np.max(np.abs(np.asarray(got) - ref) / np.maximum(scale, 1e-300)))


def mixed_batch(n, seed):
    """[plain N(0,1) + 2I, zero diagonal, Hubbard G0, non-finite entry, plain]."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((5, n, n))
    A[0] += 2.0 * np.eye(n)
    np.fill_diagonal(A[1], 0.0)
    A[2] = I.hubbard_batch(1, n, seed=seed)[0]
    A[3] += 2.0 * np.eye(n)
    A[3, n - 2, 1] = np.inf
    A[4] += 2.0 * np.eye(n)
    return A


@pytest.mark.parametrize("n", [13, 14])
def test_fixed_order_mixed_flags_against_oracle(apm, n):
    A = mixed_batch(n, 1700 + n)
    c, mo, st = apm.cdet_connected(dev(A), return_minors=True, return_status=True)
    c, mo, st = c.cpu().numpy(), mo.cpu().numpy(), st.cpu().numpy()
    good = [0, 1, 2, 4]
    sub = A[good]
    mref = oracle.minors_lu(sub)
    mscale = oracle.minors_scale(sub)
    assert scaled_err(mo[good], mref, mscale) <= TOL
    cref = oracle.cdet_recursion(mref * mref)
    cscale = oracle.cdet_scale(mscale * mscale)
    assert scaled_err(c[good], cref, cscale) <= TOL
    # the Hubbard matrix meets no small pivot; the random ones may (corrected by
    # the fused kernel), but none has an error bit
    assert st[2] == 0 and np.all(st[[0, 4]] & ~apm.ST_PIVOT_CORRECTED == 0), st
    assert st[1] & apm.ST_PIVOT_CORRECTED, st
    assert st[3] & apm.ST_NONFINITE_INPUT, st
    assert not np.isfinite(c[3]).all()
    # without the minors requested they go through the output row first:
    # the connected sums are the same, bit for bit
    c2, st2 = apm.cdet_connected(dev(A), return_status=True)
    assert np.array_equal(c2.cpu().numpy(), c, equal_nan=True)
    assert np.array_equal(st2.cpu().numpy(), st)


def test_fixed_order_single_det_and_order_16(apm):
    """det weights at order 13, and order 16 (the fast subset convolution after
    the warp minors) on a Hubbard matrix (no small pivot: its minors are the warp
    kernel's) and a zero-diagonal one (recomputed with the correction)."""
    A = mixed_batch(13, 1750)[[0, 1]]
    c, mo = apm.cdet_connected(dev(A), single_det=True, return_minors=True)
    mref = oracle.minors_lu(A)
    mscale = oracle.minors_scale(A)
    assert scaled_err(mo.cpu().numpy(), mref, mscale) <= TOL
    err = scaled_err(c.cpu().numpy(), oracle.cdet_recursion(mref), oracle.cdet_scale(mscale))
    assert err <= TOL, err
    rng = np.random.default_rng(1751)
    B = rng.standard_normal((2, 16, 16))
    B[0] = I.hubbard_batch(1, 16, seed=1752)[0]
    np.fill_diagonal(B[1], 0.0)
    c, mo, st = apm.cdet_connected(dev(B), return_minors=True, return_status=True)
    st = st.cpu().numpy()
    assert st[0] == 0 and st[1] & apm.ST_PIVOT_CORRECTED, st
    mref = oracle.minors_lu(B)
    ms = oracle.minors_scale(B)
    assert scaled_err(mo.cpu().numpy(), mref, ms) <= TOL
    err = scaled_err(c.cpu().numpy(), oracle.cdet_recursion(mref * mref), oracle.cdet_scale(ms * ms))
    assert err <= TOL, err


def test_uneven_batch_with_flagged_items_equals_fixed(apm):
    """Orders 9..14 mixed, with zero-diagonal and non-finite matrices among the
    orders 13 and 14: the uneven launch equals the fixed-order launches bit for
    bit (connected sums, minors, status)."""
    rng = np.random.default_rng(1760)
    orders = np.array([13, 9, 14, 13, 12, 14, 13, 10, 14, 11], dtype=np.int32)
    mats = []
    for k, n in enumerate(orders):
        M = rng.standard_normal((n, n)) + 2.0 * np.eye(n)
        if k in (2, 3):
            np.fill_diagonal(M, 0.0)
        if k == 6:
            M[0, n - 1] = np.nan
        mats.append(M)
    flat = np.concatenate([M.ravel() for M in mats])
    a_off = np.concatenate([[0], np.cumsum([n * n for n in orders])[:-1]]).astype(np.int64)
    A, ao, nt = dev(flat), dev(a_off), dev(orders)
    c, mo, st = apm.cdet_connected_varlen(A, ao, nt, return_minors=True, return_status=True)
    c_off = apm.varlen_out_offsets(nt).cpu().numpy()
    c, mo, st = c.cpu().numpy(), mo.cpu().numpy(), st.cpu().numpy()
    # without the minors requested (they pass through the connected-sum rows)
    c2, st2 = apm.cdet_connected_varlen(A, ao, nt, return_status=True)
    assert np.array_equal(c2.cpu().numpy(), c, equal_nan=True)
    assert np.array_equal(st2.cpu().numpy(), st)
    assert st[2] & apm.ST_PIVOT_CORRECTED and st[3] & apm.ST_PIVOT_CORRECTED, st
    assert st[6] & apm.ST_NONFINITE_INPUT, st
    for n in np.unique(orders):
        idx = np.nonzero(orders == n)[0]
        cf, mf, sf = apm.cdet_connected(dev(np.stack([mats[b] for b in idx])), return_minors=True,
                                        return_status=True)
        cf, mf, sf = cf.cpu().numpy(), mf.cpu().numpy(), sf.cpu().numpy()
        for k, b in enumerate(idx):
            N = 1 << int(n)
            assert np.array_equal(c[c_off[b]:c_off[b] + N], cf[k], equal_nan=True), (b, n)
            assert np.array_equal(mo[c_off[b]:c_off[b] + N], mf[k], equal_nan=True), (b, n)
            assert st[b] == sf[k], (b, st[b], sf[k])
    # the zero-diagonal order-14 item against the oracle
    b = 2
    mref = oracle.minors_lu(mats[b][None])
    ms = oracle.minors_scale(mats[b][None])
    N = 1 << 14
    assert scaled_err(mo[None, c_off[b]:c_off[b] + N], mref, ms) <= TOL
    cref = oracle.cdet_recursion(mref * mref)
    assert scaled_err(c[None, c_off[b]:c_off[b] + N], cref, oracle.cdet_scale(ms * ms)) <= TOL
