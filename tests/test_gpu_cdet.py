"""Parity of the CUDA minors / connected-sum path with the CPU oracle.

Tolerance: |gpu - oracle| <= 1e-10
times the sum of the absolute values of the terms: perm(|A[S]|) for a minor,
and for c[S] the recursion run on those scales with all signs positive.
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
    return m


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def scaled_err(got, ref, scale):
    got, ref = np.asarray(got), np.asarray(ref)
    return float(np.max(np.abs(got - ref) / np.maximum(scale, 1e-300)))


def check_minors(apm, A, tol=TOL, expect_corrected=None):
    m, st = apm.all_minors(dev(A), return_status=True)
    m = m.cpu().numpy()
    ref = oracle.minors_lu(A)
    scale = oracle.minors_scale(A)
    err = scaled_err(m, ref, scale)
    assert err <= tol, err
    assert np.all(m[:, 0] == 1.0)
    st = st.cpu().numpy()
    assert np.all((st & ~apm.ST_PIVOT_CORRECTED) == 0), st
    if expect_corrected is not None:
        assert bool(np.all(st & apm.ST_PIVOT_CORRECTED)) == expect_corrected
    return m, scale


def check_cdet(apm, A, single_det=False, tol=TOL):
    c, mo = apm.cdet_connected(dev(A), single_det=single_det, return_minors=True)
    c, mo = c.cpu().numpy(), mo.cpu().numpy()
    mref = oracle.minors_lu(A)
    mscale = oracle.minors_scale(A)
    assert scaled_err(mo, mref, mscale) <= tol
    a = mref if single_det else mref * mref
    ahat = mscale if single_det else mscale * mscale
    cref = oracle.cdet_recursion(a)
    cscale = oracle.cdet_scale(ahat)
    err = scaled_err(c, cref, cscale)
    assert err <= tol, err
    assert np.all(c[:, 0] == 0.0)
    return c


def test_cfg_single_n10_gaussian(apm):
    A = I.gaussian_plus_2I(10, 1, seed=1)
    check_minors(apm, A)
    check_cdet(apm, A)
    check_cdet(apm, A, single_det=True)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 9, 11, 12, 13])
def test_orders_random(apm, n):
    rng = np.random.default_rng(100 + n)
    A = rng.standard_normal((5, n, n)) + 1.5 * np.eye(n)
    check_minors(apm, A)
    check_cdet(apm, A)


def test_order_14_global_scratch_variant(apm):
    rng = np.random.default_rng(114)
    A = rng.standard_normal((2, 14, 14)) + 2.0 * np.eye(14)
    check_minors(apm, A)
    check_cdet(apm, A)


@pytest.mark.parametrize("n", [15, 16])
def test_orders_15_16_hubbard(apm, n):
    """The largest orders: the blocked recursion (n = 15) and the fast subset
    convolution that apm_cdet_connected takes at n = 16, for det^2, det and
    two-matrix weights."""
    A = I.hubbard_batch(2, n, seed=600 + n)
    check_minors(apm, A)
    check_cdet(apm, A)
    check_cdet(apm, A, single_det=True)
    B = I.hubbard_batch(2, n, seed=650 + n)
    c = apm.cdet_connected(dev(A), dev(B)).cpu().numpy()
    mu, md = oracle.minors_lu(A), oracle.minors_lu(B)
    su, sd = oracle.minors_scale(A), oracle.minors_scale(B)
    err = scaled_err(c, oracle.cdet_recursion(mu * md), oracle.cdet_scale(su * sd))
    assert err <= TOL, err


@pytest.mark.parametrize("n", [6, 10, 12])
def test_zero_diagonal_forces_pivot_correction(apm, n):
    rng = np.random.default_rng(200 + n)
    A = rng.standard_normal((3, n, n))
    for b in range(3):
        np.fill_diagonal(A[b], 0.0)
    check_minors(apm, A, expect_corrected=True)
    check_cdet(apm, A)


def test_rank_one_and_zero_matrix(apm):
    rng = np.random.default_rng(300)
    n = 10
    u, v = rng.standard_normal((2, n)), rng.standard_normal((2, n))
    R = np.einsum("bi,bj->bij", u, v)
    m, scale = check_minors(apm, R, expect_corrected=True)
    Z = np.zeros((2, n, n))
    mz = apm.all_minors(dev(Z)).cpu().numpy()
    ref = np.zeros((2, 1 << n))
    ref[:, 0] = 1.0
    assert np.array_equal(mz, ref)
    cz = apm.cdet_connected(dev(Z)).cpu().numpy()
    assert np.array_equal(cz, np.zeros_like(cz))


def test_diagonal_and_triangular_products(apm):
    rng = np.random.default_rng(301)
    n = 11
    d = rng.uniform(0.5, 2.0, n) * rng.choice([-1, 1], n)
    U = np.triu(rng.standard_normal((n, n)), 1) + np.diag(d)
    masks = np.arange(1 << n)
    prods = np.array([np.prod(d[[e for e in range(n) if (S >> e) & 1]]) for S in masks])
    for A in (np.diag(d), U, U.T.copy()):
        m = apm.all_minors(dev(A[None])).cpu().numpy()[0]
        np.testing.assert_allclose(m, prods, rtol=1e-13, atol=0)


def test_two_matrices(apm):
    rng = np.random.default_rng(400)
    n = 9
    Au = rng.standard_normal((4, n, n)) + 2 * np.eye(n)
    Ad = rng.standard_normal((4, n, n)) + 2 * np.eye(n)
    c, mo = apm.cdet_connected(dev(Au), dev(Ad), return_minors=True)
    mu, md = oracle.minors_lu(Au), oracle.minors_lu(Ad)
    su, sd = oracle.minors_scale(Au), oracle.minors_scale(Ad)
    mo = mo.cpu().numpy()
    assert scaled_err(mo[:, 0], mu, su) <= TOL and scaled_err(mo[:, 1], md, sd) <= TOL
    err = scaled_err(c.cpu().numpy(), oracle.cdet_recursion(mu * md), oracle.cdet_scale(su * sd))
    assert err <= TOL, err


@pytest.mark.parametrize("n", [3, 8, 12, 13, 14])
def test_cdet_from_weights(apm, n):
    rng = np.random.default_rng(500 + n)
    a = rng.standard_normal((3, 1 << n))
    c = apm.cdet_from_weights(dev(a)).cpu().numpy()
    a[:, 0] = 1.0
    err = scaled_err(c, oracle.cdet_recursion(a), oracle.cdet_scale(np.abs(a)))
    assert err <= TOL, err


def test_nonfinite_input_flagged(apm):
    A = I.gaussian_plus_2I(8, 3, seed=9)
    A[1, 2, 3] = np.nan
    m, st = apm.all_minors(dev(A), return_status=True)
    st = st.cpu().numpy()
    assert st[1] & apm.ST_NONFINITE_INPUT and not (st[0] & apm.ST_NONFINITE_INPUT)
    code, bits = apm.status_reduce(st_t := torch.as_tensor(st).cuda())
    assert code == apm.APM_ERR_NUMERIC and bits & apm.ST_NONFINITE_INPUT


def test_empty_batch_and_bad_args(apm):
    A = torch.zeros((0, 8, 8), dtype=torch.float64, device="cuda")
    assert apm.all_minors(A).shape == (0, 256)
    with pytest.raises(apm.ApmError):
        apm.all_minors(torch.zeros((1, 25, 25), dtype=torch.float64, device="cuda"))


def test_hubbard_n12_full_batch_sampled(apm):
    """The benchmark's workload (65536 Hubbard G0 matrices, n=12) in the same
    launch configuration; 1024 seeded sampled matrices (and the first and last)
    against the oracle with the perm(|A[S]|) scale, plus properties of every
    output."""
    A = I.hubbard_batch(65536, 12, seed=2)
    c, mo, st = apm.cdet_connected(dev(A), return_minors=True, return_status=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    idx = np.sort(rng.choice(np.arange(1, 65535), 1024, replace=False))
    idx = np.concatenate([[0, 65535], idx])
    sub = A[idx]
    mref = oracle.minors_lu(sub)
    mscale = oracle.minors_scale(sub)
    assert scaled_err(mo[idx].cpu().numpy(), mref, mscale) <= TOL
    cref = oracle.cdet_recursion(mref * mref)
    cscale = oracle.cdet_scale(mscale * mscale)
    assert scaled_err(c[idx].cpu().numpy(), cref, cscale) <= TOL
    st = st.cpu().numpy()
    assert np.all((st & ~1) == 0)
    assert torch.isfinite(c).all() and torch.isfinite(mo).all()
    assert bool((mo[:, 0] == 1).all()) and bool((c[:, 0] == 0).all())
    # singletons: c[{i}] = a[{i}] = G0(0,0^-)^2 on every matrix
    single = c[:, [1 << i for i in range(12)]]
    assert torch.allclose(single, mo[:, [1 << i for i in range(12)]] ** 2, rtol=0, atol=0)


def test_deterministic(apm):
    A = dev(I.hubbard_batch(512, 12, seed=11))
    c1 = apm.cdet_connected(A)
    c2 = apm.cdet_connected(A)
    assert torch.equal(c1, c2)
