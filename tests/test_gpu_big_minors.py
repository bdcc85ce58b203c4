"""All principal minors for orders 17..24 (apm_all_minors beyond the fused
kernel's own range): the upper tree levels breadth first, the 12 x 12 leaves
by the fused kernel, scaled, and the upper pivot corrections back-propagated.
Against the oracle's one elimination per minor, within 1e-10 of the row-sum
bound prod_{i in S} sum_{j in S} |A_ij| (perm(|A[S]|) costs 3^n here), and at
n = 24 on sampled masks against numpy determinants."""
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


ERROR_BITS = 2 | 4 | 8 | 16   # non-finite input, zero pivot, correction overflow, bad order


def check_full(apm, A, expect_corrected=False, tol=TOL, **kw):
    """Every minor against the oracle; no error bit; with expect_corrected the
    correction bit on every matrix (without it, a correction here and there
    among the 2^n tree nodes is allowed: it does not change the minors)."""
    m, st = apm.all_minors(dev(A), return_status=True, **kw)
    m, st = m.cpu().numpy(), st.cpu().numpy()
    ref = oracle.minors_lu(A)
    scale = oracle.minors_rowsum_bound(A)
    err = float(np.max(np.abs(m - ref) / np.maximum(scale, 1e-300)))
    assert err <= tol, err
    assert np.all(m[:, 0] == 1.0)
    assert np.all((st & ERROR_BITS) == 0), st
    if expect_corrected:
        assert np.all(st & apm.ST_PIVOT_CORRECTED), st


@pytest.mark.parametrize("n", [17, 18, 20])
def test_random_matrices_against_oracle(apm, n):
    rng = np.random.default_rng(7000 + n)
    check_full(apm, rng.standard_normal((2, n, n)) + 2.0 * np.eye(n))


def test_hubbard_matrices_n19(apm):
    check_full(apm, I.hubbard_batch(2, 19, seed=7100))


@pytest.mark.parametrize("n", [17, 19])
def test_upper_and_leaf_pivot_corrections(apm, n):
    """A zero diagonal corrects the first pivot of the upper levels and of the
    leaves; a threshold of 0.7 ||A||max corrects most of the upper ones, nested."""
    rng = np.random.default_rng(7200 + n)
    A = rng.standard_normal((2, n, n))
    for b in range(2):
        np.fill_diagonal(A[b], 0.0)
    check_full(apm, A, expect_corrected=True)
    B = rng.standard_normal((2, n, n))
    check_full(apm, B, expect_corrected=True, piv_threshold=0.7)


def small_pivot_matrices(n, deltas, seed):
    """N(0,1) + 2I matrices whose tree meets pivots of about delta ||A||max: the
    first pivot of either elimination order (A_00 and A_{n-1,n-1}), and the
    pivot of element c once element a is kept, for four pairs (a, c) in both
    orders: A_cc = A_ca A_ac / A_aa + delta ||A||max makes the 2 x 2 minor of
    {a, c} equal to A_aa delta ||A||max."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((len(deltas), n, n)) + 2 * np.eye(n)
    for b, d in enumerate(deltas):
        amax = np.abs(A[b]).max()
        A[b, 0, 0] = 1.3 * d * amax
        A[b, n - 1, n - 1] = 0.7 * d * amax
        for a, c in [(1, 3), (2, 6), (n - 2, n - 5), (n - 3, 4)]:
            A[b, c, c] = A[b, c, a] * A[b, a, c] / A[b, a, a] + d * amax * (1 + 0.1 * a)
    return A


@pytest.mark.parametrize("n", [12, 17])
def test_pivots_between_1e6_and_1e3_of_the_norm(apm, n):
    """Pivots of 1e-6 .. 1e-3 ||A||max on both sides of the default threshold
    (1e-4): the ones below are shifted, the ones above are divided by, and every
    minor stays within 1e-10 of the row-sum bound (at n = 12 also through the
    fused minors + connected-sum kernel, against the Leibniz scale)."""
    A = small_pivot_matrices(n, [1e-6, 1e-5, 1e-4, 1e-3], 7800 + n)
    check_full(apm, A)
    if n <= 16:
        c, mo = apm.cdet_connected(dev(A), return_minors=True)
        ref = oracle.minors_lu(A)
        sc = oracle.minors_scale(A)
        assert np.max(np.abs(mo.cpu().numpy() - ref) / sc) <= TOL
        cref = oracle.cdet_recursion(ref * ref)
        csc = oracle.cdet_scale(sc * sc)
        assert np.all(c.cpu().numpy()[:, 0] == 0.0)
        assert np.max(np.abs(c.cpu().numpy() - cref)[:, 1:] / csc[:, 1:]) <= TOL


def test_order_12_bench_size_sampled(apm):
    """The launch the benchmark times for the minors alone (65536 Hubbard G0
    matrices of order 12, the warp-per-matrix kernel and its redo launch):
    1024 seeded sampled matrices and the first and last against the oracle
    with the perm(|A[S]|) scale, and properties of every output (finite, the
    empty set's minor 1, every singleton's minor its diagonal entry exactly:
    its tree path drops every other element)."""
    A = I.hubbard_batch(65536, 12, seed=2)
    m, st = apm.all_minors(dev(A), return_status=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(12)
    idx = np.concatenate([[0, 65535], np.sort(rng.choice(np.arange(1, 65535), 1024, replace=False))])
    ref = oracle.minors_lu(A[idx])
    scale = oracle.minors_scale(A[idx])
    err = float(np.max(np.abs(m[idx].cpu().numpy() - ref) / np.maximum(scale, 1e-300)))
    assert err <= TOL, err
    assert int(st.cpu().numpy().max()) & ERROR_BITS == 0
    assert bool(torch.isfinite(m).all()) and bool((m[:, 0] == 1.0).all())
    diag = torch.as_tensor(np.ascontiguousarray(np.diagonal(A, axis1=1, axis2=2))).cuda()
    assert torch.equal(m[:, [1 << i for i in range(12)]], diag)


def test_order_24_sampled(apm):
    rng = np.random.default_rng(7300)
    n = 24
    A = rng.standard_normal((1, n, n)) + 2.0 * np.eye(n)
    m, st = apm.all_minors(dev(A), return_status=True)
    m = m[0].cpu().numpy()
    assert int(st.cpu()[0]) & ERROR_BITS == 0 and m.shape == (1 << n,) and m[0] == 1.0
    masks = np.concatenate([rng.integers(1, 1 << n, 3000), [(1 << n) - 1, 1 << 23, (1 << 12) - 1, 1 << 12]])
    absA = np.abs(A[0])
    for S in masks:
        idx = [i for i in range(n) if S >> i & 1]
        sub = A[0][np.ix_(idx, idx)]
        bound = np.prod(absA[np.ix_(idx, idx)].sum(axis=1))
        assert abs(m[S] - np.linalg.det(sub)) <= TOL * bound, S


def test_leading_block_matches_order_16_path(apm):
    """Masks within the first 16 elements are the minors of the leading 16 x 16
    block, which the fused kernel computes directly."""
    rng = np.random.default_rng(7400)
    A = rng.standard_normal((2, 18, 18)) + 2.0 * np.eye(18)
    big = apm.all_minors(dev(A)).cpu().numpy()[:, :1 << 16]
    small = apm.all_minors(dev(A[:, :16, :16])).cpu().numpy()
    scale = oracle.minors_rowsum_bound(A[:, :16, :16])
    assert np.all(np.abs(big - small) <= 2 * TOL * scale)


def test_nonfinite_input_and_workspace_query(apm):
    rng = np.random.default_rng(7500)
    A = rng.standard_normal((3, 17, 17)) + 2.0 * np.eye(17)
    A[1, 3, 5] = np.inf
    m, st = apm.all_minors(dev(A), return_status=True)
    st = st.cpu().numpy()
    # a corrected pivot (APM_ST_PIVOT_CORRECTED) is no error; which pivots come
    # out small depends on the tree's elimination order
    assert st[1] & apm.ST_NONFINITE_INPUT and st[0] & ERROR_BITS == 0 and st[2] & ERROR_BITS == 0
    assert bool(torch.isnan(m[1]).all()) and bool(torch.isfinite(m[0]).all())
    assert apm.workspace_size(apm.OP_ALL_MINORS, 24, 4) > apm.workspace_size(apm.OP_ALL_MINORS, 17, 4) > 0
    with pytest.raises(apm.ApmError):
        apm.all_minors(dev(rng.standard_normal((1, 25, 25))))


@pytest.mark.parametrize("n", [9, 10, 12, 13, 16])
def test_warp_minors_path(apm, n):
    """Orders 9..16 (one warp per matrix), random and Hubbard matrices."""
    rng = np.random.default_rng(7600 + n)
    check_full(apm, rng.standard_normal((5, n, n)) + 2.0 * np.eye(n))
    check_full(apm, I.hubbard_batch(3, n, seed=7650 + n))


@pytest.mark.parametrize("n", [10, 11, 12])
def test_warp_path_nested_corrections(apm, n):
    """A threshold of 0.7 ||A||max shifts most pivots of the tail, nested in
    the lanes' subtrees and across the breadth-first levels (the warp kernel's
    correcting pass). Orders above 12 are left out: there most pivots of the
    depth-first part are shifted too, which sends the matrix to the fused
    kernel, whose record of up to 256 corrections such a threshold overflows
    (NaN and APM_ST_CORRECTION_OVERFLOW by design)."""
    rng = np.random.default_rng(7300 + n)
    check_full(apm, rng.standard_normal((3, n, n)), expect_corrected=True, piv_threshold=0.7)


@pytest.mark.parametrize("n", [9, 10, 11, 12, 14])
def test_warp_path_redo_and_nonfinite(apm, n):
    """In one batch: plain matrices (the warp kernel's fast pass), matrices
    with a zero diagonal entry (a zero pivot of the tail, flagged by the fast
    pass and corrected by the warp kernel's correcting pass; at n = 14 the zero
    of element n-1 is a pivot of the depth-first part above the tail, which
    sends the matrix on to the fused kernel, whose own pivots are corrected
    where small) and a non-finite one (flagged by the fused kernel, as in
    apm_cdet_connected)."""
    rng = np.random.default_rng(7700 + n)
    A = rng.standard_normal((6, n, n)) + 2.0 * np.eye(n)
    A[1, n - 1, n - 1] = 0.0          # the first pivot of the tree
    A[3, 2, 2] = 0.0                  # a pivot of the tail
    A[4] = rng.standard_normal((n, n))
    np.fill_diagonal(A[4], 0.0)
    ok = [0, 1, 2, 3, 4]
    check_full(apm, A[ok])
    A[5, 0, 1] = np.nan
    m, st = apm.all_minors(dev(A), return_status=True)
    m, st = m.cpu().numpy(), st.cpu().numpy()
    assert st[4] & apm.ST_PIVOT_CORRECTED and np.all(st[:5] & ERROR_BITS == 0)
    assert st[5] & apm.ST_NONFINITE_INPUT and np.isnan(m[5, -1])   # flagged; NaN where the entry enters
    ref = oracle.minors_lu(A[ok])
    assert np.all(np.abs(m[ok] - ref) <= TOL * oracle.minors_rowsum_bound(A[ok]))
