"""Parity of the CUDA NAND minors and the two-vertex-type CDet (Sections III.C,
V.C) with the CPU oracle (one elimination per kept submatrix; the type sums
and the CDet recursion on them). Tolerance: 1e-10 times the row-sum bound of
the kept submatrices summed over the type assignments of the same vertex
subset (for a single minor this is at least its own bound); for c, the
recursion run on those scales with all signs positive."""
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


def support_of_ternary(n):
    t = np.arange(3 ** n)
    S = np.zeros_like(t)
    for v in range(n):
        S |= ((t // 3 ** v) % 3 != 0).astype(np.int64) << v
    return S


def check_minors3(apm, M):
    n = M.shape[-1] // 2
    x, st = apm.nand_minors(dev(M), return_status=True)
    x = x.cpu().numpy()
    ab, sc, m3 = oracle.nand(M, minors=True)
    scale = sc[:, support_of_ternary(n)]
    err = float(np.max(np.abs(x - m3) / scale))
    assert err <= TOL, err
    assert int((st.cpu().numpy() & ~apm.ST_PIVOT_CORRECTED).max()) == 0   # a corrected pivot is no error
    assert np.all(x[:, 0] == 1.0)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9])
def test_random_matrices_all_minors(apm, n):
    """Orders on both sides of the 6-vertex tail: breadth first only (n <= 6),
    one to three depth-first levels (n = 7..9; the stack from n = 8)."""
    rng = np.random.default_rng(4000 + n)
    M = rng.standard_normal((4, 2 * n, 2 * n)) + 1.5 * np.eye(2 * n)
    check_minors3(apm, M)


@pytest.mark.parametrize("n", [6, 8, 13])
def test_two_type_matrices_all_minors(apm, n):
    check_minors3(apm, I.two_type_batch(1 if n == 13 else 3, n, seed=4100 + n))


@pytest.mark.parametrize("n", [3, 7, 10, 14])
def test_two_type_cdet_against_oracle(apm, n):
    M = I.two_type_batch(1 if n == 14 else 3, n, seed=4200 + n)
    c, ab = apm.two_type_cdet(dev(M), return_weights=True)
    c, ab = c.cpu().numpy(), ab.cpu().numpy()
    abr, sc = oracle.nand(M)
    assert np.all(np.abs(ab - abr) <= TOL * sc)
    cr = oracle.cdet_recursion(abr)
    cs = oracle.cdet_scale(sc)
    assert np.all(np.abs(c - cr) <= TOL * np.maximum(cs, 1e-300))
    assert np.all(ab[:, 0] == 1.0) and np.all(c[:, 0] == 0.0)


def test_order_16_equal_types_closed_form(apm):
    """Both types of every vertex identical (M = g x ones(2,2)): each of the
    2^|S| minors of a subset is det g[S], so abar[S] = 2^|S| det g[S]."""
    rng = np.random.default_rng(4300)
    n = 16
    g = rng.standard_normal((n, n)) * 0.05 + np.eye(n)   # strictly diagonally dominant: no small pivots
    M = np.kron(g, np.ones((2, 2)))[None]
    c, ab = apm.two_type_cdet(dev(M), return_weights=True)
    ab = ab.cpu().numpy()[0]
    ref = oracle.minors_lu(g)
    pop = np.array([bin(S).count("1") for S in range(1 << n)])
    scale = oracle.minors_rowsum_bound(g) * 2.0 ** pop
    assert np.all(np.abs(ab - 2.0 ** pop * ref) <= TOL * scale)


def test_zero_pivot_corrected_and_nonfinite_flagged(apm):
    """A zero pivot is shifted and corrected (Section III.C); with a zero shift
    it is flagged and the row is NaN, as is a non-finite input."""
    n = 7
    M = I.two_type_batch(4, n, seed=4400)
    M[1, 2 * n - 2, 2 * n - 2] = 0.0          # type 1 of the last vertex: a pivot of the first step
    M[2, 0, 3] = np.nan
    ab, st = apm.two_type_cdet(dev(M), return_weights=True, return_status=True)[1:]
    st, ab = st.cpu().numpy(), ab.cpu().numpy()
    assert st[1] == apm.ST_PIVOT_CORRECTED and st[2] & apm.ST_NONFINITE_INPUT and st[0] == 0 and st[3] == 0
    abr, sc = oracle.nand(M[[0, 1, 3]])
    assert np.all(np.abs(ab[[0, 1, 3]] - abr) <= TOL * sc)
    assert np.all(np.isnan(ab[2]))
    ab0, st0 = apm.two_type_cdet(dev(M), return_weights=True, return_status=True, piv_shift=0.0)[1:]
    st0, ab0 = st0.cpu().numpy(), ab0.cpu().numpy()
    assert st0[1] & apm.ST_ZERO_PIVOT and np.all(np.isnan(ab0[1])) and np.array_equal(ab0[0], ab[0])


def zero_corner(M):
    """A zero pivot on the first step of every matrix: entry (2n-2, 2n-2)."""
    M = M.copy()
    M[:, -2, -2] = 0.0
    return M


@pytest.mark.parametrize("n", [3, 5, 6, 7, 9])
def test_pivot_correction_all_minors(apm, n):
    """A threshold of 0.7 ||M||max shifts most pivots of the tree, tail and depth
    first, nested in one another: every one of the 3^n minors is still the
    oracle's."""
    rng = np.random.default_rng(4500 + n)
    M = zero_corner(rng.standard_normal((3, 2 * n, 2 * n)))
    x, st = apm.nand_minors(dev(M), return_status=True, piv_threshold=0.7)
    x, st = x.cpu().numpy(), st.cpu().numpy()
    ab, sc, m3 = oracle.nand(M, minors=True)
    err = float(np.max(np.abs(x - m3) / sc[:, support_of_ternary(n)]))
    assert err <= TOL, err
    assert np.all(st == apm.ST_PIVOT_CORRECTED)


@pytest.mark.parametrize("n", [4, 7, 10])
def test_pivot_correction_type_sums(apm, n):
    """The same thresholds for the type sums: tail corrections inside the
    vertex-by-vertex reduction, depth-first ones through the target lists (up to
    2^4 targets at n = 10); then the connected sums."""
    rng = np.random.default_rng(4600 + n)
    M = zero_corner(rng.standard_normal((3, 2 * n, 2 * n)))
    c, ab, st = apm.two_type_cdet(dev(M), return_weights=True, return_status=True, piv_threshold=0.7)
    c, ab, st = c.cpu().numpy(), ab.cpu().numpy(), st.cpu().numpy()
    abr, sc = oracle.nand(M)
    assert np.all(np.abs(ab - abr) <= TOL * sc)
    cr = oracle.cdet_recursion(abr)
    assert np.all(np.abs(c - cr) <= TOL * np.maximum(oracle.cdet_scale(sc), 1e-300))
    assert np.all(st == apm.ST_PIVOT_CORRECTED)


@pytest.mark.parametrize("n", [8, 12])
def test_near_singular_blocks_default_threshold(apm, n):
    """Weakly coupled 2 x 2 blocks (coupling 1e-4) whose diagonal has exact zeros:
    the default threshold corrects the pivots of those rows wherever they fall."""
    rng = np.random.default_rng(4700 + n)
    M = 1e-4 * rng.standard_normal((2, 2 * n, 2 * n))
    for i in range(n):
        M[:, 2 * i:2 * i + 2, 2 * i:2 * i + 2] += rng.standard_normal((2, 2, 2))
    for r in (1, 4, 2 * n - 1, 2 * n - 4):
        M[:, r, r] = 0.0
    ab, st = apm.two_type_cdet(dev(M), return_weights=True, return_status=True)[1:]
    ab, st = ab.cpu().numpy(), st.cpu().numpy()
    abr, sc = oracle.nand(M)
    assert np.all(np.abs(ab - abr) <= TOL * sc)
    assert np.all(st == apm.ST_PIVOT_CORRECTED)
    if n <= 9:
        x = apm.nand_minors(dev(M)).cpu().numpy()
        m3 = oracle.nand(M, minors=True)[2]
        assert np.all(np.abs(x - m3) <= TOL * sc[:, support_of_ternary(n)])


def test_correction_records_overflow(apm):
    """A threshold above every pivot corrects all of them: more depth-first
    records than the 256 kept (all-minor mode, n = 13) or more than 16 targets
    on a path (type sums, n = 16) set the overflow bit and a NaN row."""
    rng = np.random.default_rng(4800)
    M = rng.standard_normal((1, 26, 26))
    x, st = apm.nand_minors(dev(M), return_status=True, piv_threshold=1e3)
    assert int(st.cpu()[0]) & apm.ST_CORRECTION_OVERFLOW and bool(torch.isnan(x).all())
    M = rng.standard_normal((1, 32, 32))
    ab, st = apm.two_type_cdet(dev(M), return_weights=True, return_status=True, piv_threshold=1e3)[1:]
    assert int(st.cpu()[0]) & apm.ST_CORRECTION_OVERFLOW and bool(torch.isnan(ab).all())


def test_bench_size_sampled_and_deterministic(apm):
    """The launch the benchmark times (16384 two-type matrices of order 10),
    sampled rows against the oracle, and two calls bit for bit equal."""
    M = I.two_type_batch(16384, 10, seed=7)
    Md = dev(M)
    c1, ab1 = apm.two_type_cdet(Md, return_weights=True)
    c2 = apm.two_type_cdet(Md)
    assert torch.equal(c1, c2)
    idx = [0, 5000, 16383]
    abr, sc = oracle.nand(M[idx])
    assert np.all(np.abs(ab1[idx].cpu().numpy() - abr) <= TOL * sc)
    cr = oracle.cdet_recursion(abr)
    assert np.all(np.abs(c1[idx].cpu().numpy() - cr) <= TOL * np.maximum(oracle.cdet_scale(sc), 1e-300))
