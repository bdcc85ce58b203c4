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
    assert int(st.cpu().numpy().max()) == 0
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


def test_zero_pivot_and_nonfinite_flagged(apm):
    n = 7
    M = I.two_type_batch(4, n, seed=4400)
    M[1, 2 * n - 2, 2 * n - 2] = 0.0          # type 1 of the last vertex: a pivot of the first step
    M[2, 0, 3] = np.nan
    ab, st = apm.two_type_cdet(dev(M), return_weights=True, return_status=True)[1:]
    st, ab = st.cpu().numpy(), ab.cpu().numpy()
    assert st[1] & apm.ST_ZERO_PIVOT and st[2] & apm.ST_NONFINITE_INPUT and st[0] == 0 and st[3] == 0
    assert np.all(np.isnan(ab[1])) and np.all(np.isnan(ab[2])) and np.all(np.isfinite(ab[0]))


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
