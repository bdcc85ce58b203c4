"""Value pins for the oracle's error scales.

Every parity tolerance is 1e-10 times a scale that the oracle computes, so a
scale inflated by mistake would loosen every parity test without failing one.
Each scale function is therefore compared here, by value, with a quantity
computed another way: brute-force Leibniz sums over permutations (itertools),
set partitions enumerated in the test, and closed forms for matrices whose
entries all have one modulus or whose only nonzero entries sit on the diagonal.
A factor of two, a dropped term or a wrong index in any of them fails a check.

  minors_scale / minors_rowsum_bound  perm(|A[S]|) and prod_i sum_j |A_ij| (Section II)
  perm_ryser_term_scale               sum over T of |prod_i r_i(T)| (Eq. ryser)
  cdet_scale                          the recursion of Eq. recursion with every sign +
  keldysh_scale / keldysh2_scale      sums over the Keldysh assignments (Section V.D)
  xnor_scale                          perm or row-sum bound of each kept 2|S| x 2|S| block (Section III.B)
  nand (scale output)                 row-sum bounds summed over the vertex types (Section III.C)
"""
import itertools
import math

import numpy as np
import pytest

import oracle


def leibniz_abs(M):
    """sum over permutations of prod_i |M_{i, p(i)}| (the absolute Leibniz terms)."""
    k = M.shape[0]
    A = np.abs(M)
    return float(sum(math.prod(A[i, p[i]] for i in range(k)) for p in itertools.permutations(range(k))))


def set_partitions(elems):
    """Every partition of the list elems into non-empty blocks."""
    if not elems:
        yield []
        return
    first, rest = elems[0], elems[1:]
    for part in set_partitions(rest):
        # first joins one of the blocks, or starts its own
        for i in range(len(part)):
            yield part[:i] + [[first] + part[i]] + part[i + 1:]
        yield [[first]] + part


def mask_of(block):
    return sum(1 << e for e in block)


def elems_of(S, n):
    return [e for e in range(n) if (S >> e) & 1]


def unit_phases(rng, shape):
    return np.exp(2j * np.pi * rng.random(shape))


# --------------------------------------------------------------------------
# minors: perm(|A[S]|) and the row-sum bound
# --------------------------------------------------------------------------

def test_minors_scales_equal_modulus_closed_forms():
    # |A_ij| = g for all i, j: perm(|A[S]|) = k! g^k and prod_i sum_j |A_ij| = (k g)^k
    rng = np.random.default_rng(3001)
    n, g = 7, 0.37
    A = g * np.sign(rng.standard_normal((n, n)))
    ps, rb = oracle.minors_scale(A), oracle.minors_rowsum_bound(A)
    for S in range(1 << n):
        k = bin(S).count("1")
        assert abs(ps[S] - math.factorial(k) * g ** k) <= 1e-13 * math.factorial(k) * g ** k
        assert abs(rb[S] - (k * g) ** k) <= 1e-13 * max(1.0, (k * g) ** k)


def test_minors_rowsum_bound_by_value():
    rng = np.random.default_rng(3002)
    n = 6
    A = rng.standard_normal((n, n))
    rb = oracle.minors_rowsum_bound(A)
    for S in range(1 << n):
        e = elems_of(S, n)
        ref = math.prod(sum(abs(A[i, j]) for j in e) for i in e)
        assert abs(rb[S] - ref) <= 1e-13 * ref
    # diagonal matrix: both scales are prod_{i in S} |A_ii|
    d = rng.standard_normal(n)
    D = np.diag(d)
    ref = np.array([math.prod(abs(d[i]) for i in elems_of(S, n)) for S in range(1 << n)])
    np.testing.assert_allclose(oracle.minors_rowsum_bound(D), ref, rtol=1e-14)
    np.testing.assert_allclose(oracle.minors_scale(D), ref, rtol=1e-14)


# --------------------------------------------------------------------------
# Ryser's term scale
# --------------------------------------------------------------------------

def test_perm_ryser_term_scale_diagonal_and_rank_one():
    rng = np.random.default_rng(3003)
    n = 6
    # diagonal: r_i(T) = [i in T] A_ii, so only T = S contributes: prod |A_ii|
    d = rng.standard_normal(n)
    ref = np.array([math.prod(abs(d[i]) for i in elems_of(S, n)) for S in range(1 << n)])
    np.testing.assert_allclose(oracle.perm_ryser_term_scale(np.diag(d)), ref, rtol=1e-14)
    # A = u v^T with u, v > 0: r_i(T) = u_i v(T), terms prod_i u_i * v(T)^k
    u, v = rng.random(n) + 0.1, rng.random(n) + 0.1
    sc = oracle.perm_ryser_term_scale(np.outer(u, v))
    for S in range(1 << n):
        e = elems_of(S, n)
        k = len(e)
        ref = math.prod(u[i] for i in e) * sum(sum(v[j] for j in T) ** k
                                               for r in range(k + 1) for T in itertools.combinations(e, r))
        assert abs(sc[S] - ref) <= 1e-13 * ref


# --------------------------------------------------------------------------
# connected sums: the scale equals the all-positive set-partition sum
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [1, 2, 3, 5, 6])
def test_cdet_scale_is_positive_partition_sum(n):
    """The recursion with every sign positive is the set-partition sum
    sum_pi (|pi| - 1)! prod_B ahat[B] (the Moebius formula with all signs +);
    the partitions are enumerated here, independently of the oracle."""
    rng = np.random.default_rng(3010 + n)
    ahat = rng.random(1 << n) + 0.05
    ahat[0] = 1.0
    sc = oracle.cdet_scale(ahat)
    assert sc[0] == 0.0
    for S in range(1, 1 << n):
        ref = 0.0
        for part in set_partitions(elems_of(S, n)):
            ref += math.factorial(len(part) - 1) * math.prod(ahat[mask_of(B)] for B in part)
        assert abs(sc[S] - ref) <= 1e-13 * ref, (S, sc[S], ref)


def test_cdet_scale_all_ones_is_ordered_bell_like_count():
    # ahat = 1 everywhere: the scale of a k-set is sum over partitions of (|pi|-1)!,
    # i.e. sum_m S(k, m) (m-1)! with S the Stirling numbers of the second kind
    n = 8
    sc = oracle.cdet_scale(np.ones(1 << n))

    def stirling2(k, m):
        return sum((-1) ** (m - j) * math.comb(m, j) * j ** k for j in range(m + 1)) // math.factorial(m)

    for S in range(1, 1 << n):
        k = bin(S).count("1")
        ref = sum(stirling2(k, m) * math.factorial(m - 1) for m in range(1, k + 1))
        assert sc[S] == ref


# --------------------------------------------------------------------------
# Keldysh sums
# --------------------------------------------------------------------------

def keldysh_sub(Mt, al, n):
    rows = [2 * i + ((al >> i) & 1) for i in range(n)]
    return Mt[np.ix_(rows, rows)]


@pytest.mark.parametrize("n", [1, 2, 4])
def test_keldysh_scale_perm_path_is_abs_leibniz(n):
    rng = np.random.default_rng(3020 + n)
    Mt = rng.standard_normal((2, 2 * n, 2 * n)) + 1j * rng.standard_normal((2, 2 * n, 2 * n))
    sc = oracle.keldysh_scale(Mt, use_perm=True)
    for b in range(2):
        ref = sum(leibniz_abs(keldysh_sub(Mt[b], al, n)) for al in range(1 << n))
        assert abs(sc[b] - ref) <= 1e-13 * ref


@pytest.mark.parametrize("use_perm", [True, False])
def test_keldysh_scale_closed_forms(use_perm):
    rng = np.random.default_rng(3030)
    n, g = 5, 0.6
    # every |entry| = g: each M_alpha has perm(|M|) = n! g^n and row-sum product (n g)^n
    Mt = g * unit_phases(rng, (2 * n, 2 * n))
    ref = 2 ** n * (math.factorial(n) * g ** n if use_perm else (n * g) ** n)
    assert abs(oracle.keldysh_scale(Mt, use_perm=use_perm) - ref) <= 1e-13 * ref
    # only the diagonal entries of the 2 x 2 blocks: M_alpha is diagonal with
    # entries Mt[2i + alpha_i, 2i + alpha_i], and the sum over alpha factorises
    x, y = rng.random(n) + 0.1, rng.random(n) + 0.1
    D = np.zeros((2 * n, 2 * n), complex)
    for i in range(n):
        D[2 * i, 2 * i] = x[i] * unit_phases(rng, ())
        D[2 * i + 1, 2 * i + 1] = y[i] * unit_phases(rng, ())
    ref = math.prod(x[i] + y[i] for i in range(n))
    assert abs(oracle.keldysh_scale(D, use_perm=use_perm) - ref) <= 1e-13 * ref
    # only the (+, +) blocks: every alpha with a minus index has a zero row
    P = np.zeros((2 * n, 2 * n), complex)
    G = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    P[0::2, 0::2] = G
    ref = leibniz_abs(G) if use_perm else math.prod(np.abs(G).sum(axis=1))
    assert abs(oracle.keldysh_scale(P, use_perm=use_perm) - ref) <= 1e-13 * ref


def test_keldysh_scale_rowsum_path_by_value():
    rng = np.random.default_rng(3031)
    n = 4
    Mt = rng.standard_normal((2 * n, 2 * n)) + 1j * rng.standard_normal((2 * n, 2 * n))
    ref = sum(math.prod(np.abs(keldysh_sub(Mt, al, n)).sum(axis=1)) for al in range(1 << n))
    assert abs(oracle.keldysh_scale(Mt, use_perm=False) - ref) <= 1e-13 * ref


def test_keldysh2_scale_closed_forms():
    rng = np.random.default_rng(3040)
    n, gu, gd = 5, 0.7, 1.3
    Mu = gu * unit_phases(rng, (2 * n, 2 * n))
    Md = gd * unit_phases(rng, (2 * n, 2 * n))
    ref = 2 ** n * (n * gu) ** n * (n * gd) ** n
    assert abs(oracle.keldysh2_scale(Mu, Md) - ref) <= 1e-13 * ref
    # diagonal 2 x 2 block entries only: sum_alpha prod_i |U_i^alpha_i| |D_i^alpha_i|
    xu, yu, xd, yd = (rng.random(n) + 0.1 for _ in range(4))
    U = np.zeros((2 * n, 2 * n), complex)
    D = np.zeros((2 * n, 2 * n), complex)
    for i in range(n):
        U[2 * i, 2 * i], U[2 * i + 1, 2 * i + 1] = xu[i], -yu[i]
        D[2 * i, 2 * i], D[2 * i + 1, 2 * i + 1] = 1j * xd[i], yd[i]
    ref = math.prod(xu[i] * xd[i] + yu[i] * yd[i] for i in range(n))
    assert abs(oracle.keldysh2_scale(U, D) - ref) <= 1e-13 * ref
    # a partner with every |entry| = g has row-sum product (n g)^n for every alpha,
    # so the two-spin scale is that times the single-spin row-sum scale
    Mx = rng.standard_normal((2 * n, 2 * n)) + 1j * rng.standard_normal((2 * n, 2 * n))
    ref = (n * gd) ** n * oracle.keldysh_scale(Mx, use_perm=False)
    assert abs(oracle.keldysh2_scale(Mx, Md) - ref) <= 1e-13 * ref


def test_keldysh2_scale_by_value():
    rng = np.random.default_rng(3041)
    n = 3
    Mu = rng.standard_normal((2 * n, 2 * n)) + 1j * rng.standard_normal((2 * n, 2 * n))
    Md = rng.standard_normal((2 * n, 2 * n)) + 1j * rng.standard_normal((2 * n, 2 * n))
    ref = 0.0
    for al in itertools.product([0, 1], repeat=n):
        rows = [2 * i + a for i, a in enumerate(al)]
        ref += math.prod(np.abs(Mu[np.ix_(rows, rows)]).sum(axis=1)) * \
            math.prod(np.abs(Md[np.ix_(rows, rows)]).sum(axis=1))
    assert abs(oracle.keldysh2_scale(Mu, Md) - ref) <= 1e-13 * ref


# --------------------------------------------------------------------------
# XNOR (Nambu) minors and NAND type sums
# --------------------------------------------------------------------------

def xnor_sub(M, S, n):
    idx = [r for v in range(n) if (S >> v) & 1 for r in (2 * v, 2 * v + 1)]
    return M[np.ix_(idx, idx)]


def test_xnor_scale_perm_path_is_abs_leibniz():
    rng = np.random.default_rng(3050)
    n = 3
    M = rng.standard_normal((2 * n, 2 * n))
    sp = oracle.xnor_scale(M, use_perm=True)
    sb = oracle.xnor_scale(M, use_perm=False)
    assert sp[0] == 1.0 and sb[0] == 1.0
    for S in range(1, 1 << n):
        sub = xnor_sub(M, S, n)
        ref = leibniz_abs(sub)
        assert abs(sp[S] - ref) <= 1e-13 * ref
        ref = math.prod(np.abs(sub).sum(axis=1))
        assert abs(sb[S] - ref) <= 1e-13 * ref


@pytest.mark.parametrize("use_perm", [True, False])
def test_xnor_scale_closed_forms(use_perm):
    rng = np.random.default_rng(3051)
    n, g = 4, 0.45
    M = g * np.sign(rng.standard_normal((2 * n, 2 * n)))
    s = oracle.xnor_scale(M, use_perm=use_perm)
    for S in range(1 << n):
        m = 2 * bin(S).count("1")
        ref = math.factorial(m) * g ** m if use_perm else (m * g) ** m
        # the perm path evaluates Ryser's alternating sum, whose rounding scale is
        # its term sum sum_t C(m, t) t^m g^m (thousands of times perm at m = 8)
        tol = 1e-14 * sum(math.comb(m, t) * t ** m for t in range(m + 1)) * g ** m if use_perm else 1e-13 * ref
        assert abs(s[S] - ref) <= max(tol, 1e-15), (S, s[S], ref)
    # block diagonal: the kept submatrix is block diagonal, so both scales factorise
    # over the kept 2 x 2 blocks [[a, b], [c, d]]: perm = |a d| + |b c|, bound = (|a|+|b|)(|c|+|d|)
    B = rng.standard_normal((n, 2, 2))
    Mb = np.zeros((2 * n, 2 * n))
    for v in range(n):
        Mb[2 * v:2 * v + 2, 2 * v:2 * v + 2] = B[v]
    s = oracle.xnor_scale(Mb, use_perm=use_perm)
    for S in range(1 << n):
        f = []
        for v in elems_of(S, n):
            a, b, c, d = np.abs(B[v]).ravel()
            f.append(a * d + b * c if use_perm else (a + b) * (c + d))
        ref = math.prod(f)
        assert abs(s[S] - ref) <= 1e-13 * max(ref, 1e-300)


def test_nand_scale_closed_forms_and_value():
    rng = np.random.default_rng(3060)
    n, g = 4, 0.8
    # every |entry| = g: each of the 2^k assignments of a k-set keeps a k x k
    # submatrix with row-sum product (k g)^k
    M = g * np.sign(rng.standard_normal((2 * n, 2 * n)))
    _, sc = oracle.nand(M)
    for S in range(1 << n):
        k = bin(S).count("1")
        ref = 2 ** k * (k * g) ** k
        assert abs(sc[S] - ref) <= 1e-13 * max(ref, 1.0)
    # diagonal entries only: the kept submatrix is diagonal, so the sum over the
    # types of each kept vertex factorises: prod_{i in S} (|M_2i,2i| + |M_2i+1,2i+1|)
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    D = np.zeros((2 * n, 2 * n))
    D[0::2, 0::2] = np.diag(x)
    D[1::2, 1::2] = np.diag(y)
    _, sc = oracle.nand(D)
    for S in range(1 << n):
        ref = math.prod(abs(x[i]) + abs(y[i]) for i in elems_of(S, n))
        assert abs(sc[S] - ref) <= 1e-13 * ref
    # general matrix, by enumeration of the type assignments
    R = rng.standard_normal((2 * n, 2 * n))
    _, sc = oracle.nand(R)
    for S in range(1 << n):
        e = elems_of(S, n)
        ref = 0.0
        for types in itertools.product([0, 1], repeat=len(e)):
            idx = [2 * v + t for v, t in zip(e, types)]
            ref += math.prod(np.abs(R[np.ix_(idx, idx)]).sum(axis=1)) if idx else 1.0
        assert abs(sc[S] - ref) <= 1e-13 * ref
