"""Pins for the CPU oracle against facts fixed by mathematics, not by the oracle.

Every check here is independent of the oracle's own code path: brute-force
Leibniz expansion, closed forms (diagonal, triangular, matrix-determinant
lemma, all-ones permanents, rank-one permanents), perfect-matching counts,
numpy's LAPACK determinant, the set-partition route against the recursion,
the cycle formula for connected determinants, block-diagonal factorisation, and
the largest-time identity of the Keldysh sum.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle
from paper_2104_07638_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def masks_elems(n):
    return [[e for e in range(n) if (S >> e) & 1] for S in range(1 << n)]


def perm_sign(p):
    s, seen = 1, [False] * len(p)
    for i in range(len(p)):
        if not seen[i]:
            j, L = i, 0
            while not seen[j]:
                seen[j] = True
                j = p[j]
                L += 1
            if L % 2 == 0:
                s = -s
    return s


def leibniz_det(M):
    k = M.shape[0]
    tot = 0.0
    for p in itertools.permutations(range(k)):
        tot += perm_sign(p) * math.prod(M[i, p[i]] for i in range(k))
    return tot


def leibniz_perm(M):
    k = M.shape[0]
    return sum(math.prod(M[i, p[i]] for i in range(k)) for p in itertools.permutations(range(k)))


def rel_err(x, ref, scale):
    return np.max(np.abs(np.asarray(x) - np.asarray(ref)) / np.maximum(scale, 1e-300))


# --------------------------------------------------------------------------
# golden worked example (hand expanded)
# --------------------------------------------------------------------------

def test_golden_tridiagonal_3x3():
    rows = np.loadtxt(os.path.join(GOLDEN, "tridiag3_int.txt"))
    A = np.array([[2., 1, 0], [1, 3, 1], [0, 1, 4]])
    m = oracle.minors_lu(A)
    p = oracle.perm_ryser(A)
    np.testing.assert_allclose(m, rows[:, 1], rtol=0, atol=1e-12)
    np.testing.assert_allclose(p, rows[:, 2], rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle.cdet_recursion(m), rows[:, 3], atol=1e-12)
    np.testing.assert_allclose(oracle.cdet_recursion(m * m), rows[:, 4], atol=1e-10)


# --------------------------------------------------------------------------
# principal minors
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n,seed", [(1, 0), (3, 1), (5, 2), (6, 3)])
def test_minors_vs_leibniz(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    m = oracle.minors_lu(A)
    ref = np.array([leibniz_det(A[np.ix_(e, e)]) if e else 1.0 for e in masks_elems(n)])
    scale = oracle.minors_scale(A)
    assert m[0] == 1.0
    assert rel_err(m, ref, scale) < 1e-13


def test_minors_vs_numpy_det():
    rng = np.random.default_rng(7)
    n = 9
    A = rng.standard_normal((n, n))
    m = oracle.minors_lu(A)
    ref = np.array([np.linalg.det(A[np.ix_(e, e)]) if e else 1.0 for e in masks_elems(n)])
    assert rel_err(m, ref, oracle.minors_scale(A)) < 1e-13


def test_minors_diagonal_and_triangular_products():
    rng = np.random.default_rng(11)
    n = 8
    d = rng.uniform(-2, 2, n)
    U = np.triu(rng.standard_normal((n, n)), 1) + np.diag(d)
    L = U.T.copy()
    prods = np.array([np.prod(d[e]) for e in masks_elems(n)])
    for A in (np.diag(d), U, L):
        np.testing.assert_allclose(oracle.minors_lu(A), prods, rtol=1e-13, atol=1e-15)


def test_minors_matrix_determinant_lemma():
    # det(I + u v^T)[S] = 1 + sum_{i in S} u_i v_i
    rng = np.random.default_rng(12)
    n = 9
    u, v = rng.standard_normal(n), rng.standard_normal(n)
    A = np.eye(n) + np.outer(u, v)
    ref = np.array([1.0 + np.sum(u[e] * v[e]) for e in masks_elems(n)])
    assert rel_err(oracle.minors_lu(A), ref, oracle.minors_scale(A)) < 1e-13


def test_minors_rank_one_and_zero_diagonal():
    rng = np.random.default_rng(13)
    n = 7
    u, v = rng.standard_normal(n), rng.standard_normal(n)
    R = np.outer(u, v)
    m = oracle.minors_lu(R)
    size = np.array([len(e) for e in masks_elems(n)])
    assert np.all(np.abs(m[size >= 2]) <= 1e-13 * oracle.minors_scale(R)[size >= 2])
    Z = rng.standard_normal((n, n))
    np.fill_diagonal(Z, 0.0)
    ref = np.array([leibniz_det(Z[np.ix_(e, e)]) if e else 1.0 for e in masks_elems(n)])
    assert rel_err(oracle.minors_lu(Z), ref, oracle.minors_scale(Z)) < 1e-13


def test_minors_leading_are_lu_pivot_products():
    # leading minors (masks 2^l - 1) = products of the pivots of elimination
    # without pivoting (Section III.A)
    A = I.gaussian_plus_2I(10)[0]
    n = 10
    U = A.copy()
    piv = []
    for k in range(n):
        piv.append(U[k, k])
        U[k + 1:, k:] -= np.outer(U[k + 1:, k] / U[k, k], U[k, k:])
    m = oracle.minors_lu(A)
    for l in range(1, n + 1):
        assert abs(m[(1 << l) - 1] - np.prod(piv[:l])) <= 1e-12 * abs(np.prod(piv[:l]))


def test_minors_scale_is_abs_leibniz():
    rng = np.random.default_rng(14)
    A = rng.standard_normal((5, 5))
    s = oracle.minors_scale(A)
    ref = [leibniz_perm(np.abs(A[np.ix_(e, e)])) if e else 1.0 for e in masks_elems(5)]
    np.testing.assert_allclose(s, ref, rtol=1e-13)
    assert np.all(oracle.minors_rowsum_bound(A) >= s * (1 - 1e-12))


# --------------------------------------------------------------------------
# permanents
# --------------------------------------------------------------------------

def test_perm_all_ones_factorial():
    n = 10
    p = oracle.perm_ryser(np.ones((n, n)))
    ref = np.array([math.factorial(len(e)) for e in masks_elems(n)], dtype=float)
    np.testing.assert_allclose(p, ref, rtol=1e-13)


@pytest.mark.parametrize("n,seed", [(4, 0), (6, 1), (7, 2)])
def test_perm_vs_leibniz(n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    ref = np.array([leibniz_perm(A[np.ix_(e, e)]) if e else 1.0 for e in masks_elems(n)])
    scale = oracle.perm_ryser(A, absval=True)
    assert rel_err(oracle.perm_ryser(A), ref, scale) < 1e-13


def test_perm_rank_one_and_diagonal():
    rng = np.random.default_rng(21)
    n = 8
    u, v = rng.uniform(0.5, 1.5, n), rng.uniform(0.5, 1.5, n)
    ref = np.array([math.factorial(len(e)) * np.prod(u[e] * v[e]) for e in masks_elems(n)])
    np.testing.assert_allclose(oracle.perm_ryser(np.outer(u, v)), ref, rtol=1e-12)
    d = rng.standard_normal(n)
    ref = np.array([np.prod(d[e]) for e in masks_elems(n)])
    np.testing.assert_allclose(oracle.perm_ryser(np.diag(d)), ref, rtol=1e-12, atol=1e-15)


def test_perm_ryser_term_scale_closed_forms():
    # all-ones k x k: the Ryser terms are C(k,t) t^k in magnitude
    n = 7
    sc = oracle.perm_ryser_term_scale(np.ones((n, n)))
    for S, e in enumerate(masks_elems(n)):
        k = len(e)
        ref = sum(math.comb(k, t) * t ** k for t in range(k + 1)) if k else 1
        assert abs(sc[S] - ref) <= 1e-12 * ref
    rng = np.random.default_rng(23)
    A = rng.standard_normal((6, 6))
    assert np.all(oracle.perm_ryser_term_scale(A) >= np.abs(oracle.perm_ryser(A)) * (1 - 1e-12))


def test_perm_zero_one_counts_perfect_matchings():
    rng = np.random.default_rng(22)
    n = 7
    B = (rng.random((n, n)) < 0.5).astype(float)
    p = oracle.perm_ryser(B)
    for S, e in enumerate(masks_elems(n)):
        cnt = sum(all(B[e[i], e[q[i]]] for i in range(len(e)))
                  for q in itertools.permutations(range(len(e)))) if e else 1
        assert p[S] == cnt


# --------------------------------------------------------------------------
# connected sums
# --------------------------------------------------------------------------

def test_cdet_n2_closed_form_and_singletons():
    rng = np.random.default_rng(30)
    a = np.concatenate([[1.0], rng.standard_normal(3)])
    c = oracle.cdet_recursion(a)
    assert c[0] == 0 and c[1] == a[1] and c[2] == a[2]
    assert abs(c[3] - (a[3] - a[1] * a[2])) < 1e-15


@pytest.mark.parametrize("n", [3, 6, 9])
def test_cdet_recursion_vs_set_partitions(n):
    rng = np.random.default_rng(31 + n)
    a = rng.standard_normal(1 << n)
    a[0] = 1.0
    c1 = oracle.cdet_recursion(a)
    c2 = oracle.cdet_partition(a)
    scale = oracle.cdet_scale(np.abs(a))
    assert rel_err(c1, c2, scale) < 1e-13


def test_cdet_single_determinant_is_cycle_sum():
    # with a[S] = det M[S] the connected part keeps exactly the permutations of S
    # that are one single cycle: c[S] = (-1)^{|S|-1} sum_{cycles} prod M_{i,s(i)}
    rng = np.random.default_rng(32)
    n = 6
    M = rng.standard_normal((n, n))
    c = oracle.cdet_recursion(oracle.minors_lu(M))
    for S, e in enumerate(masks_elems(n)):
        if not e:
            continue
        k = len(e)
        tot = 0.0
        first = e[0]
        for rest in itertools.permutations(e[1:]):
            cyc = (first,) + rest                  # the cycle first->rest[0]->...->first
            succ = {cyc[i]: cyc[(i + 1) % k] for i in range(k)}
            tot += math.prod(M[i, succ[i]] for i in e)
        ref = (-1) ** (k - 1) * tot
        assert abs(c[S] - ref) <= 1e-12 * (1 + abs(ref))


@pytest.mark.parametrize("square", [False, True])
def test_cdet_block_diagonal_vanishes_across_blocks(square):
    rng = np.random.default_rng(33)
    n = 8
    M = rng.standard_normal((n, n)) + 2 * np.eye(n)
    blk = np.array([0, 1, 0, 1, 1, 0, 0, 1])
    M[blk[:, None] != blk[None, :]] = 0.0
    m = oracle.minors_lu(M)
    a = m * m if square else m
    c = oracle.cdet_recursion(a)
    scale = oracle.cdet_scale(np.abs(a))
    for S, e in enumerate(masks_elems(n)):
        if len(set(blk[e])) == 2:
            assert abs(c[S]) <= 1e-13 * scale[S]


def test_cdet_scale_bounds_partition_route():
    # the error scale must bound |c| computed by the independent partition route
    rng = np.random.default_rng(35)
    n = 8
    a = rng.standard_normal(1 << n)
    a[0] = 1.0
    assert np.all(oracle.cdet_scale(np.abs(a)) >= np.abs(oracle.cdet_partition(a)) * (1 - 1e-12))


def test_cdet_independent_of_choice_of_j():
    # Eq. recursion with j = the highest element instead of the lowest (written
    # here independently) must give the same connected sums.
    rng = np.random.default_rng(34)
    n = 7
    a = rng.standard_normal(1 << n)
    a[0] = 1.0
    c = np.zeros(1 << n)
    for S in range(1, 1 << n):
        j = 1 << (S.bit_length() - 1)
        acc = a[S]
        for T in range(1, S):
            if (T & S) == T and (T & j):
                acc -= c[T] * a[S & ~T]
        c[S] = acc
    assert rel_err(oracle.cdet_recursion(a), c, oracle.cdet_scale(np.abs(a))) < 1e-13


# --------------------------------------------------------------------------
# Keldysh sums
# --------------------------------------------------------------------------

def keldysh_numpy(Mt, signed):
    n = Mt.shape[0] // 2
    tot = 0j
    for al in range(1 << n):
        idx = [2 * i + ((al >> i) & 1) for i in range(n)]
        d = np.linalg.det(Mt[np.ix_(idx, idx)]) if n else 1.0
        tot += (-1) ** bin(al).count("1") * d if signed else d
    return tot


@pytest.mark.parametrize("n", [1, 3, 6])
def test_keldysh_vs_numpy_bruteforce(n):
    rng = np.random.default_rng(40 + n)
    Mt = rng.standard_normal((2 * n, 2 * n)) + 1j * rng.standard_normal((2 * n, 2 * n))
    for signed in (False, True):
        s = oracle.keldysh(Mt, signed=signed)
        assert abs(s - keldysh_numpy(Mt, signed)) <= 1e-12 * oracle.keldysh_scale(Mt)


def test_keldysh_equal_blocks_closed_form():
    rng = np.random.default_rng(45)
    n = 6
    g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    Mt = np.kron(g, np.ones((2, 2)))
    s = oracle.keldysh(Mt)
    ref = 2 ** n * np.linalg.det(g)
    assert abs(s - ref) <= 1e-12 * oracle.keldysh_scale(Mt)


def test_keldysh_largest_time_identity():
    # physical contour G0: the two Keldysh indices of the latest vertex give the
    # same matrix, so the (-1)^{#-} weighted sum vanishes and the plain sum is
    # twice the sum with that index fixed.
    n = 7
    x, m = I.keldysh_vertices(4, n, seed=5)
    Mt = I.keldysh_matrices_from_vertices(x, m)
    s_signed = oracle.keldysh(Mt, signed=True)
    s_plain = oracle.keldysh(Mt, signed=False)
    scale = oracle.keldysh_scale(Mt)
    assert np.all(np.abs(s_signed) <= 1e-13 * scale)
    for b in range(4):
        last = int(np.argmax(m[b]))
        half = 0j
        for al in range(1 << n):
            if (al >> last) & 1:
                continue
            idx = [2 * i + ((al >> i) & 1) for i in range(n)]
            half += np.linalg.det(Mt[b][np.ix_(idx, idx)])
        assert abs(s_plain[b] - 2 * half) <= 1e-12 * scale[b]


def test_keldysh_partial_sums_are_leading_blocks():
    rng = np.random.default_rng(46)
    n = 5
    Mt = rng.standard_normal((2 * n, 2 * n)) + 1j * rng.standard_normal((2 * n, 2 * n))
    s, p = oracle.keldysh(Mt, partial=True)
    assert p[0] == 1.0 and p[n] == s
    for d in range(1, n):
        sub = Mt[:2 * d, :2 * d]
        assert abs(p[d] - keldysh_numpy(sub, False)) <= 1e-12 * oracle.keldysh_scale(sub)


# --------------------------------------------------------------------------
# inputs sanity (shapes and conventions the workloads rely on)
# --------------------------------------------------------------------------

def test_inputs_shapes_and_conventions():
    A = I.hubbard_batch(4, 12, seed=2)
    assert A.shape == (4, 12, 12)
    nd = np.diag(A[0])
    assert np.allclose(nd, nd[0]) and 0.0 < nd[0] < 1.0        # density on the diagonal
    G = I.hubbard_g0_table()
    mt = I.HUB_MTAU
    # the jump at tau = 0: G(0,0^-) - G(0,0^+) = 1
    assert abs(G[0, 0, mt - 2] - G[0, 0, mt] - 1.0) < 1e-2
    P = I.perm_batch(14, 3)
    assert P.shape == (3, 14, 14) and np.all(P >= 0) and np.allclose(P != 0, (P != 0).transpose(0, 2, 1))
    M = I.keldysh_batch(2, 5)
    assert M.shape == (2, 10, 10) and M.dtype == np.complex128


# --- XNOR minors (Section III.B) and the Nambu CDet weights (Section V.B) ----

def _xnor_idx(S, n):
    return [2 * v + e for v in range(n) if (S >> v) & 1 for e in (0, 1)]


def test_xnor_minors_match_numpy_determinants():
    """Each XNOR minor is the determinant of the rows and columns 2i, 2i+1 of
    the vertices in S (numpy's LAPACK determinant as the independent check)."""
    rng = np.random.default_rng(2001)
    for n in (1, 3, 5):
        M = rng.standard_normal((3, 2 * n, 2 * n)) + 1.5 * np.eye(2 * n)
        x = oracle.xnor_minors(M)
        for b in range(3):
            assert x[b, 0] == 1.0
            for S in range(1, 1 << n):
                idx = _xnor_idx(S, n)
                ref = np.linalg.det(M[b][np.ix_(idx, idx)])
                assert abs(x[b, S] - ref) <= 1e-12 * max(1.0, abs(ref)), (n, S)


def test_xnor_block_diagonal_closed_form():
    """Only diagonal 2 x 2 blocks: every XNOR minor is the product of the block
    determinants of its vertices."""
    rng = np.random.default_rng(2002)
    n = 6
    B = rng.standard_normal((n, 2, 2))
    M = np.zeros((2 * n, 2 * n))
    for i in range(n):
        M[2 * i:2 * i + 2, 2 * i:2 * i + 2] = B[i]
    d = B[:, 0, 0] * B[:, 1, 1] - B[:, 0, 1] * B[:, 1, 0]
    x = oracle.xnor_minors(M)
    for S in range(1 << n):
        ref = np.prod([d[v] for v in range(n) if (S >> v) & 1])
        assert abs(x[S] - ref) <= 1e-13 * max(1.0, abs(ref))


def test_xnor_without_pairing_factorises():
    """Delta = 0: the Nambu matrix has no particle-hole mixing, so the XNOR
    minor is det G_00[S] * det G_11[S] (the rows and columns of each component
    reordered together, no sign)."""
    G = I.nambu_g0_table(delta=0.0)
    x_, y_, m_ = I.hubbard_vertices(2, 7, seed=2003, mtau=I.NAMBU_MTAU)
    dx = np.abs(x_[:, :, None] - x_[:, None, :])
    dy = np.abs(y_[:, :, None] - y_[:, None, :])
    dt = m_[:, :, None] - m_[:, None, :] + (I.NAMBU_MTAU - 1)
    blocks = G[dx, dy, dt]
    assert np.all(blocks[..., 0, 1] == 0.0)
    M = blocks.transpose(0, 1, 3, 2, 4).reshape(2, 14, 14)
    x = oracle.xnor_minors(M)
    for b in range(2):
        for S in range(1, 1 << 7):
            idx = [v for v in range(7) if (S >> v) & 1]
            ref = (np.linalg.det(blocks[b, :, :, 0, 0][np.ix_(idx, idx)])
                   * np.linalg.det(blocks[b, :, :, 1, 1][np.ix_(idx, idx)]))
            assert abs(x[b, S] - ref) <= 1e-12 * max(1e-3, abs(ref))


def test_xnor_leibniz_order_2():
    """n = 2: the full 4 x 4 minor as the Leibniz sum over all 24 permutations."""
    import itertools
    rng = np.random.default_rng(2004)
    M = rng.standard_normal((4, 4))
    total = 0.0
    for p in itertools.permutations(range(4)):
        sgn = 1
        for i in range(4):
            for j in range(i + 1, 4):
                if p[i] > p[j]:
                    sgn = -sgn
        total += sgn * np.prod([M[i, p[i]] for i in range(4)])
    x = oracle.xnor_minors(M)
    assert abs(x[3] - total) <= 1e-13 * max(1.0, abs(total))
    assert abs(x[1] - (M[0, 0] * M[1, 1] - M[0, 1] * M[1, 0])) <= 1e-15


def test_xnor_scale_bounds():
    rng = np.random.default_rng(2005)
    M = rng.standard_normal((2, 10, 10))
    x = oracle.xnor_minors(M)
    sp = oracle.xnor_scale(M, use_perm=True)
    sb = oracle.xnor_scale(M, use_perm=False)
    assert np.all(np.abs(x) <= sp * (1 + 1e-12))
    assert np.all(sp <= sb * (1 + 1e-12))
    assert np.all(sp[:, 0] == 1.0)


# --- NAND minors (Section III.C) and two-vertex-type weights (Section V.C) ----

def _tern(t, n):
    return [(t // 3 ** v) % 3 for v in range(n)]


def test_nand_minors_match_numpy_determinants():
    rng = np.random.default_rng(2101)
    for n in (1, 2, 4):
        M = rng.standard_normal((2 * n, 2 * n)) + np.eye(2 * n)
        ab, sc, m3 = oracle.nand(M, minors=True)
        assert m3[0] == 1.0 and ab[0] == 1.0
        for t in range(1, 3 ** n):
            idx = [2 * v + d - 1 for v, d in enumerate(_tern(t, n)) if d]
            ref = np.linalg.det(M[np.ix_(idx, idx)])
            assert abs(m3[t] - ref) <= 1e-12 * max(1.0, abs(ref)), (n, t)
        assert np.all(np.abs(ab) <= sc * (1 + 1e-12))


def test_nand_type_sums_are_real_keldysh_sums():
    """For every subset S, abar[S] is the sum over the 2^|S| type assignments of
    the kept minors, i.e. the XOR sum of Section III.D of the block matrix
    restricted to S: the independent complex route of the Keldysh oracle."""
    rng = np.random.default_rng(2102)
    n = 5
    M = rng.standard_normal((2 * n, 2 * n)) + np.eye(2 * n)
    ab, _ = oracle.nand(M)
    for S in (0b11111, 0b10101, 0b00110, 0b01000):
        vs = [v for v in range(n) if (S >> v) & 1]
        rows = [2 * v + e for v in vs for e in (0, 1)]
        ref = oracle.keldysh(M[np.ix_(rows, rows)].astype(np.complex128))
        assert abs(ab[S] - ref.real) <= 1e-12 * max(1.0, abs(ref)) and abs(ref.imag) == 0.0


def test_nand_block_diagonal_and_equal_types():
    rng = np.random.default_rng(2103)
    n = 5
    B = rng.standard_normal((n, 2, 2))
    M = np.zeros((2 * n, 2 * n))
    for i in range(n):
        M[2 * i:2 * i + 2, 2 * i:2 * i + 2] = B[i]
    ab, _, m3 = oracle.nand(M, minors=True)
    for t in range(3 ** n):
        ref = np.prod([B[v, d - 1, d - 1] for v, d in enumerate(_tern(t, n)) if d])
        assert abs(m3[t] - ref) <= 1e-14 * max(1.0, abs(ref))
    for S in range(1 << n):
        ref = np.prod([B[v, 0, 0] + B[v, 1, 1] for v in range(n) if (S >> v) & 1])
        assert abs(ab[S] - ref) <= 1e-13 * max(1.0, abs(ref))
    # both types of every vertex identical: each of the 2^|S| minors is det g[S]
    g = rng.standard_normal((n, n)) + 2 * np.eye(n)
    ab2, _ = oracle.nand(np.kron(g, np.ones((2, 2))))
    for S in range(1, 1 << n):
        vs = [v for v in range(n) if (S >> v) & 1]
        ref = 2 ** len(vs) * np.linalg.det(g[np.ix_(vs, vs)])
        assert abs(ab2[S] - ref) <= 1e-12 * max(1.0, abs(ref))


def test_two_type_inputs_conventions():
    M = I.two_type_batch(2, 6, seed=2104)
    assert M.shape == (2, 12, 12)
    # type-2 of a vertex is its type-1 copy shifted by one site at the same time
    G = I.hubbard_g0_table(win=I.HUB_WIN + 1)
    assert np.allclose(M[:, 0, 1], G[1, 0, I.HUB_MTAU - 1])
    assert np.allclose(np.diagonal(M, axis1=1, axis2=2), G[0, 0, I.HUB_MTAU - 1])


# --- two-spin Keldysh sums (Section V.D with Eq. CTINT) -------------------------

def test_keldysh2_vs_numpy_bruteforce():
    rng = np.random.default_rng(2201)
    for n in (1, 3, 5):
        Mu = rng.standard_normal((2 * n, 2 * n)) + 1j * rng.standard_normal((2 * n, 2 * n))
        Md = rng.standard_normal((2 * n, 2 * n)) + 1j * rng.standard_normal((2 * n, 2 * n))
        for signed in (False, True):
            ref = 0.0
            for al in itertools.product([0, 1], repeat=n):
                idx = [2 * i + a for i, a in enumerate(al)]
                v = np.linalg.det(Mu[np.ix_(idx, idx)]) * np.linalg.det(Md[np.ix_(idx, idx)])
                ref += -v if (signed and sum(al) % 2) else v
            got = oracle.keldysh2(Mu, Md, signed=signed)
            assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (n, signed)


def test_keldysh2_identity_partner_is_single_spin_sum():
    """With the identity as the second matrix every M_dn,alpha is the identity,
    so the two-spin sum is the (independently pinned) single-spin Keldysh sum."""
    Mu = I.keldysh_batch(2, 6, seed=2202)
    Md = np.broadcast_to(np.eye(12, dtype=np.complex128), Mu.shape).copy()
    for signed in (False, True):
        a = oracle.keldysh2(Mu, Md, signed=signed)
        b = oracle.keldysh(Mu, signed=signed)
        assert np.all(np.abs(a - b) <= 1e-12 * np.maximum(1.0, np.abs(b)))


def test_keldysh2_equal_blocks_and_largest_time():
    rng = np.random.default_rng(2203)
    n = 6
    gu = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.eye(n)
    gd = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)) + 3 * np.eye(n)
    s = oracle.keldysh2(np.kron(gu, np.ones((2, 2))), np.kron(gd, np.ones((2, 2))))
    ref = 2 ** n * np.linalg.det(gu) * np.linalg.det(gd)
    assert abs(s - ref) <= 1e-11 * abs(ref)
    # causal contour: both rows of the latest vertex agree in each spin, so the
    # sign-weighted sum over the shared assignment vanishes
    Mu, Md = I.keldysh2_batch(3, 7, seed=2204)
    sg = oracle.keldysh2(Mu, Md, signed=True)
    assert np.all(np.abs(sg) <= 1e-12 * oracle.keldysh2_scale(Mu, Md))


def test_keldysh2_partial_sums_are_leading_blocks():
    Mu, Md = I.keldysh2_batch(2, 5, seed=2205)
    s, p = oracle.keldysh2(Mu, Md, partial=True)
    assert np.all(p[:, 0] == 1.0) and np.array_equal(p[:, 5], s)
    for d in range(1, 5):
        ref = oracle.keldysh2(Mu[:, :2 * d, :2 * d], Md[:, :2 * d, :2 * d])
        assert np.all(np.abs(p[:, d] - ref) <= 1e-13 * np.maximum(1.0, np.abs(ref)))
