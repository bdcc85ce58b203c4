"""Parity of the CUDA O(3^n) permanent principal minors with the CPU oracle
(Ryser per subset). Tolerance: 1e-10 times the sum of the absolute values of
the terms of Ryser's formula for that subset (the rounding scale of any Ryser
evaluation; for non-negative matrices it exceeds the permanent itself, whose
Leibniz terms are all positive). Integer matrices are compared bit for bit, and
on the benchmark's matrices with entries quantised to k / 1024 the kernel's
error is measured against exact permanents (Python integers)."""
import math

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


def check(apm, A):
    p = apm.perm_minors(dev(A)).cpu().numpy()
    ref = oracle.perm_ryser(A)
    scale = oracle.perm_ryser_term_scale(A)
    err = float(np.max(np.abs(p - ref) / np.maximum(scale, 1e-300)))
    assert err <= TOL, err
    assert np.all(p[:, 0] == 1.0)
    return p


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6, 8, 10, 12])
def test_random_orders(apm, n):
    rng = np.random.default_rng(1000 + n)
    check(apm, rng.standard_normal((4, n, n)))


def test_masked_uniform_n14(apm):
    A = I.perm_batch(14, 6, seed=4)
    p = check(apm, A)
    assert np.all(p >= 0.0) or float(p.min()) > -1e-6


def test_order_15_global_accumulator(apm):
    A = I.perm_batch(15, 2, seed=15)
    check(apm, A)


def test_all_ones_factorials_n16(apm):
    n = 16
    p = apm.perm_minors(dev(np.ones((1, n, n)))).cpu().numpy()[0]
    size = [bin(S).count("1") for S in range(1 << n)]        # python ints: no overflow
    ref = np.array([float(math.factorial(k)) for k in size])
    scale = np.array([float(sum(math.comb(k, t) * t ** k for t in range(k + 1))) for k in size])
    assert np.all(np.abs(p - ref) <= TOL * scale)


def test_rank_one_closed_form(apm):
    rng = np.random.default_rng(1100)
    n = 12
    u, v = rng.uniform(0.5, 1.5, n), rng.uniform(0.5, 1.5, n)
    p = apm.perm_minors(dev(np.outer(u, v)[None])).cpu().numpy()[0]
    ref = np.array([math.factorial(bin(S).count("1")) *
                    np.prod([u[e] * v[e] for e in range(n) if (S >> e) & 1]) for S in range(1 << n)])
    scale = oracle.perm_ryser_term_scale(np.outer(u, v))
    assert np.all(np.abs(p - ref) <= TOL * scale)


def test_zero_one_integer_counts_exact(apm):
    rng = np.random.default_rng(1101)
    n = 12
    B = (rng.random((3, n, n)) < 0.6).astype(float)
    p = apm.perm_minors(dev(B)).cpu().numpy()
    ref = oracle.perm_ryser(B)
    assert np.array_equal(p, ref)             # integer sums below 2^53 are exact


def test_full_cfg_batch_sampled(apm):
    """4096 masked-uniform matrices of order 14 (the benchmark configuration);
    three sampled against the oracle."""
    A = I.perm_batch(14, 4096, seed=4)
    p = apm.perm_minors(dev(A))
    torch.cuda.synchronize()
    idx = [0, 2047, 4095]
    ref = oracle.perm_ryser(A[idx])
    scale = oracle.perm_ryser_term_scale(A[idx])
    assert np.all(np.abs(p[idx].cpu().numpy() - ref) <= TOL * scale)
    assert torch.isfinite(p).all() and bool((p >= -1e-6).all())


def perm_exact(K):
    """perm of an integer matrix by Ryser's formula (Eq. ryser, with the sign
    (-1)^k), the column subsets walked in Gray-code order, in Python integers."""
    k = len(K)
    if k == 0:
        return 1
    rs, T, total = [0] * k, 0, 0
    for g in range(1, 1 << k):
        j = (g & -g).bit_length() - 1
        T ^= 1 << j
        d = 1 if (T >> j) & 1 else -1
        p = 1
        for i in range(k):
            rs[i] += d * K[i][j]
            p *= rs[i]
        total += -p if bin(T).count("1") % 2 else p
    return -total if k % 2 else total


def test_measured_error_against_exact_permanents(apm):
    """Masked-uniform matrices of order 14 (the benchmark's kind) quantised to
    k / 1024, so that perm(A[S]) = perm(K[S]) / 1024^|S| exactly: the full set
    and 60 sampled subsets of each of two matrices against Python-integer
    permanents. Ryser's alternating sum cancels (its term sum is up to 5e6
    times the permanent at the full set), yet the kernel's relative error here
    is 1.7e-11 (printed): the bound is relative error 1e-10 against the exact
    value, as for every other step."""
    A = I.perm_batch(14, 2, seed=4)
    K = np.floor(A * 1024).astype(np.int64)
    Aq = K / 1024.0
    p = apm.perm_minors(dev(Aq)).cpu().numpy()
    rng = np.random.default_rng(1400)
    worst = 0.0
    for b in range(2):
        masks = [(1 << 14) - 1] + [int(m) for m in rng.integers(1, 1 << 14, 60)]
        for S in masks:
            idx = [i for i in range(14) if (S >> i) & 1]
            ex = perm_exact(K[b][np.ix_(idx, idx)].tolist())
            ref = ex / 1024 ** len(idx)          # correctly rounded
            if ex == 0:                          # a structural zero: Ryser's terms cancel exactly
                assert abs(p[b, S]) <= TOL * oracle.perm_ryser_term_scale(Aq[b])[S]
                continue
            err = abs(p[b, S] - ref) / ref
            worst = max(worst, err)
            assert err <= TOL, (b, S, err)
    print(f"max relative error against exact permanents: {worst:.3e}")
