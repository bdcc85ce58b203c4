"""The benchmark's second CPU baseline (the paper's depth-first tree with pivot
correction and the CDet recursion, cpu_baseline/) against the oracle: minors
within 1e-10 of perm(|A[S]|) (the sum of the absolute values of the Leibniz
terms), connected sums within 1e-10 of the recursion run on those scales."""
import numpy as np
import pytest

import cpu_baseline
import oracle

TOL = 1e-10


def check(A, thr=cpu_baseline.DEFAULT_PIV_THRESHOLD, expect_corrected=None):
    m, c, st = cpu_baseline.fpm_sc(A, nthreads=2, piv_threshold=thr)
    mref = oracle.minors_lu(A)
    mscale = oracle.minors_scale(A)
    assert np.all(np.abs(m - mref) <= TOL * mscale)
    cref = oracle.cdet_recursion(mref * mref)
    cscale = oracle.cdet_scale(mscale * mscale)
    assert np.all(np.abs(c - cref) <= TOL * np.maximum(cscale, 1e-300))
    assert np.all((st & 2) == 0)
    if expect_corrected is not None:
        assert bool(np.all(st & 1)) == expect_corrected


@pytest.mark.parametrize("n", [1, 2, 5, 8, 10])
def test_random_matrices(n):
    rng = np.random.default_rng(6000 + n)
    check(rng.standard_normal((4, n, n)) + 2.0 * np.eye(n), expect_corrected=False)


@pytest.mark.parametrize("n", [4, 7, 10])
def test_zero_diagonal_and_nested_corrections(n):
    """A zero diagonal forces a correction at the first node of every level;
    a threshold of 0.7 ||A||max corrects most pivots, nested in one another."""
    rng = np.random.default_rng(6100 + n)
    A = rng.standard_normal((3, n, n))
    for b in range(3):
        np.fill_diagonal(A[b], 0.0)
    check(A, expect_corrected=True)
    check(rng.standard_normal((3, n, n)), thr=0.7, expect_corrected=True)


def test_hubbard_rows_and_empty_set():
    from paper_2104_07638_gb300 import inputs
    A = inputs.hubbard_batch(6, 12, seed=2)
    check(A)
    m, c, _ = cpu_baseline.fpm_sc(A[:1])
    assert m[0, 0] == 1.0 and c[0, 0] == 0.0
