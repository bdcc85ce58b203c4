"""Parity of the connected sums by the fast subset convolution (Section V.A:
Eq. recursion evaluated in O(n^2 2^n)) with the CPU oracle's recursion, and
with the direct O(3^n) kernel. Tolerance: 1e-10 times the recursion run on
the absolute weights' bounds with all signs positive (as for the recursion)."""
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


def weights(A, single=False):
    m = oracle.minors_lu(A)
    s = oracle.minors_rowsum_bound(A)
    return (m, s) if single else (m * m, s * s)


def check(apm, a, ahat):
    c = apm.cdet_from_weights_fsc(torch.as_tensor(a).cuda()).cpu().numpy()
    cref = oracle.cdet_recursion(a)
    scale = np.maximum(oracle.cdet_scale(ahat), 1e-300)
    err = float(np.max(np.abs(c - cref) / scale))
    assert err <= TOL, err
    assert np.all(c[:, 0] == 0.0)
    return c


@pytest.mark.parametrize("n", list(range(1, 17)))
def test_hubbard_weights_all_orders(apm, n):
    """One tile (n <= 9) and the three passes through the workspace (n >= 10,
    one to seven high elements)."""
    A = I.hubbard_batch(3 if n <= 12 else 1, n, seed=7000 + n)
    check(apm, *weights(A))


@pytest.mark.parametrize("n", [4, 9, 10, 13])
def test_signed_single_determinant_weights(apm, n):
    rng = np.random.default_rng(7100 + n)
    A = rng.standard_normal((2, n, n)) + 2.0 * np.eye(n)
    check(apm, *weights(A, single=True))


def test_matches_direct_recursion_kernel(apm):
    A = I.hubbard_batch(512, 12, seed=7200)
    a, ahat = weights(A)
    ad = torch.as_tensor(a).cuda()
    c1 = apm.cdet_from_weights_fsc(ad).cpu().numpy()
    c2 = apm.cdet_from_weights(ad).cpu().numpy()
    assert np.all(np.abs(c1 - c2) <= TOL * oracle.cdet_scale(ahat))


def test_a_empty_is_ignored_and_batch_deterministic(apm):
    A = I.hubbard_batch(700, 10, seed=7300)   # more matrices than resident CTAs: each CTA loops
    a, _ = weights(A)
    ad = torch.as_tensor(a).cuda()
    c1 = apm.cdet_from_weights_fsc(ad)
    ad2 = ad.clone()
    ad2[:, 0] = 123.0
    c2 = apm.cdet_from_weights_fsc(ad2)
    assert torch.equal(c1, c2)
    assert torch.equal(c1, apm.cdet_from_weights_fsc(ad))


def test_empty_batch(apm):
    c = apm.cdet_from_weights_fsc(torch.zeros((0, 256), dtype=torch.float64, device="cuda"))
    assert c.shape == (0, 256)


def test_bench_size_sampled(apm):
    """The launch the benchmark row times at the largest order (456 weight rows
    of order 16, every resident CTA busy): sampled rows against the oracle, and
    the direct recursion on the same weights within the tolerance."""
    A = I.hubbard_batch(456, 16, seed=9)
    ah = oracle.minors_lu(A) ** 2
    a = torch.as_tensor(ah).cuda()
    c = apm.cdet_from_weights_fsc(a)
    assert torch.equal(c, apm.cdet_from_weights_fsc(a))
    idx = [0, 455]
    cref = oracle.cdet_recursion(ah[idx])
    bound = oracle.minors_rowsum_bound(A[idx]) ** 2
    scale = np.maximum(oracle.cdet_scale(bound), 1e-300)
    assert np.all(np.abs(c[idx].cpu().numpy() - cref) <= TOL * scale)
    cd = apm.cdet_from_weights(a)
    full_scale = np.maximum(oracle.cdet_scale(oracle.minors_rowsum_bound(A) ** 2), 1e-300)
    assert np.all(np.abs(c.cpu().numpy() - cd.cpu().numpy()) <= TOL * full_scale)
