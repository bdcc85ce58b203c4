"""Parity of the CUDA two-spin Keldysh sum (Section V.D with Eq. CTINT) with the
CPU oracle (two complex eliminations per shared assignment). Tolerance: 1e-10
times the sum over the assignments of the products of the two row-sum bounds."""
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


def check(apm, Mu, Md, signed=False, partial=True):
    scale = oracle.keldysh2_scale(Mu, Md)
    if partial:
        s, p, st = apm.keldysh2_sum(dev(Mu), dev(Md), signed=signed, partial=True, return_status=True)
        sref, pref = oracle.keldysh2(Mu, Md, signed=signed, partial=True)
        p = p.cpu().numpy()
        n = Mu.shape[-1] // 2
        assert np.all(p[:, 0] == 1.0)
        assert np.array_equal(p[:, n], s.cpu().numpy())
        assert float(np.max(np.abs(p - pref) / scale[:, None])) <= TOL
    else:
        s, st = apm.keldysh2_sum(dev(Mu), dev(Md), signed=signed, return_status=True)
        sref = oracle.keldysh2(Mu, Md, signed=signed)
    err = float(np.max(np.abs(s.cpu().numpy() - sref) / scale))
    assert err <= TOL, err
    assert int(st.cpu().numpy().max()) == 0


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_random_complex_pairs(apm, n):
    """Orders on both sides of the 6-vertex tail: breadth first only (n <= 6),
    one and two depth-first levels (n = 7, 8; the stack from n = 8)."""
    rng = np.random.default_rng(5000 + n)
    shape = (4, 2 * n, 2 * n)
    Mu = rng.standard_normal(shape) + 1j * rng.standard_normal(shape) + 2.0 * np.eye(2 * n)
    Md = rng.standard_normal(shape) + 1j * rng.standard_normal(shape) + 2.0 * np.eye(2 * n)
    for signed in (False, True):
        check(apm, Mu, Md, signed=signed)


@pytest.mark.parametrize("n", [9, 12])
def test_chain_pairs(apm, n):
    Mu, Md = I.keldysh2_batch(3, n, seed=5100 + n)
    check(apm, Mu, Md, partial=n <= 9)


def test_order_14_against_oracle(apm):
    Mu, Md = I.keldysh2_batch(1, 14, seed=5114)
    check(apm, Mu, Md, partial=False)


def test_order_16_identity_partner_is_single_spin_sum(apm):
    """With the identity as the down-spin matrix, every down determinant is 1:
    the two-spin sum is the single-spin sum of the up matrix (another kernel)."""
    Mu, _ = I.keldysh2_batch(2, 16, seed=5116)
    Md = np.broadcast_to(np.eye(32, dtype=np.complex128), Mu.shape).copy()
    a = apm.keldysh2_sum(dev(Mu), dev(Md)).cpu().numpy()
    b = apm.keldysh_sum(dev(Mu)).cpu().numpy()
    scale = oracle.keldysh_scale(Mu, use_perm=False)
    assert np.all(np.abs(a - b) <= TOL * scale)


@pytest.mark.parametrize("n", [10, 14])
def test_largest_time_identity(apm, n):
    """Causal contour: both rows of the latest vertex agree in each spin, so the
    sign-weighted sum over the shared assignments vanishes."""
    Mu, Md = I.keldysh2_batch(32, n, seed=5200 + n)
    s = apm.keldysh2_sum(dev(Mu), dev(Md), signed=True).cpu().numpy()
    assert np.all(np.abs(s) <= TOL * oracle.keldysh2_scale(Mu, Md))


def test_zero_pivot_flagged(apm):
    n = 5
    Mu, Md = I.keldysh2_batch(3, n, seed=5300)
    Md[1, 0, 0] = 0.0                      # down spin, vertex 0, index +: a pivot of the root
    s, st = apm.keldysh2_sum(dev(Mu), dev(Md), return_status=True)
    st, s = st.cpu().numpy(), s.cpu().numpy()
    assert st[1] & apm.ST_ZERO_PIVOT and st[0] == 0 and st[2] == 0
    assert np.isnan(s[1]) and np.isfinite(s[0]) and np.isfinite(s[2])


def test_bench_size_sampled_and_deterministic(apm):
    """The launch the benchmark times (16384 chain pairs of order 12), sampled
    pairs against the oracle, and two calls bit for bit equal."""
    Mu, Md = I.keldysh2_batch(16384, 12, seed=8)
    du, dd = dev(Mu), dev(Md)
    a = apm.keldysh2_sum(du, dd)
    b = apm.keldysh2_sum(du, dd)
    assert torch.equal(a, b)
    idx = [0, 9999, 16383]
    ref = oracle.keldysh2(Mu[idx], Md[idx])
    assert np.all(np.abs(a[idx].cpu().numpy() - ref) <= TOL * oracle.keldysh2_scale(Mu[idx], Md[idx]))
