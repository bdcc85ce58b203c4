"""Parity of the CUDA XNOR minors and the Nambu CDet (Sections III.B, V.B) with
the CPU oracle (one elimination per kept submatrix; the CDet recursion on
those minors). Tolerance: 1e-10 times the sum of the absolute Leibniz terms of
each minor (perm of the absolute submatrix for n <= 8, else the row-sum
bound); for c, the recursion run on those scales with all signs positive."""
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


def check_minors(apm, M):
    x, st = apm.xnor_minors(dev(M), return_status=True)
    x = x.cpu().numpy()
    ref = oracle.xnor_minors(M)
    scale = oracle.xnor_scale(M)
    err = float(np.max(np.abs(x - ref) / scale))
    assert err <= TOL, err
    assert int(st.cpu().numpy().max()) == 0
    assert np.all(x[:, 0] == 1.0)
    return x


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11])
def test_random_matrices(apm, n):
    """Orders on both sides of the 8-vertex tail: breadth first only (n <= 8),
    one and two depth-first levels (n = 9, 10; the stack from n = 10)."""
    rng = np.random.default_rng(3000 + n)
    M = rng.standard_normal((5, 2 * n, 2 * n)) + 1.5 * np.eye(2 * n)
    check_minors(apm, M)


@pytest.mark.parametrize("n", [6, 9, 12])
def test_nambu_propagator_matrices(apm, n):
    check_minors(apm, I.nambu_batch(4, n, seed=3100 + n))


def test_order_16_against_oracle(apm):
    check_minors(apm, I.nambu_batch(1, 16, seed=3116))


@pytest.mark.parametrize("n", [5, 9, 12])
def test_nambu_cdet_against_oracle(apm, n):
    M = I.nambu_batch(3, n, seed=3200 + n)
    c, x = apm.nambu_cdet(dev(M), return_minors=True)
    c, x = c.cpu().numpy(), x.cpu().numpy()
    xr = oracle.xnor_minors(M)
    cr = oracle.cdet_recursion(xr)
    cs = oracle.cdet_scale(oracle.xnor_scale(M))
    assert np.all(np.abs(x - xr) <= TOL * oracle.xnor_scale(M))
    assert np.all(np.abs(c - cr) <= TOL * np.maximum(cs, 1e-300))
    assert np.all(c[:, 0] == 0.0)


def test_nambu_cdet_equals_recursion_on_device_minors(apm):
    """The connected sums are the recursion of apm_cdet_from_weights on the
    same minors, bit for bit (same kernel, same weights)."""
    M = dev(I.nambu_batch(64, 10, seed=3300))
    c, x = apm.nambu_cdet(M, return_minors=True)
    c2 = apm.cdet_from_weights(x)
    assert torch.equal(c, c2)


def test_singular_pivot_flagged(apm):
    n = 6
    M = I.nambu_batch(3, n, seed=3400)
    M[1, 2 * n - 2:, 2 * n - 2:] = 0.0       # last vertex's diagonal block: the first pivot
    x, st = apm.xnor_minors(dev(M), return_status=True)
    st, x = st.cpu().numpy(), x.cpu().numpy()
    assert st[1] & apm.ST_ZERO_PIVOT and st[0] == 0 and st[2] == 0
    assert np.all(np.isnan(x[1])) and np.all(np.isfinite(x[0])) and np.all(np.isfinite(x[2]))


def test_nonfinite_input_flagged(apm):
    M = I.nambu_batch(2, 9, seed=3401)
    M[0, 3, 5] = np.inf
    x, st = apm.xnor_minors(dev(M), return_status=True)
    st = st.cpu().numpy()
    assert st[0] & apm.ST_NONFINITE_INPUT and st[1] == 0
    assert np.all(np.isnan(x[0].cpu().numpy()))


def test_bench_size_sampled_and_deterministic(apm):
    """The launch the benchmark times (65536 Nambu matrices of order 12),
    sampled rows against the oracle, and two calls bit for bit equal."""
    M = I.nambu_batch(65536, 12, seed=6)
    Md = dev(M)
    c1, x1 = apm.nambu_cdet(Md, return_minors=True)
    c2 = apm.nambu_cdet(Md)
    assert torch.equal(c1, c2)
    idx = [0, 777, 40000, 65535]
    xr = oracle.xnor_minors(M[idx])
    sc = oracle.xnor_scale(M[idx])
    assert np.all(np.abs(x1[idx].cpu().numpy() - xr) <= TOL * sc)
    cr = oracle.cdet_recursion(xr)
    cs = oracle.cdet_scale(sc)
    assert np.all(np.abs(c1[idx].cpu().numpy() - cr) <= TOL * np.maximum(cs, 1e-300))
