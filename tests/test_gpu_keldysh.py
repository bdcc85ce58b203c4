"""Parity of the CUDA Keldysh (XOR-minor) sum with the CPU oracle (one complex
elimination per index assignment). Tolerance: 1e-10 times the sum over
assignments of the absolute Leibniz terms (perm(|M_alpha|), n <= 10) or of the
row-sum bound prod_i sum_j |M_alpha,ij| (larger n)."""
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


def check(apm, Mt, signed=False, partial=True):
    if partial:
        s, p, st = apm.keldysh_sum(dev(Mt), signed=signed, partial=True, return_status=True)
        sref, pref = oracle.keldysh(Mt, signed=signed, partial=True)
    else:
        s, st = apm.keldysh_sum(dev(Mt), signed=signed, return_status=True)
        sref = oracle.keldysh(Mt, signed=signed)
    scale = oracle.keldysh_scale(Mt)
    s = s.cpu().numpy()
    err = float(np.max(np.abs(s - sref) / scale))
    assert err <= TOL, err
    assert int(st.cpu().numpy().max()) == 0
    if partial:
        p = p.cpu().numpy()
        n = Mt.shape[-1] // 2
        assert np.all(p[:, 0] == 1.0)
        assert np.array_equal(p[:, n], s)
        # lower orders: each partial is the sum for the leading block, whose
        # scale is at most the full one
        perr = float(np.max(np.abs(p - pref) / scale[:, None]))
        assert perr <= TOL, perr
    return s


@pytest.mark.parametrize("n", [1, 2, 3, 5, 6, 7, 8])
def test_random_complex_small_orders(apm, n):
    rng = np.random.default_rng(600 + n)
    Mt = rng.standard_normal((6, 2 * n, 2 * n)) + 1j * rng.standard_normal((6, 2 * n, 2 * n))
    Mt += 2.0 * np.eye(2 * n)
    for signed in (False, True):
        check(apm, Mt, signed=signed)


@pytest.mark.parametrize("n", [4, 9, 11, 12])
def test_chain_green_function(apm, n):
    Mt = I.keldysh_batch(5, n, seed=700 + n)
    check(apm, Mt, signed=False, partial=n <= 11)


def test_order_16_against_oracle(apm):
    Mt = I.keldysh_batch(2, 16, seed=716)
    check(apm, Mt, signed=False, partial=False)


@pytest.mark.parametrize("n", [10, 14, 16])
def test_largest_time_identity(apm, n):
    """With a causal contour G0 the two indices of the latest vertex give equal
    matrices, so the sign-weighted sum vanishes at every order."""
    Mt = I.keldysh_batch(64, n, seed=800 + n)
    s = apm.keldysh_sum(dev(Mt), signed=True).cpu().numpy()
    scale = oracle.keldysh_scale(Mt, use_perm=False)
    assert np.all(np.abs(s) <= TOL * scale)


def test_equal_blocks_closed_form(apm):
    rng = np.random.default_rng(900)
    n = 9
    g = rng.standard_normal((3, n, n)) + 1j * rng.standard_normal((3, n, n)) + 3 * np.eye(n)
    Mt = np.stack([np.kron(gb, np.ones((2, 2))) for gb in g])
    # all four entries of each 2x2 block equal g_ij: every assignment keeps one
    # copy of each row and column of g, so each of the 2^n minors is det(g)
    s = apm.keldysh_sum(dev(Mt)).cpu().numpy()
    ref = 2 ** n * np.linalg.det(g)
    assert np.all(np.abs(s - ref) <= TOL * oracle.keldysh_scale(Mt))


def test_zero_pivot_flagged(apm):
    n = 5
    Mt = I.keldysh_batch(3, n, seed=901)
    Mt[1, 0, 0] = 0.0                      # vertex 0, index +: zero pivot at the root
    s, st = apm.keldysh_sum(dev(Mt), return_status=True)
    st = st.cpu().numpy()
    s = s.cpu().numpy()
    assert st[1] & apm.ST_ZERO_PIVOT and st[0] == 0 and st[2] == 0
    assert np.isnan(s[1]) and np.isfinite(s[0]) and np.isfinite(s[2])


def test_many_matrices_and_determinism(apm):
    Mt = dev(I.keldysh_batch(3000, 9, seed=902))
    a = apm.keldysh_sum(Mt)
    b = apm.keldysh_sum(Mt)
    assert torch.equal(a, b)
    idx = [0, 1234, 2999]
    sref = oracle.keldysh(Mt[idx].cpu().numpy())
    scale = oracle.keldysh_scale(Mt[idx].cpu().numpy())
    assert np.all(np.abs(a[idx].cpu().numpy() - sref) <= TOL * scale)


@pytest.mark.parametrize("n,batch", [(13, 5), (14, 3)])
def test_small_batch_split_over_warps(apm, n, batch):
    """A batch far smaller than the number of warps is split into chunks of
    depth-first leaves per matrix; sums and every partial order must still match
    the oracle, and repeated calls must agree bit for bit."""
    Mt = I.keldysh_batch(batch, n, seed=950 + n)
    for signed in (False, True):
        check(apm, Mt, signed=signed, partial=True)
    d = dev(Mt)
    a = apm.keldysh_sum(d, partial=True)
    b = apm.keldysh_sum(d, partial=True)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
