"""Every entry point on an empty batch: no launch, no error, outputs of the
right shape with no rows (the C functions return APM_OK before any launch when
batch == 0)."""
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_07638_gb300 import apm as m
    m.lib()
    return m


def empty(*shape, dtype=torch.float64):
    return torch.empty((0,) + shape, dtype=dtype, device="cuda")


@pytest.mark.parametrize("n", [4, 8, 12, 14, 20])
def test_all_minors(apm, n):
    m, st = apm.all_minors(empty(n, n), return_status=True)
    assert m.shape == (0, 1 << n) and st.numel() == 0


@pytest.mark.parametrize("n", [6, 12, 16])
def test_connected_sums(apm, n):
    c, mo = apm.cdet_connected(empty(n, n), return_minors=True)
    assert c.shape == (0, 1 << n) and mo.shape[0] == 0
    assert apm.cdet_from_weights(empty(1 << n)).shape == (0, 1 << n)
    assert apm.cdet_from_weights_fsc(empty(1 << n)).shape == (0, 1 << n)


def test_permanents(apm):
    assert apm.perm_minors(empty(14, 14)).shape == (0, 1 << 14)


@pytest.mark.parametrize("n", [5, 12])
def test_keldysh_sums(apm, n):
    s = apm.keldysh_sum(empty(2 * n, 2 * n, dtype=torch.complex128))
    assert s.shape[0] == 0
    s2 = apm.keldysh2_sum(empty(2 * n, 2 * n, dtype=torch.complex128), empty(2 * n, 2 * n, dtype=torch.complex128))
    assert s2.shape[0] == 0


def test_keldysh_noalloc(apm):
    s = apm.keldysh_sum_noalloc(empty(24, 24, dtype=torch.complex128))
    assert s.shape[0] == 0


@pytest.mark.parametrize("n", [3, 12])
def test_nambu_and_two_type(apm, n):
    assert apm.xnor_minors(empty(2 * n, 2 * n)).shape == (0, 1 << n)
    assert apm.nambu_cdet(empty(2 * n, 2 * n)).shape == (0, 1 << n)
    assert apm.two_type_cdet(empty(2 * n, 2 * n)).shape == (0, 1 << n)
    if n <= 10:
        assert apm.nand_minors(empty(2 * n, 2 * n)).shape == (0, 3 ** n)


def test_uneven_batches(apm):
    n = torch.empty(0, dtype=torch.int32, device="cuda")
    off = torch.empty(0, dtype=torch.int64, device="cuda")
    c = apm.cdet_connected_varlen(empty(), off, n, n_max=12)
    assert c.numel() == 0
    s = apm.keldysh_sum_varlen(empty(dtype=torch.complex128), off, n, n_max=12)
    assert s.shape[0] == 0
