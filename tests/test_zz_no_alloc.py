"""apm_keldysh_sum_noalloc, the entry point for callers that cannot allocate
device memory around the call (their own pool allocator owns the device, or a
plugin host only hands in device pointers): its results must match the
allocating apm_keldysh_sum within the Keldysh parity tolerance, on two calls in
a row (the second call reuses the library's array as the first left it), and
the oracle's sums directly; a call must leave the device's free memory as it
found it.

The file is named so that pytest collects it last."""
import ctypes

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


@pytest.mark.parametrize("n,batch", [(6, 900), (9, 1500), (12, 1200), (14, 700)])
def test_noalloc_matches_workspace_entry_point_twice(apm, n, batch):
    """Order 6 has no depth-first stack (every warp is handed the array's base
    address and never touches it); 9..14 use a slot of the array per warp."""
    Mt_np = I.keldysh_batch(batch, n, seed=1200 + n)
    Mt = torch.as_tensor(Mt_np).cuda()
    ref_s, ref_p = apm.keldysh_sum(Mt, partial=True)
    ref_s, ref_p = ref_s.cpu().numpy(), ref_p.cpu().numpy()
    scale = oracle.keldysh_scale(Mt_np, use_perm=False)
    for _ in range(2):
        s, p, st = apm.keldysh_sum_noalloc(Mt, partial=True, return_status=True)
        s, p = s.cpu().numpy(), p.cpu().numpy()
        assert int(st.cpu().numpy().max()) == 0
        assert np.all(np.abs(s - ref_s) <= TOL * scale)
        assert np.all(np.abs(p - ref_p) <= TOL * scale[:, None])


@pytest.mark.parametrize("signed", [False, True])
def test_noalloc_matches_oracle(apm, signed):
    """A few order-9 matrices against the oracle's 2^n separate eliminations."""
    Mt_np = I.keldysh_batch(6, 9, seed=1290)
    s = apm.keldysh_sum_noalloc(torch.as_tensor(Mt_np).cuda(), signed=signed).cpu().numpy()
    ref = oracle.keldysh(Mt_np, signed=signed)
    scale = oracle.keldysh_scale(Mt_np, use_perm=True)
    assert np.all(np.abs(s - ref) <= TOL * scale)


def test_noalloc_call_leaves_free_memory_unchanged(apm):
    """A call with batch 0 sets the entry point up (address lookup, module
    load); a later call with outputs allocated beforehand must not change the
    device's free memory or torch's allocation count."""
    L = apm.lib()
    n, b = 12, 800
    Mt = torch.as_tensor(I.keldysh_batch(b, n, seed=1291)).cuda()
    s = torch.empty((b, 2), dtype=torch.float64, device="cuda")
    p = torch.empty((b, n + 1, 2), dtype=torch.float64, device="cuda")
    st = torch.zeros(b, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call(batch):
        return L.apm_keldysh_sum_noalloc(ctypes.c_void_p(Mt.data_ptr()), n, batch, 0,
                                         ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(p.data_ptr()),
                                         ctypes.c_void_p(st.data_ptr()), stream)

    assert call(0) == apm.APM_OK
    assert call(b) == apm.APM_OK          # first launch of the kernel on this path
    torch.cuda.synchronize()
    free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
    assert call(b) == apm.APM_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert int(st.max()) == 0 and bool(torch.isfinite(s).all())


def test_noalloc_rejects_orders_above_its_limit(apm):
    Mt = torch.zeros((1, 30, 30), dtype=torch.complex128, device="cuda")
    with pytest.raises(apm.ApmError) as ei:
        apm.keldysh_sum_noalloc(Mt)
    assert ei.value.code == apm.APM_ERR_UNSUPPORTED_N
