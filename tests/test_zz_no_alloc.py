"""apm_keldysh_sum_noalloc, the entry point for callers that cannot allocate
device memory around the call (their own pool allocator owns the device, or a
plugin host only hands in device pointers): its results must match the
allocating apm_keldysh_sum within the Keldysh parity tolerance, on two calls in
a row (the second call reuses the library's array as the first left it).

The file is named so that pytest collects it last."""
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


@pytest.mark.parametrize("n,batch", [(9, 1500), (12, 1200), (14, 700)])
def test_noalloc_matches_workspace_entry_point_twice(apm, n, batch):
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


def test_noalloc_rejects_orders_above_its_limit(apm):
    Mt = torch.zeros((1, 30, 30), dtype=torch.complex128, device="cuda")
    with pytest.raises(apm.ApmError) as ei:
        apm.keldysh_sum_noalloc(Mt)
    assert ei.value.code == apm.APM_ERR_UNSUPPORTED_N
