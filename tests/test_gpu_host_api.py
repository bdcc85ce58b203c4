"""The host-memory entry apm_cdet_connected_host: the same outputs as the
device call apm_cdet_connected, bit for bit (the same kernels on the same
matrices), for page-locked and pageable host buffers, ragged last chunks, odd
chunk offsets, one and several streams, two matrices per configuration and the
order-16 hand-off to the fast subset convolution; sampled rows against the CPU
oracle (tolerance 1e-10 times the sum of the absolute values of the terms, as
for the device call)."""
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


def host(x, pinned):
    t = torch.as_tensor(np.ascontiguousarray(x))
    return t.pin_memory() if pinned else t


@pytest.mark.parametrize("n,batch,chunk,nstreams,pinned", [
    (10, 1000, 96, 3, True),      # 10 full chunks and a ragged one of 40
    (12, 700, 128, 4, True),
    (7, 300, 37, 2, True),        # odd chunk x odd n: host offsets not 16-byte aligned
    (8, 33, 1000, 2, False),      # chunk above the batch, pageable memory
    (5, 257, 16, 8, False),
    (6, 100, 10, 1, True),        # one stream
])
def test_host_equals_device(apm, n, batch, chunk, nstreams, pinned):
    A = I.hubbard_batch(batch, n, seed=5100 + n)
    c_h, m_h, st_h = apm.cdet_connected_host(host(A, pinned), return_minors=True, return_status=True,
                                             chunk=chunk, nstreams=nstreams)
    assert c_h.device.type == "cpu" and c_h.is_pinned() == pinned
    c_d, m_d, st_d = apm.cdet_connected(torch.as_tensor(A).cuda(), return_minors=True, return_status=True)
    assert torch.equal(c_h, c_d.cpu()) and torch.equal(m_h, m_d.cpu()) and torch.equal(st_h, st_d.cpu())
    idx = [0, batch // 2, batch - 1]
    mref = oracle.minors_lu(A[idx])
    mscale = oracle.minors_scale(A[idx])
    assert np.all(np.abs(m_h.numpy()[idx] - mref) <= TOL * mscale)
    cref = oracle.cdet_recursion(mref * mref)
    cscale = oracle.cdet_scale(mscale * mscale)
    assert np.all(np.abs(c_h.numpy()[idx] - cref) <= TOL * np.maximum(cscale, 1e-300))


def test_host_two_matrices_and_single_det(apm):
    n, batch = 9, 301
    Au = I.hubbard_batch(batch, n, seed=5200)
    Ad = I.hubbard_batch(batch, n, seed=5201)
    c_d, m_d = apm.cdet_connected(torch.as_tensor(Au).cuda(), torch.as_tensor(Ad).cuda(), return_minors=True)
    c_h, m_h = apm.cdet_connected_host(host(Au, True), host(Ad, True), return_minors=True, chunk=50,
                                       nstreams=4)
    assert torch.equal(c_h, c_d.cpu()) and torch.equal(m_h, m_d.cpu())
    assert m_h.shape == (batch, 2, 1 << n)
    c1 = apm.cdet_connected_host(host(Au, False), single_det=True, chunk=64, nstreams=2)
    c2 = apm.cdet_connected(torch.as_tensor(Au).cuda(), single_det=True)
    assert torch.equal(c1, c2.cpu())


def test_host_order_16_fast_subset_convolution(apm):
    """Order 16 goes through the workspace scratch and the in-place fast subset
    convolution of every chunk."""
    A = I.hubbard_batch(12, 16, seed=5300)
    c_d = apm.cdet_connected(torch.as_tensor(A).cuda())
    c_h = apm.cdet_connected_host(host(A, True), chunk=5, nstreams=2)
    assert torch.equal(c_h, c_d.cpu())


def test_host_caller_workspace_and_empty_batch(apm):
    n, batch, chunk, ns = 11, 200, 64, 4
    A = I.hubbard_batch(batch, n, seed=5400)
    nb = apm.cdet_connected_host_workspace_size(n, chunk, ns)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    out = torch.empty((batch, 1 << n), dtype=torch.float64).pin_memory()
    c = apm.cdet_connected_host(host(A, True), out_c=out, chunk=chunk, nstreams=ns, workspace=ws)
    assert c.data_ptr() == out.data_ptr()
    assert torch.equal(c, apm.cdet_connected(torch.as_tensor(A).cuda()).cpu())
    small = torch.empty(nb - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(apm.ApmError) as e:
        apm.cdet_connected_host(host(A, True), chunk=chunk, nstreams=ns, workspace=small)
    assert e.value.code == apm.APM_ERR_WORKSPACE
    empty = torch.empty((0, n, n), dtype=torch.float64)
    assert apm.cdet_connected_host(empty).shape == (0, 1 << n)
