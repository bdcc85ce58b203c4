"""The device half of the data-parallel exchange: apm_order_sums against its
definition (per order: count, sum, sum of magnitudes and sum of squares of the
whole-set connected sums c[2^m - 1]) on fixed-order and uneven batches, and the
split training step (apm_mlp_gradient, then apm_mlp_adam_step) bit for bit
against apm_mlp_train_step."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2104_07638_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_07638_gb300 import apm as m
    m.lib()
    return m


def table(vals_by_order, n_max):
    t = np.zeros((n_max + 1, 4))
    for m, v in vals_by_order.items():
        v = np.asarray(v, dtype=np.float64)
        t[m] = [v.size, v.sum(), np.abs(v).sum(), (v * v).sum()]
    return t


def test_fixed_order_sums(apm):
    A = I.hubbard_batch(3000, 10, seed=41)
    c = apm.cdet_connected(torch.as_tensor(A).cuda())
    got = apm.order_sums(c, n=10, n_max=12).cpu().numpy()
    ref = table({10: c[:, -1].cpu().numpy()}, 12)
    assert got[10, 0] == 3000 and np.all(got[:10] == 0) and np.all(got[11:] == 0)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
    again = apm.order_sums(c, n=10, n_max=12).cpu().numpy()
    assert np.array_equal(got, again)               # fixed summation order


def test_uneven_batch_sums(apm):
    rng = np.random.default_rng(42)
    orders = rng.integers(4, 13, size=2500).astype(np.int32)
    c_off = np.zeros(orders.size, dtype=np.int64)
    c_off[1:] = np.cumsum(1 << orders.astype(np.int64))[:-1]
    c = torch.zeros(int(c_off[-1] + (1 << int(orders[-1]))), dtype=torch.float64, device="cuda")
    c.uniform_(-1.0, 1.0)
    n_t = torch.as_tensor(orders).cuda()
    off_t = torch.as_tensor(c_off).cuda()
    got = apm.order_sums(c, n_arr=n_t, c_off=off_t, n_max=12).cpu().numpy()
    ch = c.cpu().numpy()
    last = ch[c_off + (1 << orders.astype(np.int64)) - 1]
    ref = table({m: last[orders == m] for m in range(4, 13)}, 12)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-300)
    assert got[:, 0].sum() == orders.size


def test_split_training_step_matches_fused_step(apm):
    from paper_2104_07638_gb300 import mc
    L = mc.lib()
    F = torch.randint(-2000, 2000, (512, 64), dtype=torch.int16, device="cuda")
    F = (F.to(torch.float32) / 4000).to(torch.bfloat16).view(torch.int16).contiguous()
    t = torch.randn(512, dtype=torch.float32, device="cuda")
    a, b = mc.Surrogate(seed=3, max_batch=512), mc.Surrogate(seed=3, max_batch=512)
    for step in (1, 2, 3):
        la = torch.zeros(1, dtype=torch.float32, device="cuda")
        lb = torch.zeros(1, dtype=torch.float32, device="cuda")
        s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        assert L.apm_mlp_train_step(ctypes.byref(a.net), mc._p(F), mc._p(t), 512, 500, ctypes.c_float(1e-3), step,
                                    mc._p(la), mc._p(a.ws), a.ws.numel(), s) == 0
        assert L.apm_mlp_gradient(ctypes.byref(b.net), mc._p(F), mc._p(t), 512, 500, mc._p(lb), mc._p(b.ws),
                                  b.ws.numel(), s) == 0
        assert L.apm_mlp_adam_step(ctypes.byref(b.net), ctypes.c_float(1e-3), step, s) == 0
        torch.cuda.synchronize()
        assert torch.equal(a.grad, b.grad) and torch.equal(a.param, b.param)
        assert torch.equal(a.param_bf16, b.param_bf16) and torch.equal(la, lb)
    a.check()
    b.check()
