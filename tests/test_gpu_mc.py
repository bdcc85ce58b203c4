"""Learned proposal: surrogate-network kernels against the FP64 reference,
exactness of the delayed-acceptance chain on a state space small enough to
enumerate, and the gain of the trained network over the plain proposal."""
import itertools

import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as omlp
from paper_2104_07638_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2104_07638_gb300 import mc as m
    m.lib()
    return m


def bf16_bits(x: torch.Tensor) -> torch.Tensor:
    return x.to(torch.bfloat16).view(torch.int16)


def test_forward_and_gradients_match_fp64_reference(mc):
    net = mc.Surrogate(seed=7, max_batch=256)
    rng = np.random.default_rng(8)
    B = 256
    X = torch.as_tensor(rng.standard_normal((B, 64)) * 0.5, dtype=torch.float32)
    X[:, 57:] = 0.0
    Xb = bf16_bits(X).cuda()
    t = torch.as_tensor(rng.standard_normal(B), dtype=torch.float32).cuda()
    flat = net.param.cpu().numpy().astype(np.float64)
    p = omlp.unpack(net.param.cpu().numpy(), round_weights=True)
    Xr = omlp.bf16_round(X.numpy())
    y_ref, _ = omlp.forward(p, Xr, storage_bf16=True)
    y = torch.zeros(B, dtype=torch.float32, device="cuda")
    net.forward_raw(Xb, y)
    y = y.cpu().numpy()
    assert np.linalg.norm(y - y_ref) <= 2e-3 * np.linalg.norm(y_ref)
    y64, _ = omlp.forward(p, Xr)                         # unrounded FP64: BF16-level agreement
    assert np.linalg.norm(y - y64) <= 2e-2 * np.linalg.norm(y64)
    # one step with learning rate 0: gradients only
    net.step += 1
    net.loss_acc.zero_()
    import ctypes
    from paper_2104_07638_gb300 import apm
    code = mc.lib().apm_mlp_train_step(ctypes.byref(net.net), mc._p(Xb), mc._p(t), B, B, ctypes.c_float(0.0),
                                       net.step, mc._p(net.loss_acc), mc._p(net.ws), net.ws.numel(), mc._s(Xb))
    assert code == 0
    tt = t.cpu().numpy().astype(np.float64)
    loss_ref, g_ref = omlp.loss_and_grad(p, Xr, tt, storage_bf16=True)
    _, g64 = omlp.loss_and_grad(p, Xr, tt)
    assert abs(float(net.loss_acc.item()) - loss_ref) <= 2e-3 * loss_ref
    g = net.grad.cpu().numpy().astype(np.float64)
    o = 0
    for name, shape in omlp.SHAPES:
        k = int(np.prod(shape))
        ref = np.asarray(g_ref[name]).ravel()
        err = np.linalg.norm(g[o:o + k] - ref) / max(np.linalg.norm(ref), 1e-30)
        assert err <= 5e-3, (name, err)            # same storage rounding: FP32-vs-FP64 accumulation
        ref64 = np.asarray(g64[name]).ravel()
        err64 = np.linalg.norm(g[o:o + k] - ref64) / max(np.linalg.norm(ref64), 1e-30)
        assert err64 <= 1e-1, (name, err64)        # BF16 operands of cancelling sums
        o += k
    assert np.allclose(net.param.cpu().numpy(), flat.astype(np.float32))   # lr = 0: unchanged


def test_training_reduces_loss(mc):
    net = mc.Surrogate(seed=9, max_batch=4096)
    rng = np.random.default_rng(10)
    N = 32768
    X = torch.as_tensor(rng.uniform(-1, 1, (N, 64)), dtype=torch.float32)
    X[:, 43:] = 0.0
    target = (torch.sin(3 * X[:, 0]) + X[:, 1] * X[:, 2] - 0.5 * X[:, 5] ** 2).cuda()
    losses = net.train(bf16_bits(X).cuda(), target, epochs=12, batch=2048, lr=2e-3)
    assert np.mean(losses[-8:]) < 0.3 * losses[0], losses


def tiny_weights(win, mtau, n):
    """Exact |c_n| of every configuration of n vertices on win x win x mtau
    (oracle route: per-minor LU + plain recursion), ordered like the walker codes."""
    G = I.hubbard_g0_table(win=win, mtau=mtau)
    states = [(x, y, m) for x in range(win) for y in range(win) for m in range(mtau)]
    confs = list(itertools.product(range(len(states)), repeat=n))
    A = np.empty((len(confs), n, n))
    for k, cf in enumerate(confs):
        v = [states[s] for s in cf]
        for i in range(n):
            for j in range(n):
                A[k, i, j] = G[abs(v[i][0] - v[j][0]), abs(v[i][1] - v[j][1]), v[i][2] - v[j][2] + mtau - 1]
    m = oracle.minors_lu(A)
    c = oracle.cdet_recursion(m * m)[:, -1]
    return states, confs, np.abs(c)


def chi2_pvalue(counts, p):
    """Pearson's chi-square test of counts against the distribution p: bins
    whose expected count is below 5 are pooled into one (dropped if the pool
    itself expects fewer than 5)."""
    from scipy.stats import chi2
    E = counts.sum() * p
    big = E >= 5.0
    O, Ex = list(counts[big]), list(E[big])
    if E[~big].sum() >= 5.0:
        O.append(counts[~big].sum())
        Ex.append(E[~big].sum())
    O, Ex = np.array(O), np.array(Ex)
    stat = float(((O - Ex) ** 2 / Ex).sum())
    return float(chi2.sf(stat, O.size - 1)), stat, O.size - 1


@pytest.mark.parametrize("learned", [False, True])
def test_chain_samples_the_exact_distribution(mc, learned):
    """On n = 2 vertices in a 2 x 2 window with 4 time bins (256 configurations,
    enumerated with their exact |c_2| by the oracle) the chains' states must
    follow |c_2| / Z: a chi-square test at the 1e-3 level over the 16384
    independent walkers, at four times spaced by five integrated autocorrelation
    times (measured on the chain itself), so that the counts are independent.
    The same counts must reject a uniform and a square-root target."""
    import math
    n, win, mtau = 2, 2, 4
    states, confs, w = tiny_weights(win, mtau, n)
    pi = w / w.sum()
    G = torch.as_tensor(I.hubbard_g0_table(win=win, mtau=mtau)).cuda()
    W = 16384
    wk = mc.Walkers(W, n, G, win, mtau, seed=11 + learned)
    net = None
    if learned:
        net = mc.Surrogate(seed=12, max_batch=W)      # untrained: a deliberately poor surrogate
        wk.init_surrogate(net)

    def step(rec=None):
        wk.step_da(net, rec) if learned else wk.step_plain(rec)

    for _ in range(100):
        step()
    rec = []
    for _ in range(300):
        step(rec)
    tau = mc.integrated_autocorr(torch.stack([r[1] for r in rec]).cpu().numpy())
    gap = max(1, math.ceil(5 * tau))
    code = {s: i for i, s in enumerate(states)}
    counts = np.zeros(len(confs))
    for _ in range(4):
        for _ in range(gap):
            step()
        X = wk.X.cpu().numpy()
        idx = np.array([code[tuple(v)] for v in X[:, 0]]) * len(states) + \
            np.array([code[tuple(v)] for v in X[:, 1]])
        counts += np.bincount(idx, minlength=len(confs))
    p, stat, dof = chi2_pvalue(counts, pi)
    print(f"tau_int {tau:.2f}, gap {gap}, chi2 {stat:.1f} on {dof} dof, p = {p:.3g}")
    assert p > 1e-3, (p, stat, dof)
    assert chi2_pvalue(counts, np.full(len(confs), 1.0 / len(confs)))[0] < 1e-6
    assert chi2_pvalue(counts, np.sqrt(pi) / np.sqrt(pi).sum())[0] < 1e-6


def test_trained_network_gains_over_plain(mc):
    """At order 10 the trained surrogate cuts the exact evaluations needed per
    effective sample of log|c_n| (same chain length, same start)."""
    n = 10
    G = torch.as_tensor(I.hubbard_g0_table()).cuda()
    W = 4096
    wk = mc.Walkers(W, n, G, I.HUB_WIN, I.HUB_MTAU, seed=21)
    F, t = wk.collect(60)                         # burn-in + training pairs
    net = mc.Surrogate(seed=22, max_batch=W)
    net.train(F, t, epochs=3, batch=4096, lr=1e-3)
    X0, w0, s0 = wk.X.clone(), wk.weight.clone(), wk.sign.clone()
    rec_p, rec_d = [], []
    e0 = wk.exact_evals
    for _ in range(150):
        wk.step_plain(rec_p)
    evals_plain = wk.exact_evals - e0
    wk.X.copy_(X0); wk.weight.copy_(w0); wk.sign.copy_(s0)
    wk.init_surrogate(net)
    e0 = wk.exact_evals
    for _ in range(150):
        wk.step_da(net, rec_d)
    evals_da = wk.exact_evals - e0
    ess_p, ess_d = mc.ess(rec_p, 1), mc.ess(rec_d, 1)
    cost_p, cost_d = evals_plain / ess_p, evals_da / ess_d
    print(f"exact evals per ESS: plain {cost_p:.2f}, learned {cost_d:.2f}; "
          f"ESS {ess_p:.0f} vs {ess_d:.0f}; evals {evals_plain} vs {evals_da}")
    assert cost_d < cost_p


def test_trained_network_gains_effective_samples_per_second(mc):
    """At order 12 (16384 walkers, 300 steps after 60 collection steps) the
    learned chain makes more effective samples per second of wall time than
    the plain chain, for the sign of c_n where it fluctuates and for log|c_n|,
    with the surrogate's forward passes and the stage-1 filter inside the
    learned chain's time."""
    n = 12
    G = torch.as_tensor(I.hubbard_g0_table()).cuda()
    W = 16384
    wk = mc.Walkers(W, n, G, I.HUB_WIN, I.HUB_MTAU, seed=31)
    F, t = wk.collect(60)
    net = mc.Surrogate(seed=32, max_batch=W)
    net.train(F, t, epochs=2, batch=8192, lr=3e-3)
    # an untimed delayed-acceptance step first (the first use of a kernel in a
    # process may load it); both timed chains start from the state after it
    wk.init_surrogate(net)
    wk.step_da(net, [])
    X0, w0, s0 = wk.X.clone(), wk.weight.clone(), wk.sign.clone()
    rec_p, rec_d = [], []
    _, t_p = mc.timed(lambda: [wk.step_plain(rec_p) for _ in range(300)])
    wk.X.copy_(X0); wk.weight.copy_(w0); wk.sign.copy_(s0)

    def run_da():
        wk.init_surrogate(net)
        for _ in range(300):
            wk.step_da(net, rec_d)
    _, t_d = mc.timed(run_da)
    for which in (0, 1):
        ess_p, ess_d = mc.ess(rec_p, which), mc.ess(rec_d, which)
        if not (np.isfinite(ess_p) and np.isfinite(ess_d)):
            continue                          # the observable does not fluctuate
        print(f"observable {which}: ESS/s plain {ess_p / t_p:.0f}, learned {ess_d / t_d:.0f}")
        assert ess_d / t_d > ess_p / t_p
