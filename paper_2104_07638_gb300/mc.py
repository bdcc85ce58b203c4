"""Monte Carlo over CDet vertex configurations with a learned proposal filter.

The target is pi(X) ~ |c_n(X)|, the connected sum over all n vertices (CDet
recursion of Section V.A on M_ij = G0(X_i - X_j), a = det^2). The plain chain
redraws one vertex uniformly (the single-vertex move of Section V.E) and
accepts with the exact ratio. The learned chain uses the same move filtered by
a surrogate network s(X) ~ log|c_n(X)| (delayed acceptance): stage 1 passes a
move with probability min(1, e^{s(X')-s(X)}); only survivors are evaluated by
the exact FP64 kernel, and stage 2 accepts with min(1, |c(X')| e^{s(X)} /
(|c(X)| e^{s(X')})), so the chain keeps the exact target.

Everything runs in the library's kernels (proposal, matrix build, features,
network forward/backward/Adam, stage-1 filter and compaction, exact minors and
connected sums, acceptance); torch supplies device memory, uniform random
numbers and the one host read of the survivor count per step. Effective sample
size uses Sokal's adaptive window on the mean autocorrelation over walkers.
"""
from __future__ import annotations

import ctypes
import math
import time

import numpy as np
import torch

from . import apm, dist

MLP_IN, MLP_PARAMS = 64, 148488


class ApmMlp(ctypes.Structure):
    _fields_ = [("param", ctypes.c_void_p), ("param_bf16", ctypes.c_void_p), ("grad", ctypes.c_void_p),
                ("adam_m", ctypes.c_void_p), ("adam_v", ctypes.c_void_p)]


def _sig(L):
    P, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    for name, args in {
        "apm_mc_propose": [P, i32, i32, i32, i32, P, P, P],
        "apm_mc_build_matrices": [P, P, i32, i32, i32, i32, P, P, P],
        "apm_mc_features": [P, P, i32, i32, i32, i32, P, P, i32, P],
        "apm_mc_stage1": [P, P, P, i32, P, P, P],
        "apm_mc_accept": [P, P, P, P, P, P, P, i64, P, i32, P, i32, P, P],
        "apm_mlp_workspace_size": [i32, ctypes.POINTER(sz)],
        "apm_mlp_sync_bf16": [ctypes.POINTER(ApmMlp), P],
        "apm_mlp_forward": [ctypes.POINTER(ApmMlp), P, i32, P, P, sz, P],
        "apm_mlp_train_step": [ctypes.POINTER(ApmMlp), P, P, i32, i32, ctypes.c_float, i32, P, P, sz, P],
        "apm_mlp_gradient": [ctypes.POINTER(ApmMlp), P, P, i32, i32, P, P, sz, P],
        "apm_mlp_adam_step": [ctypes.POINTER(ApmMlp), ctypes.c_float, i32, P],
        "apm_mlp_status": [P, sz, ctypes.POINTER(ctypes.c_uint32), P],
        "apm_mlp_gemm_tn": [P, P, P, P, P, i32, i32, i32, i32, P, sz, P],
    }.items():
        f = getattr(L, name)
        if f.argtypes is None:
            f.argtypes = args
            f.restype = ctypes.c_int
    return L


def lib():
    return _sig(apm.lib())


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _s(t):
    return apm._stream(t)


def pad64(b: int) -> int:
    return (b + 63) // 64 * 64


class Surrogate:
    """The surrogate network: parameters, Adam state and scratch on one device."""

    def __init__(self, device="cuda", seed=0, max_batch=16384):
        g = torch.Generator(device="cpu").manual_seed(seed)
        p = torch.zeros(MLP_PARAMS, dtype=torch.float32)
        o = 0
        for fan_out, fan_in in ((256, 64), (256, 256), (256, 256)):
            p[o:o + fan_out * fan_in] = torch.randn(fan_out * fan_in, generator=g) * math.sqrt(2.0 / fan_in)
            o += fan_out * fan_in + fan_out
        p[o:o + 256] = torch.randn(256, generator=g) * math.sqrt(1.0 / 256)
        self.param = p.to(device)
        self.param_bf16 = torch.zeros(MLP_PARAMS, dtype=torch.int16, device=device)
        self.grad = torch.zeros(MLP_PARAMS, dtype=torch.float32, device=device)
        self.m = torch.zeros_like(self.grad)
        self.v = torch.zeros_like(self.grad)
        self.net = ApmMlp(self.param.data_ptr(), self.param_bf16.data_ptr(), self.grad.data_ptr(),
                          self.m.data_ptr(), self.v.data_ptr())
        self.max_batch = pad64(max_batch)
        nb = ctypes.c_size_t(0)
        apm._check(lib().apm_mlp_workspace_size(self.max_batch, ctypes.byref(nb)), "apm_mlp_workspace_size")
        self.ws = torch.zeros(nb.value, dtype=torch.uint8, device=device)  # status word starts clear
        self.loss_acc = torch.zeros(1, dtype=torch.float32, device=device)
        self.step = 0
        self.y_mean, self.y_std = 0.0, 1.0
        apm._check(lib().apm_mlp_sync_bf16(ctypes.byref(self.net), _s(self.param)), "apm_mlp_sync_bf16")

    def forward_raw(self, F: torch.Tensor, y: torch.Tensor):
        Bp = F.shape[0]
        assert Bp % 64 == 0 and Bp <= self.max_batch
        apm._check(lib().apm_mlp_forward(ctypes.byref(self.net), _p(F), Bp, _p(y), _p(self.ws), self.ws.numel(),
                                         _s(F)), "apm_mlp_forward")

    def check(self):
        """Synchronise and raise if a tensor-core GEMM reported a timed-out wait."""
        flags = ctypes.c_uint32(0)
        apm._check(lib().apm_mlp_status(_p(self.ws), self.ws.numel(), ctypes.byref(flags), _s(self.ws)),
                   "apm_mlp_status")

    def log_weight(self, F: torch.Tensor, y: torch.Tensor):
        """y <- predicted log|c| (de-normalised)."""
        self.forward_raw(F, y)
        y.mul_(self.y_std).add_(self.y_mean)

    def train(self, F_all: torch.Tensor, target: torch.Tensor, epochs=3, batch=4096, lr=1e-3, seed=0):
        """Adam on normalised targets; F_all [N, 64] bf16 (int16 storage), target [N] float32.

        Under an initialised process group with several processes, each holding
        its own rows, the training is data-parallel: the target normalisation
        and the number of batches per epoch are agreed over the processes, and
        before every Adam step the gradient is averaged over them
        (dist.average_gradient_), so that every process applies the same step."""
        _, ws = dist.world()
        N = target.numel()
        mom = dist.allreduce_sum_(torch.tensor([float(N), float(target.double().sum()),
                                                float((target.double() ** 2).sum())], dtype=torch.float64))
        cnt = float(mom[0])
        self.y_mean = float(mom[1] / cnt)
        self.y_std = max(math.sqrt(max(float(mom[2] / cnt) - self.y_mean ** 2, 0.0) * cnt / max(cnt - 1.0, 1.0)),
                         1e-6)
        t_norm = ((target - self.y_mean) / self.y_std).contiguous()
        batch = pad64(batch)
        nb = N // batch
        if ws > 1:   # every process takes the same number of steps
            nbt = torch.tensor([nb], dtype=torch.int64)
            import torch.distributed as tdist
            tdist.all_reduce(nbt, op=tdist.ReduceOp.MIN)
            nb = int(nbt)
        g = torch.Generator(device="cpu").manual_seed(seed)
        losses = []
        for _ in range(epochs):
            perm = torch.randperm(N, generator=g).to(F_all.device)
            for s0 in range(0, nb * batch, batch):
                sel = perm[s0:s0 + batch]
                Fb = F_all[sel].contiguous()
                tb = t_norm[sel].contiguous()
                self.step += 1
                self.loss_acc.zero_()
                if ws == 1:
                    apm._check(lib().apm_mlp_train_step(ctypes.byref(self.net), _p(Fb), _p(tb), batch, batch,
                                                        ctypes.c_float(lr), self.step, _p(self.loss_acc),
                                                        _p(self.ws), self.ws.numel(), _s(Fb)), "apm_mlp_train_step")
                else:
                    apm._check(lib().apm_mlp_gradient(ctypes.byref(self.net), _p(Fb), _p(tb), batch, batch,
                                                      _p(self.loss_acc), _p(self.ws), self.ws.numel(), _s(Fb)),
                               "apm_mlp_gradient")
                    dist.average_gradient_(self.grad, batch)
                    apm._check(lib().apm_mlp_adam_step(ctypes.byref(self.net), ctypes.c_float(lr), self.step,
                                                       _s(Fb)), "apm_mlp_adam_step")
                losses.append(self.loss_acc)
                self.loss_acc = torch.zeros(1, dtype=torch.float32, device=F_all.device)
        self.check()
        return torch.cat(losses).cpu().numpy() if losses else np.zeros(0)


class Walkers:
    """W independent chains at order n on the Hubbard G0 table g0 [win][win][2mtau-1]."""

    def __init__(self, W, n, g0: torch.Tensor, win: int, mtau: int, seed=0):
        self.W, self.n, self.win, self.mtau = W, n, win, mtau
        self.g0 = g0.contiguous()
        dev = g0.device
        self.gen = torch.Generator(device=dev).manual_seed(seed)
        x = torch.randint(0, win, (W, n, 2), device=dev, generator=self.gen)
        m = torch.randint(0, mtau, (W, n, 1), device=dev, generator=self.gen)
        self.X = torch.cat([x, m], 2).to(torch.int32).contiguous()
        self.Xp = torch.empty_like(self.X)
        self.weight = torch.zeros(W, dtype=torch.float64, device=dev)
        self.sign = torch.zeros(W, dtype=torch.float64, device=dev)
        self.s_cur = torch.zeros(W, dtype=torch.float32, device=dev)
        self.A = torch.empty((W, n, n), dtype=torch.float64, device=dev)
        self.c = torch.empty((W, 1 << n), dtype=torch.float64, device=dev)
        self.idx = torch.empty(W, dtype=torch.int32, device=dev)
        self.count = torch.zeros(1, dtype=torch.int32, device=dev)
        self.accepted = torch.zeros(1, dtype=torch.int32, device=dev)
        self.Fp = torch.zeros((pad64(W), MLP_IN), dtype=torch.int16, device=dev)
        self.s_new = torch.zeros(pad64(W), dtype=torch.float32, device=dev)
        self.exact_evals = 0
        self.steps = 0
        self._exact_all(self.X)
        self.weight.copy_(self.c[:, -1].abs())
        self.sign.copy_(torch.where(self.c[:, -1] >= 0, 1.0, -1.0))

    # exact connected sums of configurations X (all walkers or idx[:count])
    def _exact_all(self, X, idx=None, count=None):
        count = self.W if count is None else count
        if count == 0:
            return
        apm._check(lib().apm_mc_build_matrices(_p(X), _p(idx), count, self.n, self.win, self.mtau, _p(self.g0),
                                               _p(self.A), _s(X)), "apm_mc_build_matrices")
        apm.cdet_connected(self.A[:count], out_c=self.c[:count])
        self.exact_evals += count

    def _propose(self):
        u = torch.rand((self.W, 4), device=self.X.device, generator=self.gen)
        apm._check(lib().apm_mc_propose(_p(self.X), self.W, self.n, self.win, self.mtau, _p(u), _p(self.Xp),
                                        _s(u)), "apm_mc_propose")

    def features(self, X, F, idx=None, count=None):
        count = self.W if count is None else count
        apm._check(lib().apm_mc_features(_p(X), _p(idx), count, self.n, self.win, self.mtau, _p(self.g0), _p(F),
                                         F.shape[0], _s(X)), "apm_mc_features")

    def step_plain(self, record=None):
        self._propose()
        self._exact_all(self.Xp)
        u2 = torch.rand(self.W, device=self.X.device, generator=self.gen)
        apm._check(lib().apm_mc_accept(_p(self.X), _p(self.Xp), _p(self.weight), _p(self.sign), None, None,
                                       _p(self.c[:, -1]), self.c.shape[1], None, self.W, _p(u2), self.n,
                                       _p(self.accepted), _s(u2)), "apm_mc_accept")
        self.steps += 1
        if record is not None:
            record.append(self.observables())

    def init_surrogate(self, net: Surrogate):
        self.features(self.X, self.Fp)
        net.log_weight(self.Fp, self.s_new)
        self.s_cur.copy_(self.s_new[:self.W])

    def step_da(self, net: Surrogate, record=None):
        self._propose()
        self.features(self.Xp, self.Fp)
        net.log_weight(self.Fp, self.s_new)
        u1 = torch.rand(self.W, device=self.X.device, generator=self.gen)
        apm._check(lib().apm_mc_stage1(_p(self.s_new), _p(self.s_cur), _p(u1), self.W, _p(self.idx),
                                       _p(self.count), _s(u1)), "apm_mc_stage1")
        count = int(self.count.item())           # the one host read per step
        self._exact_all(self.Xp, self.idx, count)
        u2 = torch.rand(self.W, device=self.X.device, generator=self.gen)
        apm._check(lib().apm_mc_accept(_p(self.X), _p(self.Xp), _p(self.weight), _p(self.sign), _p(self.s_cur),
                                       _p(self.s_new), _p(self.c[:, -1]), self.c.shape[1], _p(self.idx), count,
                                       _p(u2), self.n, _p(self.accepted), _s(u2)), "apm_mc_accept")
        self.steps += 1
        if record is not None:
            record.append(self.observables())

    def observables(self):
        """(sign, log|c|, log(|c| / surrogate)) of every walker, kept on the
        device; the last row is meaningful for the learned chain only (the
        plain chain keeps no surrogate value)."""
        lw = torch.log(self.weight.clamp_min(1e-300))
        return torch.stack([self.sign, lw, lw - self.s_cur.double()])

    def collect(self, steps):
        """Plain steps that also return training pairs (features, log|c|) of
        every exactly evaluated proposal."""
        feats, targets = [], []
        for _ in range(steps):
            self._propose()
            self._exact_all(self.Xp)
            F = torch.zeros((pad64(self.W), MLP_IN), dtype=torch.int16, device=self.X.device)
            self.features(self.Xp, F)
            feats.append(F[:self.W])
            targets.append(torch.log(self.c[:, -1].abs().clamp_min(1e-300)).float())
            u2 = torch.rand(self.W, device=self.X.device, generator=self.gen)
            apm._check(lib().apm_mc_accept(_p(self.X), _p(self.Xp), _p(self.weight), _p(self.sign), None, None,
                                           _p(self.c[:, -1]), self.c.shape[1], None, self.W, _p(u2), self.n,
                                           _p(self.accepted), _s(u2)), "apm_mc_accept")
            self.steps += 1
        F = torch.cat(feats)
        t = torch.cat(targets)
        # clip the far lower tail (near-cancelling configurations) for the
        # regression; a non-finite target (a matrix the kernel flagged, e.g. a
        # correction-log overflow) gets the same clip value. The 1 % quantile
        # is taken on the host (a few MB): the device sort behind a quantile
        # costs seconds on its first use in a process
        th = t[:min(t.numel(), 1 << 20)].cpu().numpy()
        fin = th[np.isfinite(th)]
        lo = float(np.quantile(fin, 0.01)) if fin.size else 0.0
        t = torch.where(torch.isfinite(t), t, torch.full_like(t, lo))
        return F, t.clamp_min(lo)


def integrated_autocorr(series: np.ndarray, c: float = 5.0) -> float:
    """Sokal's adaptive-window integrated autocorrelation time of a (T, W)
    array of W independent chains (mean autocorrelation over chains)."""
    x = np.asarray(series, dtype=np.float64)
    T, W = x.shape
    x = x - x.mean(axis=0, keepdims=True)
    var = np.mean(x * x)
    if var == 0.0:
        return float("nan")
    nfft = 1 << (2 * T - 1).bit_length()
    f = np.fft.rfft(x, n=nfft, axis=0)
    acf = np.fft.irfft(f * np.conj(f), n=nfft, axis=0)[:T].mean(axis=1)
    rho = acf / acf[0]
    tau = 1.0
    for M in range(1, T):
        tau += 2.0 * rho[M]
        if M >= c * tau:
            break
    return max(tau, 1.0)


def ess(record, which=0) -> float:
    """Effective sample size of observable `which` (0 sign, 1 log|c|, 2 log of
    |c| over the surrogate) over all walkers; NaN if it does not fluctuate."""
    arr = torch.stack([r[which] for r in record]).cpu().numpy()      # (T, W)
    tau = integrated_autocorr(arr)
    if not math.isfinite(tau):
        return float("nan")
    return arr.size / tau


def timed(fn):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0
