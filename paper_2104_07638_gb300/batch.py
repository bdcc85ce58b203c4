"""Uneven batches: CUDA-graph capture of the persistent longest-first launches,
and the per-order autotuner of the connected-sum lane mapping.

``CdetVarlenGraph`` / ``KeldyshVarlenGraph`` own preallocated outputs and
workspace, run one ordinary call (which also uploads the library's constant
tables), then capture the call -- a one-block counting sort by decreasing order
followed by the persistent kernel -- into a CUDA graph. ``replay()`` relaunches
it on the current inputs (write new matrices into ``A``/``Mt`` in place).

``autotune`` searches, on the GPU at hand, the lane-group size of every
popcount layer of the recursion per order, the order from which the connected
sums take the fast subset convolution, the resident CTAs per SM of the
persistent uneven batch and the warps per CTA of the uneven Keldysh batch, and
installs the result (``apm_cdet_tune_set``, ``apm_tune_options_set``); results
are cached per GPU name in ``_build/``.
"""
from __future__ import annotations

import json
import os

import torch

from . import apm
from . import build as _build


class CdetVarlenGraph:
    def __init__(self, A: torch.Tensor, a_off: torch.Tensor, n: torch.Tensor, n_max: int | None = None,
                 with_minors: bool = True):
        self.A, self.a_off, self.n = A, a_off, n
        self.n_max = int(n.max().item()) if n_max is None else n_max
        self.c_off = apm.varlen_out_offsets(n)
        total = int((self.c_off[-1] + (1 << int(n[-1].item()))).item())
        dev = A.device
        self.c = torch.empty(total, dtype=torch.float64, device=dev)
        self.minors = torch.empty(total, dtype=torch.float64, device=dev) if with_minors else None
        self.status = torch.zeros(n.numel(), dtype=torch.int32, device=dev)
        nb = apm.workspace_size(apm.OP_CDET_VARLEN, self.n_max, n.numel())
        self.workspace = torch.empty(max(nb, 16), dtype=torch.uint8, device=dev)
        self._call()                       # eager run: tables uploaded, attributes set
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._call()

    def _call(self):
        code = apm.lib().apm_cdet_connected_varlen(
            apm._ptr(self.A), None, apm._ptr(self.a_off), apm._ptr(self.n), self.n.numel(), self.n_max, 0,
            apm._ptr(self.c), apm._ptr(self.minors), apm._ptr(self.c_off), None, apm._ptr(self.status),
            apm._ptr(self.workspace), self.workspace.numel(), apm._stream(self.A))
        apm._check(code, "apm_cdet_connected_varlen")

    def replay(self):
        self.graph.replay()
        return self.c


class KeldyshVarlenGraph:
    def __init__(self, Mt: torch.Tensor, m_off: torch.Tensor, n: torch.Tensor, n_max: int | None = None,
                 signed: bool = False):
        self.Mt, self.m_off, self.n = Mt, m_off, n
        self.n_max = int(n.max().item()) if n_max is None else n_max
        self.flags = apm.KELDYSH_SIGNED if signed else 0
        dev = Mt.device
        self.sum = torch.empty((n.numel(), 2), dtype=torch.float64, device=dev)
        self.status = torch.zeros(n.numel(), dtype=torch.int32, device=dev)
        nb = apm.workspace_size(apm.OP_KELDYSH_VARLEN, self.n_max, n.numel())
        self.workspace = torch.empty(max(nb, 16), dtype=torch.uint8, device=dev)
        self._call()
        torch.cuda.synchronize(dev)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._call()

    def _call(self):
        code = apm.lib().apm_keldysh_sum_varlen(
            apm._ptr(self.Mt), apm._ptr(self.m_off), apm._ptr(self.n), self.n.numel(), self.n_max, self.flags,
            apm._ptr(self.sum), None, apm._ptr(self.status), apm._ptr(self.workspace), self.workspace.numel(),
            apm._stream(self.Mt))
        apm._check(code, "apm_keldysh_sum_varlen")

    def replay(self):
        self.graph.replay()
        return torch.view_as_complex(self.sum)


# ---------------------------------------------------------------------------
# autotuner
# ---------------------------------------------------------------------------

def _shift_table(packed: int, n: int, delta: int) -> int:
    out = 0
    for k in range(17):
        r = (packed >> (3 * k)) & 7
        if 2 <= k <= n:
            r = max(0, min(5, k - 1, r + delta))
        else:
            r = 0
        out |= r << (3 * k)
    return out


def _with_layer(packed: int, k: int, r: int) -> int:
    return (packed & ~(7 << (3 * k))) | (r << (3 * k))


def _cache_path() -> str:
    name = torch.cuda.get_device_name().replace(" ", "_")
    return os.path.join(_build.BUILD, f"tune_{name}.json")


def _event_ms(fn, reps: int) -> float:
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _layer_terms(n: int, k: int) -> int:
    """Submask terms of popcount layer k of Eq. recursion at order n."""
    from math import comb
    return comb(n, k) * ((1 << (k - 1)) - 1)


def install(tuned: dict):
    """Installs a table returned by autotune (lane groups and launch options)."""
    apm.tune_set([int(tuned["lane_groups"].get(str(n), 0)) for n in range(17)])
    apm.tune_options_set(int(tuned["fsc_from_n"]), int(tuned["cdet_ctas_per_sm"]), int(tuned["keldysh_warps"]))


def autotune(orders=range(4, 13), fsc_orders=range(13, 17), reps: int = 3, use_cache: bool = True,
             tune_launch: bool = True, verbose: bool = False) -> dict:
    """Searches, on this GPU, the per-order mappings of the connected-sum path
    and the launch shapes of the uneven batches, installs the result and
    returns it (cached per GPU name under _build/):

      lane_groups[n]  (orders in `orders`) the lane-group size of every popcount
                      layer of Eq. recursion: starting from the cost model, each
                      layer holding at least 5 % of the order's submask terms
                      tries one size smaller and one larger, kept when faster
                      (orders above 12 run the recursion in blocks of 10 low
                      elements, so the order-10 table serves them);
      fsc_from_n      the order from which the connected sums take the fast
                      subset convolution: the smallest m in `fsc_orders` such
                      that it beats the recursion at every order from m on;
      cdet_ctas_per_sm  resident CTAs per SM of the persistent uneven batch
                      (2 or 3), timed on a sample of the uneven workload;
      keldysh_warps   warps per CTA of the uneven Keldysh batch (4, 6, 8, 10, 12),
                      timed on a sample of its uneven workload.

    Every choice gives the same results up to rounding (the uneven batch stays
    bit for bit equal to fixed-order launches under the same table)."""
    import time

    import numpy as np

    from . import inputs
    path = _cache_path()
    if use_cache and os.path.exists(path):
        tuned = json.load(open(path))
        install(tuned)
        return tuned
    t_start = time.perf_counter()
    apm.tune_set(None)
    apm.tune_options_set(0, 0, 0)
    timings = {}
    lane = {}
    for n in orders:
        base = apm.tune_get(n)
        batch = int(max(1216, min(65536, 4e9 / (3 ** n))))
        A = torch.as_tensor(inputs.hubbard_batch(batch, n, seed=50 + n)).cuda()
        c = torch.empty((batch, 1 << n), dtype=torch.float64, device="cuda")
        ws = torch.empty(max(apm.workspace_size(apm.OP_CDET, n, batch), 16), dtype=torch.uint8, device="cuda")

        def run(table):
            apm.tune_set([table if m == n else 0 for m in range(17)])
            return _event_ms(lambda: apm.cdet_connected(A, out_c=c, workspace=ws), reps)

        best, t_best = base, run(base)
        t_base = t_best
        total = sum(_layer_terms(n, k) for k in range(2, n + 1))
        heavy = sorted((k for k in range(2, n + 1) if _layer_terms(n, k) >= 0.05 * total),
                       key=lambda k: -_layer_terms(n, k))
        for k in heavy:
            r0 = (best >> (3 * k)) & 7
            for r in (r0 - 1, r0 + 1):
                if 0 <= r <= min(5, k - 1):
                    cand = _with_layer(best, k, r)
                    t = run(cand)
                    if t < t_best:
                        best, t_best = cand, t
        lane[str(n)] = best
        timings[f"lane_groups_n{n}"] = {"default_ms": t_base, "tuned_ms": t_best, "batch": batch}
        if verbose:
            print(f"n={n}: cost model {t_base:.3f} ms, tuned {t_best:.3f} ms", flush=True)
        del A, c, ws
    apm.tune_set([lane.get(str(m), 0) for m in range(17)])
    # hand-off from the recursion to the fast subset convolution
    faster = {}
    for n in fsc_orders:
        batch = {13: 8208, 14: 2280, 15: 1368, 16: 456}.get(n, 456)
        A = torch.as_tensor(inputs.hubbard_batch(batch, n, seed=60 + n)).cuda()
        c = torch.empty((batch, 1 << n), dtype=torch.float64, device="cuda")
        t = {}
        for m in (n, 17):      # the fast subset convolution at n, or not at all
            apm.tune_options_set(m, 0, 0)
            ws = torch.empty(max(apm.workspace_size(apm.OP_CDET, n, batch), 16), dtype=torch.uint8, device="cuda")
            t[m] = _event_ms(lambda: apm.cdet_connected(A, out_c=c, workspace=ws), reps)
            del ws
        faster[n] = t[n] < t[17]
        timings[f"fsc_n{n}"] = {"fsc_ms": t[n], "recursion_ms": t[17], "batch": batch}
        if verbose:
            print(f"n={n}: fast subset convolution {t[n]:.3f} ms, recursion {t[17]:.3f} ms", flush=True)
        del A, c
        torch.cuda.empty_cache()
    fsc_from = 17
    for n in sorted(faster, reverse=True):
        if not faster[n]:
            break
        fsc_from = n
    ctas, kw = 0, 0
    if tune_launch:
        orders_s = inputs.varlen_orders(16384, 4, 16, seed=70)
        flat, off = inputs.hubbard_varlen(orders_s, seed=70)
        A = torch.as_tensor(flat).cuda()
        a_off = torch.as_tensor(off).cuda()
        n_t = torch.as_tensor(orders_s).cuda()
        t = {}
        for k in (2, 3):
            apm.tune_options_set(fsc_from, k, 0)
            g = CdetVarlenGraph(A, a_off, n_t, with_minors=False)
            t[k] = _event_ms(g.replay, 2)
            del g
        ctas = min(t, key=t.get)
        timings["cdet_varlen_ctas_per_sm"] = {str(k): v for k, v in t.items()}
        del A, a_off
        kflat, koff = inputs.keldysh_varlen(orders_s, seed=71)
        Mt = torch.as_tensor(kflat).cuda()
        m_off = torch.as_tensor(koff).cuda()
        t = {}
        for w in (4, 6, 8, 10, 12):
            apm.tune_options_set(fsc_from, ctas, w)
            g = KeldyshVarlenGraph(Mt, m_off, n_t)
            t[w] = _event_ms(g.replay, 2)
            del g
        kw = min(t, key=t.get)
        timings["keldysh_varlen_warps"] = {str(k): v for k, v in t.items()}
        if verbose:
            print(f"uneven batch: CTAs per SM {ctas}, Keldysh warps per CTA {kw}", flush=True)
        del Mt, m_off, n_t
        torch.cuda.empty_cache()
    tuned = {"lane_groups": lane, "fsc_from_n": fsc_from, "cdet_ctas_per_sm": ctas, "keldysh_warps": kw,
             "timings": timings, "wall_s": time.perf_counter() - t_start, "gpu": torch.cuda.get_device_name()}
    install(tuned)
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump(tuned, f)
    return tuned


def autotune_cdet(orders=range(4, 13), reps: int = 3, use_cache: bool = True, verbose: bool = False):
    """The lane-group tables alone (autotune without the launch shapes);
    returns {n: packed table}."""
    tuned = autotune(orders=orders, fsc_orders=(), reps=reps, use_cache=use_cache, tune_launch=False,
                     verbose=verbose)
    return {int(k): int(v) for k, v in tuned["lane_groups"].items()}
