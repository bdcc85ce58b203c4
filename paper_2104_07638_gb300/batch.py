"""Uneven batches: CUDA-graph capture of the persistent longest-first launches,
and the per-order autotuner of the connected-sum lane mapping.

``CdetVarlenGraph`` / ``KeldyshVarlenGraph`` own preallocated outputs and
workspace, run one ordinary call (which also uploads the library's constant
tables), then capture the call -- a one-block counting sort by decreasing order
followed by the persistent kernel -- into a CUDA graph. ``replay()`` relaunches
it on the current inputs (write new matrices into ``A``/``Mt`` in place).

``autotune_cdet`` times the fixed-order kernel on Hubbard matrices of each
order for lane-group tables derived from the built-in cost model (all layers'
group sizes shifted by -2..+2, clamped) and installs the fastest per order with
``apm_cdet_tune_set``; results are cached per GPU name in ``_build/``.
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


def _cache_path() -> str:
    name = torch.cuda.get_device_name().replace(" ", "_")
    return os.path.join(_build.BUILD, f"tune_cdet_{name}.json")


def autotune_cdet(orders=range(4, 17), reps: int = 3, use_cache: bool = True, verbose: bool = False):
    """Returns {n: packed table} and installs it."""
    from . import inputs
    path = _cache_path()
    if use_cache and os.path.exists(path):
        table = {int(k): int(v) for k, v in json.load(open(path)).items()}
        apm.tune_set([table.get(n, 0) for n in range(17)])
        return table
    apm.tune_set(None)
    best = {}
    for n in orders:
        base = apm.tune_get(n)
        # enough matrices to fill every SM several times, bounded work
        batch = int(max(456, min(65536, 2e9 / (3 ** n))))
        A = torch.as_tensor(inputs.hubbard_batch(batch, n, seed=50 + n)).cuda()
        c = torch.empty((batch, 1 << n), dtype=torch.float64, device="cuda")
        ws_bytes = apm.workspace_size(apm.OP_CDET, n, batch)
        ws = torch.empty(max(ws_bytes, 16), dtype=torch.uint8, device="cuda")
        cands = sorted({_shift_table(base, n, d) for d in (-2, -1, 0, 1, 2)})
        timing = {}
        for t in cands:
            apm.tune_set([t if m == n else 0 for m in range(17)])
            apm.cdet_connected(A, out_c=c, workspace=ws)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                apm.cdet_connected(A, out_c=c, workspace=ws)
            e1.record()
            torch.cuda.synchronize()
            timing[t] = e0.elapsed_time(e1) / reps
        best[n] = min(timing, key=timing.get)
        if verbose:
            print(f"n={n}: base {timing[base]:.3f} ms, best {timing[best[n]]:.3f} ms "
                  f"({len(cands)} candidates)", flush=True)
    apm.tune_set([best.get(n, 0) for n in range(17)])
    os.makedirs(os.path.dirname(path), exist_ok=True)
    with open(path, "w") as f:
        json.dump({str(k): v for k, v in best.items()}, f)
    return best
