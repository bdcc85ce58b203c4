#!/usr/bin/env python3
"""Benchmark of the fused all-minors + CDet connected-sum path on GB300.

Workload (one step): 65536 Hubbard G0 matrices of order n = 12 (free 2D
square-lattice Hubbard model, t=1, mu=-0.5, beta=5, 32x32 k-grid; vertices r
uniform in an 8x8 window, tau uniform on a 2^14-point grid of [0,beta)); for
each matrix all 4096 principal minors and all 4096 connected sums c[S] of
a[S] = det(M[S])^2 are computed and written to HBM (one "minor set").

Prints ONE JSON line (rank 0):
  value      minor-sets/s over all ranks, device-timed (inputs resident in HBM)
  e2e        the same metric through the public API from pinned host buffers,
             host->device copy of the inputs and device->host copy of minors and
             c inside the timed region (chunks of 2048 matrices over 4 streams,
             the last two chunks' worth in halving pieces)
  roofline   FP64-ALU bound of the fused kernel (bound "alu")
  cpu_baseline  the CPU oracle (per-minor LU + plain recursion) on a bounded
             sample of the same workload, all host cores
--impl reference times that oracle as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ORDER = 12
BATCH = 65536
SMS = 152
SM_MAX_MHZ = 2070.0
FP64_FLOP_PER_CLK_SM = 4.0   # 1.25 TFLOP/s nominal FP64 / (152 SMs x 2.07 GHz), 2 DFMA/clk/SM
METRIC = "minor-sets/sec at n=12 FP64 (% of roofline)"
# DRAM bytes (read + write) per matrix of the fused kernel from one ncu capture
# of the benchmark's launch itself (65536 matrices: 82.6 MB read, 4233.9 MB
# written), valid only for the kernel source it was taken on: the sha256 prefix
# below is of fpm_cdet.cu followed by apm_internal.cuh.
TRAFFIC_PER_SET = (82606848 + 4233865472) / 65536
TRAFFIC_SRC_SHA = "043e95c10665ad51"
UNIT = "minor-sets/s"


def flops_per_set(n: int) -> int:
    """Algorithmic FP64 flops of one minor set (FMA = 2): Schur updates
    2*sum_l 2^l (n-l-1)^2, one reciprocal and one minor product per node
    2(2^n-1), the recursion 2((3^n-1)/2-(2^n-1)), and a = det^2 (2^n-1)."""
    fpm = 2 * sum((1 << l) * (n - l - 1) ** 2 for l in range(n - 1))
    nodes = (1 << n) - 1
    sc = (3 ** n - 1) // 2 - nodes
    return fpm + 2 * nodes + 2 * sc + nodes


def bytes_per_set(n: int) -> int:
    """HBM bytes: the n x n input read, 2^n minors and 2^n c written."""
    return 8 * n * n + 16 * (1 << n)


def max_over_ranks(seconds: float, world: int) -> float:
    """Slowest rank's time (the whole job finishes when the last rank does).
    Uses the already-initialised process group (gloo: host tensors only)."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(per_rank_units: int, world: int, steps: int, seconds: float) -> float:
    """Units processed by all ranks per second (weak scaling: each rank has its own batch)."""
    return world * per_rank_units * steps / seconds


def bench_config(n: int, batch: int, world: int) -> dict:
    """The workload, identical in the GPU and the reference (CPU oracle) arms."""
    return {"workload": f"hubbard_g0_n{n}_batch{batch}_minors+cdet", "n": n, "batch": batch,
            "per_rank_batch": batch, "ranks": world,
            "inputs": "rank r holds matrices r*batch .. (r+1)*batch-1 of one seeded batch (seed 2)",
            "outputs": "minors[2^n] and c[2^n] per matrix, FP64",
            "l2": "GPU arm: a 256 MB buffer rewritten between timed steps (outside the events); "
                  "per step 75.5 MB of inputs and 4.3 GB of outputs"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-rows", action="store_true",
                    help="skip the per-row measurements of the other hot-path steps")
    ap.add_argument("--mc-steps", type=int, default=1000,
                    help="steps per chain of the learned-proposal row at orders 10..12")
    ap.add_argument("--mc-steps-high", type=int, default=400,
                    help="steps per chain of the learned-proposal row at orders 13, 14")
    ap.add_argument("--case", default=None,
                    choices=["cdet_n12", "cdet_n12_full", "cdet_n16", "keldysh_n12", "ppm_n14", "cdet_uneven",
                             "xnor_n12", "nand_n10", "keldysh2_n12", "mlp_gemm", "fsc_n16", "minors_n12",
                             "minors_n20", "minors_n24", "fp64_probe", "keldysh_uneven"],
                    help="run 3 launches of one kernel on a small case (for profiling) and exit")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader",
                                       "-i", str(self.gpu), "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                self.out, _ = self.p.communicate()

    def summary(self):
        sm, mx, reasons = [], None, set()
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1].split()[0]))
                mx = float(f[2].split()[0])
            except ValueError:
                continue
            names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def keldysh_flops(n: int) -> int:
    """Algorithmic flops of one Keldysh sum: complex FMAs of every Schur step of
    the XOR tree (8 real flops each) over the m2 (m2 - 1) entries of a child of
    size m2 that a minor can read (an XOR minor keeps one row and column of a
    2 x 2 block, so the blocks' off-diagonal entries are never read), pivot
    reciprocals/products, leaf sums."""
    return (8 * sum((1 << (l + 1)) * (2 * (n - l - 1)) * (2 * (n - l - 1) - 1) for l in range(n - 1))
            + 12 * (2 ** (n + 1) - 2) + 2 * 2 ** n)


def xnor_flops(n: int) -> int:
    """Algorithmic flops of all XNOR minors of a 2n x 2n matrix: per tree node with
    a kept child of size m2 = 2(n-l-1), the Schur update (4 m2^2), the row factors
    C P^-1 (6 m2) and the pivot determinant, inverse and node product (9)."""
    return sum((1 << l) * (4 * (2 * (n - l - 1)) ** 2 + 12 * (n - l - 1) + 9) for l in range(n))


def keldysh2_flops(n: int) -> int:
    """Algorithmic flops of one two-spin Keldysh sum: both spins' XOR trees
    (2 keldysh_flops) plus the extra complex product per node and per leaf."""
    return 2 * keldysh_flops(n) + 6 * (2 ** (n + 1) - 2) + 8 * 2 ** n


def nand_flops(n: int) -> int:
    """Algorithmic flops of all NAND minors of a 2n x 2n matrix (the ternary
    tree): per node two kept children of size m2 = 2(n-l-1), each the rank-1
    Schur update of the m2 (m2 - 1) entries a minor can read (a minor keeps at
    most one row and column of a 2 x 2 block, so the blocks' off-diagonal
    entries are never read: 2 m2 (m2 - 1)), its row factors (m2) and the pivot
    reciprocal and node product (3)."""
    return sum(3 ** l * 2 * (2 * (2 * (n - l - 1)) * (2 * (n - l - 1) - 1) + 2 * (n - l - 1) + 3)
               for l in range(n))


def minors_flops(n: int) -> int:
    """Algorithmic flops of all 2^n minors by the tree alone (Section II): per
    node of level l a Schur complement of (n-l-1)^2 FMAs, and a reciprocal and a
    product per minor."""
    return 2 * sum(2 ** l * (n - l - 1) ** 2 for l in range(n)) + 2 * (2 ** n - 1)


def sc_flops(n: int) -> int:
    """Flops of the CDet recursion alone: one FMA per (T, S) pair with the
    lowest element of S in T, T a proper non-empty subset."""
    return 2 * ((3 ** n - 1) // 2 - (2 ** n - 1))


FSC_FROM_N = 16  # orders whose connected sums the library takes through the fast subset convolution


def cdet_path_flops(n: int, fsc_from: int = None) -> int:
    """Algorithmic flops of one minor set as the library computes it: the
    recursion's count below the hand-off order (FSC_FROM_N by default), the fast
    subset convolution's from there."""
    if n < (FSC_FROM_N if fsc_from is None else fsc_from):
        return flops_per_set(n)
    return flops_per_set(n) - sc_flops(n) + fsc_flops(n)


def fsc_flops(n: int) -> int:
    """Flops of the connected sums by the fast subset convolution: ranked zeta
    and Mobius transforms (n ranks x n elements x 2^(n-1) additions each) and,
    per mask, the power-series logarithm (k-1 FMAs and a multiply-add and a
    scaling for each of the n coefficients)."""
    return 2 * n * n * 2 ** (n - 1) + 2 ** n * (n * (n - 1) + 3 * n)


def perm_flops(n: int) -> int:
    """Algorithmic flops of all permanent minors: one product and one addition
    per (T subset of S) pair, plus the row sums."""
    return 2 * 3 ** n + n * 2 ** n


def _measured_peaks() -> dict:
    """Measured HBM and BF16 peaks of this GPU type, when the file is present."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _event_ms(fn, reps=3):
    import torch
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_rows(args, dev, peak):
    """One measurement per remaining hot-path step on its configuration."""
    import numpy as np
    import torch
    from paper_2104_07638_gb300 import apm, inputs, mc
    from paper_2104_07638_gb300.batch import CdetVarlenGraph, KeldyshVarlenGraph
    rows = {}
    from paper_2104_07638_gb300 import batch as pbatch
    # a7: uneven batch of 131072 walkers, n uniform in 4..16, minors + connected sums, graph replay;
    # first with the default mappings, then with the ones the autotuner finds on this GPU
    orders = inputs.varlen_orders(131072, 4, 16, seed=3)
    flat, off = inputs.hubbard_varlen(orders, seed=3)
    A = torch.as_tensor(flat).to(dev)
    a_off = torch.as_tensor(off).to(dev)
    n_t = torch.as_tensor(orders).to(dev)
    apm.tune_set(None)
    apm.tune_options_set(0, 0, 0)
    g = CdetVarlenGraph(A, a_off, n_t)
    ms_default = _event_ms(g.replay)
    del g
    tuned, t_tune = mc.timed(lambda: pbatch.autotune(use_cache=False))
    g = CdetVarlenGraph(A, a_off, n_t)
    ms = _event_ms(g.replay)
    fsc_from = tuned["fsc_from_n"]
    fl = sum(cdet_path_flops(int(k), fsc_from) for k in orders)
    tuned_summary = {"fsc_from_n": fsc_from, "cdet_ctas_per_sm": tuned["cdet_ctas_per_sm"],
                     "keldysh_warps": tuned["keldysh_warps"],
                     "lane_groups": {k: f"{v:#x}" for k, v in tuned["lane_groups"].items()},
                     "tuner_wall_s": t_tune}
    rows["a7_cdet_uneven_131072_n4to16"] = {
        "value": orders.size / (ms * 1e-3), "unit": "minor-sets/s", "ms": ms, "ms_default_mappings": ms_default,
        "tflops": fl / (ms * 1e-3) / 1e12, "frac_fp64_peak": fl / (ms * 1e-3) / 1e12 / peak,
        "tuned": tuned_summary,
        "launch": "CUDA graph: counting sort by order + one persistent longest-first kernel "
                  "+ the fast subset convolution of the rows of orders >= fsc_from_n",
        "flops": "recursion count below fsc_from_n, fast-subset-convolution count from it on"}
    del g, A
    # a5 on the same uneven orders: Keldysh sums of 1D-chain real-time G0
    kflat, koff = inputs.keldysh_varlen(orders, seed=3)
    Mt = torch.as_tensor(kflat).to(dev)
    m_off = torch.as_tensor(koff).to(dev)
    kg = KeldyshVarlenGraph(Mt, m_off, n_t)
    ms = _event_ms(kg.replay)
    fl = sum(keldysh_flops(int(k)) for k in orders)
    rows["a5_keldysh_uneven_131072_n4to16"] = {
        "value": orders.size / (ms * 1e-3), "unit": "sums/s", "ms": ms,
        "tflops": fl / (ms * 1e-3) / 1e12, "frac_fp64_peak": fl / (ms * 1e-3) / 1e12 / peak,
        "warps_per_cta": tuned["keldysh_warps"] or 12, "tuned_by": "the autotuner of the a7 row"}
    del kg, Mt
    # a6: permanent minors, 4096 masked-uniform matrices of order 14
    P = torch.as_tensor(inputs.perm_batch(14, 4096, seed=4)).to(dev)
    ms = _event_ms(lambda: apm.perm_minors(P))
    fl = 4096 * perm_flops(14)
    rows["a6_perm_minors_4096_n14"] = {
        "value": 4096 / (ms * 1e-3), "unit": "perm-minor-sets/s", "ms": ms,
        "tflops": fl / (ms * 1e-3) / 1e12, "frac_fp64_peak": fl / (ms * 1e-3) / 1e12 / peak}
    del P
    # next (Sections III.B, V.B): Nambu CDet, 65536 BCS Nambu matrices of order 12:
    # XNOR minors of the 24 x 24 matrices, then the CDet recursion on them
    M = torch.as_tensor(inputs.nambu_batch(65536, 12, seed=6)).to(dev)
    ms = _event_ms(lambda: apm.nambu_cdet(M))
    xm = apm.xnor_minors(M)
    ms_x = _event_ms(lambda: apm.xnor_minors(M))
    fl = 65536 * (xnor_flops(12) + sc_flops(12))
    rows["nambu_cdet_65536_n12"] = {
        "value": 65536 / (ms * 1e-3), "unit": "minor-sets/s", "ms": ms,
        "tflops": fl / (ms * 1e-3) / 1e12, "frac_fp64_peak": fl / (ms * 1e-3) / 1e12 / peak,
        "xnor_minors_ms": ms_x, "xnor_minors_tflops": 65536 * xnor_flops(12) / (ms_x * 1e-3) / 1e12,
        "launch": "XNOR-minor kernel, then the CDet recursion on the minors"}
    del M, xm
    # next (Section V.D with Eq. CTINT): two-spin Keldysh sums of 16384 chain pairs
    # of order 12 (Zeeman-split spins, one shared assignment)
    Mu, Md = inputs.keldysh2_batch(16384, 12, seed=8)
    Mu, Md = torch.as_tensor(Mu).to(dev), torch.as_tensor(Md).to(dev)
    ms = _event_ms(lambda: apm.keldysh2_sum(Mu, Md))
    fl = 16384 * keldysh2_flops(12)
    rows["keldysh2_16384_n12"] = {
        "value": 16384 / (ms * 1e-3), "unit": "sums/s", "ms": ms,
        "tflops": fl / (ms * 1e-3) / 1e12, "frac_fp64_peak": fl / (ms * 1e-3) / 1e12 / peak}
    del Mu, Md
    # next (Sections III.C, V.C): CDet summed over two vertex types, 16384 Hubbard
    # matrices of order 10 with a shifted second vertex type: NAND minors summed
    # over the types of each subset, then the CDet recursion
    M = torch.as_tensor(inputs.two_type_batch(16384, 10, seed=7)).to(dev)
    ms = _event_ms(lambda: apm.two_type_cdet(M))
    fl = 16384 * (nand_flops(10) + sc_flops(10))
    rows["two_type_cdet_16384_n10"] = {
        "value": 16384 / (ms * 1e-3), "unit": "minor-sets/s", "ms": ms,
        "tflops": fl / (ms * 1e-3) / 1e12, "frac_fp64_peak": fl / (ms * 1e-3) / 1e12 / peak,
        "launch": "NAND-minor kernel (type sums), then the CDet recursion"}
    del M
    # a1 alone (Section II): all 2^12 minors of the 65536 Hubbard matrices, no
    # recursion (one warp per matrix; small pivots redone by the fused kernel)
    A = torch.as_tensor(inputs.hubbard_batch(65536, 12, seed=2)).to(dev)
    ms = _event_ms(lambda: apm.all_minors(A))
    fl = 65536 * minors_flops(12)
    rows["all_minors_65536_n12"] = {
        "value": 65536 / (ms * 1e-3), "unit": "minor-sets/s", "ms": ms,
        "tflops": fl / (ms * 1e-3) / 1e12, "frac_fp64_peak": fl / (ms * 1e-3) / 1e12 / peak,
        "minors_written_gbs": 65536 * 8 * 4096 / (ms * 1e-3) / 1e9,
        "launch": "warp-per-matrix minors kernel, then the fused kernel on the flagged matrices"}
    del A
    torch.cuda.empty_cache()
    # Section II at orders past the fused kernel's own: all 2^24 minors of 16
    # matrices of order 24 (the upper 12 levels breadth first, 16 x 4096 leaves of
    # order 12 through the warp-per-matrix minors kernel, scaled); 2.1 GB of minors
    A = torch.as_tensor(np.random.default_rng(24).standard_normal((16, 24, 24)) + 2.0 * np.eye(24)).to(dev)
    ms = _event_ms(lambda: apm.all_minors(A))
    fl = 16 * minors_flops(24)
    out_bytes = 16 * 8 * 2 ** 24
    rows["all_minors_16_n24"] = {
        "value": 16 / (ms * 1e-3), "unit": "minor-sets/s", "ms": ms,
        "tflops": fl / (ms * 1e-3) / 1e12, "frac_fp64_peak": fl / (ms * 1e-3) / 1e12 / peak,
        "minors_written_gbs": out_bytes / (ms * 1e-3) / 1e9,
        "launch": "12 upper-level launches, the minors kernels on the 65536 leaves (the redone ones from the same root minors), back-propagation, status"}
    del A
    torch.cuda.empty_cache()
    # next (Section V.A): the connected sums by the fast subset convolution against
    # the direct recursion, from the same weights (det^2 of Hubbard matrices)
    fsc = {}
    # batches are multiples of 456 at the larger orders (3 resident CTAs on each of
    # 152 SMs for both kernels), so that no launch ends with a part-empty round
    for n, B in ((12, 16416), (13, 8208), (14, 2280), (15, 1368), (16, 456)):
        A = torch.as_tensor(inputs.hubbard_batch(B, n, seed=9)).to(dev)
        m = apm.all_minors(A)
        a = m * m
        del A, m
        ms_d = _event_ms(lambda: apm.cdet_from_weights(a))
        ms_f = _event_ms(lambda: apm.cdet_from_weights_fsc(a))
        fsc[str(n)] = {"batch": B, "recursion_ms": ms_d, "fsc_ms": ms_f, "fsc_over_recursion": ms_f / ms_d,
                       "recursion_tflops": B * sc_flops(n) / (ms_d * 1e-3) / 1e12,
                       "fsc_tflops_of_unpruned_count": B * fsc_flops(n) / (ms_f * 1e-3) / 1e12,
                       "fsc_over_recursion_flops": fsc_flops(n) / sc_flops(n)}
        del a
        torch.cuda.empty_cache()
    rows["cdet_fsc_vs_recursion_n12to16"] = fsc
    # a8: learned proposal vs plain, 16384 walkers at each order 10..14
    G = torch.as_tensor(inputs.hubbard_g0_table()).to(dev)
    W, T = 16384, args.mc_steps
    walkers, feats, targs = {}, [], []
    # untimed warm-up of every part of this row (collection, training, plain
    # and delayed-acceptance steps) on throwaway walkers and a throwaway
    # network: the first use of some kernels in a process loads or compiles
    # them, seconds on a fresh box
    wu = mc.Walkers(1024, 10, G, inputs.HUB_WIN, inputs.HUB_MTAU, seed=99)
    Fw, tw = wu.collect(2)
    net_w = mc.Surrogate(seed=99, max_batch=1024)
    net_w.train(Fw, tw, epochs=1, batch=1024)
    wu.step_plain(record=[])
    wu.init_surrogate(net_w)
    wu.step_da(net_w, record=[])
    del wu, Fw, tw, net_w
    t_collect = 0.0
    for n in range(10, 15):
        wk = mc.Walkers(W, n, G, inputs.HUB_WIN, inputs.HUB_MTAU, seed=100 + n)
        (F, t), dt = mc.timed(lambda: wk.collect(30))
        t_collect += dt
        feats.append(F)
        targs.append(t)
        walkers[n] = wk
    net = mc.Surrogate(seed=7, max_batch=W)
    losses, t_train = mc.timed(lambda: net.train(torch.cat(feats), torch.cat(targs), epochs=1, batch=8192,
                                                 lr=3e-3))
    net.check()
    # the surrogate's tensor-core GEMMs at the walkers' batch (context: not the
    # FP64 roofline): the forward pass (three GEMMs and the head), and the
    # 16384 x 256 x 256 hidden-layer GEMM alone, against the measured BF16 peak
    gen = torch.Generator(device="cpu").manual_seed(17)
    Fq = (torch.randn((W, 64), generator=gen) * 0.5).to(torch.bfloat16).view(torch.int16).to(dev)
    yq = torch.empty(W, dtype=torch.float32, device=dev)
    ms_fwd = _event_ms(lambda: net.forward_raw(Fq, yq), reps=20)
    Ag = torch.randn((W, 256), generator=gen).to(torch.bfloat16).to(dev)
    Bg = torch.randn((256, 256), generator=gen).to(torch.bfloat16).to(dev)
    Cg = torch.empty((W, 256), dtype=torch.bfloat16, device=dev)

    def hidden_gemm():
        apm._check(mc.lib().apm_mlp_gemm_tn(mc._p(Ag), mc._p(Bg), None, None, mc._p(Cg), W, 256, 256, 1,
                                            mc._p(net.ws), net.ws.numel(), mc._s(Ag)), "apm_mlp_gemm_tn")
    ms_gemm = _event_ms(hidden_gemm, reps=50)
    net.check()
    # the same product by the vendor library (torch.matmul -> cuBLAS), for context only
    ms_lib = _event_ms(lambda: torch.relu(torch.matmul(Ag, Bg.t())), reps=50)
    bf16_peak = _measured_peaks().get("bf16_tflops")
    fwd_tf = 2 * W * (64 * 256 + 2 * 256 * 256) / (ms_fwd * 1e-3) / 1e12
    gemm_tf = 2 * W * 256 * 256 / (ms_gemm * 1e-3) / 1e12
    surrogate = {"forward_us": ms_fwd * 1e3, "forward_gemm_tflops": fwd_tf,
                 "hidden_gemm_16384x256x256_us": ms_gemm * 1e3, "hidden_gemm_tflops": gemm_tf,
                 "bf16_peak_tflops": bf16_peak,
                 "hidden_gemm_frac_bf16_peak": gemm_tf / bf16_peak if bf16_peak else None,
                 "hidden_gemm_cublas_us_context": ms_lib * 1e3,
                 "train_step_8192_us": t_train / max(len(losses), 1) * 1e6,
                 "kernel": "tcgen05.mma kind::f16, TMA loads, TMEM accumulator (one 128 x 128 tile per CTA)"}
    per_n = {}
    tot = {k: 0.0 for k in ("plain_s", "learned_s", "plain_ess_sign", "learned_ess_sign", "plain_ess_logc",
                            "learned_ess_logc", "learned_ess_ratio")}
    steps = {}
    for n, wk in walkers.items():
        T = args.mc_steps if n <= 12 else args.mc_steps_high
        steps[n] = T
        X0, w0, s0 = wk.X.clone(), wk.weight.clone(), wk.sign.clone()
        rec = []
        e0 = wk.exact_evals
        _, tp = mc.timed(lambda: [wk.step_plain(rec) for _ in range(T)])
        ep = wk.exact_evals - e0
        ess_ps, ess_pl = mc.ess(rec, 0), mc.ess(rec, 1)
        del rec
        wk.X.copy_(X0); wk.weight.copy_(w0); wk.sign.copy_(s0)
        rec = []
        e0 = wk.exact_evals

        def run_learned():
            wk.init_surrogate(net)
            for _ in range(T):
                wk.step_da(net, rec)
        _, tl = mc.timed(run_learned)
        el = wk.exact_evals - e0
        ess_ls, ess_ll, ess_lr = mc.ess(rec, 0), mc.ess(rec, 1), mc.ess(rec, 2)
        sign_mean = float(torch.stack([r[0] for r in rec]).mean())
        del rec
        fin = lambda x: x if np.isfinite(x) else None
        per_n[str(n)] = {"steps": T, "plain_s": tp, "learned_s": tl, "mean_sign": sign_mean,
                         "plain_ess_per_s_sign": fin(ess_ps / tp), "learned_ess_per_s_sign": fin(ess_ls / tl),
                         "plain_ess_per_s_logc": ess_pl / tp, "learned_ess_per_s_logc": ess_ll / tl,
                         "learned_ess_per_s_log_c_over_surrogate": fin(ess_lr / tl),
                         "plain_exact_evals_per_ess_logc": ep / ess_pl,
                         "learned_exact_evals_per_ess_logc": el / ess_ll}
        tot["plain_s"] += tp
        tot["learned_s"] += tl
        tot["plain_ess_logc"] += ess_pl
        tot["learned_ess_logc"] += ess_ll
        if np.isfinite(ess_ps) and np.isfinite(ess_ls):
            tot["plain_ess_sign"] += ess_ps
            tot["learned_ess_sign"] += ess_ls
    fixed = t_collect + t_train   # the learned arm also pays for its training pairs and the training
    gain = lambda key, extra: ((tot["learned_ess_" + key] / (tot["learned_s"] + extra)) /
                               (tot["plain_ess_" + key] / tot["plain_s"])) if tot["plain_ess_" + key] else None
    rows["a8_learned_proposal_16384_walkers_n10to14"] = {
        "metric": "effective samples/s (Sokal's adaptive window, mean autocorrelation over 16384 walkers) "
                  "of sgn c_n, i.e. at equal standard error of <sgn c_n>, summed over orders 10..14; "
                  "log|c_n| alongside",
        "plain_ess_per_s_sign": tot["plain_ess_sign"] / tot["plain_s"],
        "learned_ess_per_s_sign": tot["learned_ess_sign"] / tot["learned_s"],
        "gain_sign": gain("sign", 0.0),
        "gain_sign_incl_collection_and_training": gain("sign", fixed),
        "gain_logc": gain("logc", 0.0),
        "gain_logc_incl_collection_and_training": gain("logc", fixed),
        "value": tot["learned_ess_sign"] / (tot["learned_s"] + fixed), "unit": "effective samples/s",
        "steps_per_chain": {str(k): v for k, v in steps.items()}, "train_s": t_train, "collect_s": t_collect,
        "final_train_loss": float(np.mean(losses[-5:])), "per_order": per_n, "surrogate": surrogate}
    return rows


def rows_summary(rows: dict) -> dict:
    """Three numbers per row: [value, ms, fraction of the FP64 peak] for the
    kernel rows; [fast-subset-convolution time over the recursion's at n = 15,
    at n = 16, None] for that comparison; [learned effective samples/s of
    sgn c_n with collection and training counted, gain over plain at equal
    standard error without and with them] for the learned proposal."""
    def r(x, d=4):
        return None if x is None else float(f"{x:.{d}g}")
    out = {"fields": "kernel rows: value, ms, frac_fp64_peak; fsc: ratio n15, n16; a8: value, gain, gain_incl"}
    for k, v in rows.items():
        if not isinstance(v, dict):
            continue
        if k.startswith("a8"):
            out[k] = [r(v.get("value"), 6), r(v.get("gain_sign")), r(v.get("gain_sign_incl_collection_and_training"))]
        elif k.startswith("cdet_fsc"):
            out[k] = [r(v.get(str(m), {}).get("fsc_over_recursion")) for m in (15, 16)] + [None]
        else:
            out[k] = [r(v.get("value"), 6), r(v.get("ms"), 5), r(v.get("frac_fp64_peak"))]
    return out


def cpu_rate(run, A_np, seconds: float, threads: int):
    """Minor sets per second of run(sample, threads) -> c on `threads` host
    cores, over a bounded sample of the workload sized to about `seconds`."""
    import numpy as np
    run(A_np[:2], threads)                              # build + warm
    t0 = time.perf_counter()
    probe = A_np[:threads]
    run(probe, threads)
    per = (time.perf_counter() - t0) / probe.shape[0]
    count = int(max(threads, min(A_np.shape[0], seconds / max(per, 1e-9))))
    count = (count // threads) * threads or threads
    sample = A_np[:count]
    t0 = time.perf_counter()
    c = run(sample, threads)
    dt = time.perf_counter() - t0
    assert np.isfinite(c).all()
    return count / dt, threads, count, dt


def oracle_run(sample, threads):
    """The oracle's minor sets: one partial-pivot LU per minor, then the plain recursion."""
    import oracle
    m = oracle.minors_lu(sample, nthreads=threads)
    return oracle.cdet_recursion(m * m, nthreads=threads)


def fpm_sc_run(sample, threads):
    """The paper's own algorithm on the host: the depth-first tree with pivot
    correction, then the recursion (cpu_baseline/, C with OpenMP)."""
    import cpu_baseline
    return cpu_baseline.fpm_sc(sample, nthreads=threads)[1]


def cpu_oracle_rate(A_np, seconds: float):
    """Oracle minor sets per second on all the host cores (bounded sample)."""
    return cpu_rate(oracle_run, A_np, seconds, len(os.sched_getaffinity(0)))


def run_reference(args, rank, world):
    import numpy as np
    from paper_2104_07638_gb300 import inputs
    if rank != 0:
        return
    A = inputs.hubbard_batch(args.batch, N_ORDER, seed=2)
    per_step = max(1.0, args.cpu_seconds / max(1, args.steps + args.warmup))
    rates = []
    for i in range(args.warmup + args.steps):
        r, threads, count, dt = cpu_oracle_rate(A[(i * 97) % 1024:], per_step)
        if i >= args.warmup:
            rates.append((r, count, dt))
    done = sum(c for _, c, _ in rates)
    secs = sum(d for _, _, d in rates)
    value = done / secs
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        # the time of the work each step actually did: a sample of the batch
        "ms_per_step": 1000.0 * secs / len(rates), "matrices_per_step": done / len(rates),
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(N_ORDER, args.batch, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{done / len(rates):.0f} of the {args.batch} matrices per step, "
                                   f"{secs / len(rates):.2f} s per step (per-minor partial-pivot LU + "
                                   "plain recursion, OpenMP)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def profile_case(name: str):
    """Three launches of one kernel on a small case whose inputs and outputs
    exceed L2 (129 MB) while staying a few GB on the device."""
    import numpy as np
    import torch
    from paper_2104_07638_gb300 import apm, inputs
    dev = torch.device("cuda", 0)
    if name == "cdet_n12":
        A = torch.as_tensor(inputs.hubbard_batch(4096, 12, seed=2)).to(dev)
        run = lambda: apm.cdet_connected(A, return_minors=True)
    elif name == "cdet_n12_full":
        # the benchmark's launch: 65536 matrices, 4.3 GB of outputs (33 x L2), for DRAM counters only
        A = torch.as_tensor(inputs.hubbard_batch(65536, 12, seed=2)).to(dev)
        c = torch.empty((65536, 4096), dtype=torch.float64, device=dev)
        mo = torch.empty_like(c)
        run = lambda: apm.cdet_connected(A, out_c=c, out_minors=mo)
    elif name == "fp64_probe":
        # the FP64 throughput probe of the bench line (456 CTAs of 512 threads, 2048 iterations)
        run = lambda: apm.fp64_probe(SMS * 3, 512, 2048, dev)
    elif name == "cdet_n16":
        A = torch.as_tensor(inputs.hubbard_batch(304, 16, seed=2)).to(dev)
        run = lambda: apm.cdet_connected(A, return_minors=True)
    elif name == "keldysh_n12":
        M = torch.as_tensor(inputs.keldysh_batch(8192, 12, seed=3)).to(dev)
        run = lambda: apm.keldysh_sum(M)
    elif name == "xnor_n12":
        M = torch.as_tensor(inputs.nambu_batch(8192, 12, seed=6)).to(dev)
        run = lambda: apm.xnor_minors(M)
    elif name == "keldysh2_n12":
        Mu, Md = inputs.keldysh2_batch(8192, 12, seed=8)
        Mu, Md = torch.as_tensor(Mu).to(dev), torch.as_tensor(Md).to(dev)
        run = lambda: apm.keldysh2_sum(Mu, Md)
    elif name == "minors_n12":
        # the minors alone (one warp per matrix): 4096 matrices, 134 MB of minors (> L2)
        A = torch.as_tensor(inputs.hubbard_batch(4096, 12, seed=2)).to(dev)
        run = lambda: apm.all_minors(A)
    elif name == "minors_n20":
        # orders past 16: 64 matrices of order 20 (the upper levels, then 1024 leaves each)
        A = torch.as_tensor(np.random.default_rng(20).standard_normal((64, 20, 20)) + 2.0 * np.eye(20)).to(dev)
        run = lambda: apm.all_minors(A)
    elif name == "minors_n24":
        # the benchmark row: 16 matrices of order 24 (2.1 GB of minors; 4096 leaves of order 12 each)
        A = torch.as_tensor(np.random.default_rng(24).standard_normal((16, 24, 24)) + 2.0 * np.eye(24)).to(dev)
        run = lambda: apm.all_minors(A)
    elif name == "keldysh_uneven":
        # the uneven Keldysh batch of the a5 row on 16384 walkers (orders 4..16)
        orders = inputs.varlen_orders(16384, 4, 16, seed=3)
        kflat, koff = inputs.keldysh_varlen(orders, seed=3)
        Mt = torch.as_tensor(kflat).to(dev)
        m_off = torch.as_tensor(koff).to(dev)
        n_t = torch.as_tensor(orders).to(dev)
        run = lambda: apm.keldysh_sum_varlen(Mt, m_off, n_t)
    elif name == "nand_n10":
        M = torch.as_tensor(inputs.two_type_batch(16384, 10, seed=7)).to(dev)
        run = lambda: apm.two_type_cdet(M)
    elif name == "ppm_n14":
        P = torch.as_tensor(inputs.perm_batch(14, 1368, seed=4)).to(dev)
        run = lambda: apm.perm_minors(P)
    elif name == "fsc_n16":
        # connected sums by the fast subset convolution, 152 weight rows of order 16
        A = torch.as_tensor(inputs.hubbard_batch(152, 16, seed=9)).to(dev)
        m = apm.all_minors(A)
        a = m * m
        run = lambda: apm.cdet_from_weights_fsc(a)
    elif name == "mlp_gemm":
        # the surrogate's hidden-layer GEMM at the walkers' batch (16384 x 256 x 256,
        # BF16 out with bias and ReLU); operands fit in L2 at this size
        from paper_2104_07638_gb300 import mc
        gen = torch.Generator(device="cpu").manual_seed(17)
        Ag = torch.randn((16384, 256), generator=gen).to(torch.bfloat16).to(dev)
        Bg = torch.randn((256, 256), generator=gen).to(torch.bfloat16).to(dev)
        bias = torch.zeros(256, dtype=torch.float32, device=dev)
        Cg = torch.empty((16384, 256), dtype=torch.bfloat16, device=dev)
        import ctypes
        nb = ctypes.c_size_t(0)
        apm._check(mc.lib().apm_mlp_workspace_size(0, ctypes.byref(nb)), "apm_mlp_workspace_size")
        ws = torch.zeros(nb.value, dtype=torch.uint8, device=dev)
        run = lambda: apm._check(mc.lib().apm_mlp_gemm_tn(mc._p(Ag), mc._p(Bg), mc._p(bias), None, mc._p(Cg), 16384,
                                                          256, 256, 1, mc._p(ws), ws.numel(), mc._s(Ag)),
                                 "apm_mlp_gemm_tn")
    else:
        orders = inputs.varlen_orders(16384, 4, 16, seed=3)
        flat, off = inputs.hubbard_varlen(orders, seed=3)
        A = torch.as_tensor(flat).to(dev)
        a_off = torch.as_tensor(off).to(dev)
        n_t = torch.as_tensor(orders).to(dev)
        run = lambda: apm.cdet_connected_varlen(A, a_off, n_t)
    for _ in range(3):
        run()
    torch.cuda.synchronize()
    print(json.dumps({"case": name, "ok": True}))


def main():
    args = parse()
    if args.case:
        profile_case(args.case)
        return
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import numpy as np
    import torch
    from paper_2104_07638_gb300 import apm, inputs

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, B = N_ORDER, args.batch
    A_np = inputs.hubbard_batch_slice(world * B, n, 2, rank * B, (rank + 1) * B)
    A = torch.as_tensor(A_np).to(dev)
    N = 1 << n
    c = torch.empty((B, N), dtype=torch.float64, device=dev)
    mo = torch.empty((B, N), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # 256 MB > L2 (129 MB)
    stream = torch.cuda.current_stream(dev)

    def step():
        apm.cdet_connected(A, out_c=c, out_minors=mo)

    # FP64 throughput probe (roofline context): about a second of independent
    # FMA chains, with the SM clock sampled while it runs (one full wave: the
    # probe's 38 registers admit three CTAs of 512 threads per SM; its rate does
    # not depend on the launch shape)
    blocks, threads, iters, reps = SMS * 3, 512, 2048, 64
    apm.fp64_probe(blocks, threads, 64, dev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as pcs:
        e0.record(stream)
        for _ in range(reps):
            apm.fp64_probe(blocks, threads, iters, dev)
        e1.record(stream)
        torch.cuda.synchronize()
    probe_tflops = 32.0 * blocks * threads * iters * reps / (e0.elapsed_time(e1) * 1e-3) / 1e12
    probe_clocks = pcs.summary()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t_wall0 = time.perf_counter()
    with ClockSampler(local) as cs:
        for s0, s1 in evs:
            flush.random_(0, 255)                 # evict the inputs from L2 between steps
            s0.record(stream)
            step()
            s1.record(stream)
        torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    dev_s = max_over_ranks(sum(step_ms) * 1e-3, world)
    value = job_throughput(B, world, args.steps, dev_s)
    ms_per_step = 1000.0 * dev_s / args.steps

    # ---- end to end through the C ABI on host buffers (apm_cdet_connected_host) ----
    # chunks of 2048 matrices over 4 streams inside the library: the copies of
    # one chunk overlap the kernels of the others; the library cuts the last
    # two chunks' worth into halving pieces, so that the device->host copy left
    # exposed at the end is short
    chunks, nstreams = 32, 4
    cb = B // chunks
    A_host = torch.as_tensor(A_np).pin_memory()
    c_host = torch.empty((B, N), dtype=torch.float64).pin_memory()
    m_host = torch.empty((B, N), dtype=torch.float64).pin_memory()
    ws_host = torch.empty(max(apm.cdet_connected_host_workspace_size(n, cb, nstreams), 256), dtype=torch.uint8,
                          device=dev)

    def e2e_step():
        apm.cdet_connected_host(A_host, out_c=c_host, out_minors=m_host, chunk=cb, nstreams=nstreams,
                                workspace=ws_host)

    e2e_step()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(2, min(args.steps, 5))
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world)
    e2e_value = job_throughput(B, world, e2e_steps, e2e_s)
    # spot check of the end-to-end result against the device-timed one
    assert torch.equal(c_host[:4].to(dev), c[:4]) if rank == 0 else True

    # the one exchange of the data-parallel path: per-order sums of the
    # whole-set connected sums, reduced on the device, added over the ranks
    from paper_2104_07638_gb300 import dist as pdist
    est = pdist.estimator(pdist.combine_order_sums(apm.order_sums(c, n=n)))[n]

    import hashlib
    csrc = os.path.join(ROOT, "paper_2104_07638_gb300", "csrc")
    sha = hashlib.sha256(b"".join(open(os.path.join(csrc, f), "rb").read()
                                  for f in ("fpm_cdet.cu", "apm_internal.cuh"))).hexdigest()[:16]
    traffic = TRAFFIC_PER_SET * B if sha == TRAFFIC_SRC_SHA else None
    F = flops_per_set(n)
    peak = FP64_FLOP_PER_CLK_SM * SMS * SM_MAX_MHZ * 1e6 / 1e12
    achieved = F * B / (ms_per_step * 1e-3) / 1e12
    clocks = cs.summary()
    # the per-row measurements are single-GPU kernel timings: taken at N = 1
    # only, so that a multi-GPU launch ends with its timed steps
    rows = measure_rows(args, dev, peak) if rank == 0 and world == 1 and not args.no_rows else None
    result = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
    }
    if rows:
        # every row in three numbers, early in the line (it survives a truncated tail)
        result["rows_summary"] = rows_summary(rows)
    result.update({
        "config": bench_config(n, B, world),
        "timing": "CUDA events around each step on the launching stream",
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "traffic_note": "dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture of this "
                                     "launch (65536 matrices), per launch",
                     "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2070 MHz "
                                    "(nominal 1.25 TFLOP/s FP64 at max clock)",
                     "flops_per_set": F, "fp64_probe_tflops": probe_tflops,
                     "fp64_probe_sm_mhz": probe_clocks.get("sm_mhz"),
                     "hbm_gbs": bytes_per_set(n) * B / (ms_per_step * 1e-3) / 1e9},
        "e2e": {"value": e2e_value, "unit": UNIT,
                "h2d_bytes_per_step": int(A_host.numel() * 8),
                "d2h_bytes_per_step": int((c_host.numel() + m_host.numel()) * 8)},
        "gpu_launches": args.steps,
        "clocks": clocks,
        "wall_s_timed_region": t_wall,
        "estimator": {"order": n, "ranks": world, "count": est["count"], "mean_c": est["mean"],
                      "stderr": est["stderr"], "mean_abs_c": est["mean_abs"], "sign": est["sign"],
                      "exchange": "apm_order_sums per rank, summed over the ranks on the host"},
    })
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, threads, count, dt = cpu_oracle_rate(A_np, args.cpu_seconds)
        r1, _, count1, dt1 = cpu_rate(oracle_run, A_np, args.cpu_seconds / 4, 1)
        f, _, fcount, fdt = cpu_rate(fpm_sc_run, A_np, args.cpu_seconds / 3, threads)
        f1, _, fcount1, fdt1 = cpu_rate(fpm_sc_run, A_np, args.cpu_seconds / 4, 1)
        result["cpu_baseline"] = {
            "value": r, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{count} of the {B} matrices (per-minor partial-pivot LU + plain recursion, "
                      f"OpenMP), {dt:.1f} s",
            "value_1core": r1, "sample_1core": f"{count1} matrices on 1 core, {dt1:.1f} s",
            "fpm_sc": {"value": f, "unit": UNIT, "cores": threads, "value_1core": f1,
                       "kind": "the paper's depth-first tree with pivot correction + the recursion, C/OpenMP",
                       "sample": f"{fcount} matrices on {threads} cores ({fdt:.1f} s), "
                                 f"{fcount1} on 1 core ({fdt1:.1f} s)"}}
    if rows:
        # the full rows last: the contract's keys all come before them
        result["rows"] = rows
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
