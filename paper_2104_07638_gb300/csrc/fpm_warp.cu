// All principal minors, one warp per matrix (orders 9..16, minors only).
//
// Paper: Section II (Eq. minor, Alg. 1): the minor of a kept set is the minor
// of the set without its last decided element times the pivot of the Schur
// complement reached on its tree path.
//
// The fused minors / connected-sum kernel runs one matrix per CTA, which pays
// when the recursion follows; for the minors alone its tree levels, one CTA
// barrier each, leave the SM waiting. Here a warp takes a matrix, as in the
// XNOR and NAND kernels: elements are decided from the last one down, the
// upper n-9 depth first (the matrices of kept pivots on a per-warp stack in
// caller scratch), the last 9 breadth first in shared memory (a node of level
// J holds the Schur complement on elements 0 .. 8-J of the elements kept on
// its path; child 2i drops element 8-J, the leading block; child 2i+1 keeps
// it, the leading block less the rank-1 term over the pivot), and the 16
// principal minors of every 4 x 4 node of the last level in closed form. Node
// i of that level is element e's decision in bit e-4 of i, so lane i writes
// the 16 minors of the sets (i << 4) | X contiguously, and a tail fills 2^9
// consecutive entries of the row.
//
// Pivot correction (Section II): this kernel shifts nothing. A matrix that
// meets a pivot with |p| <= thr ||A||max is flagged, and the fused kernel,
// launched after it on the flagged matrices only, computes them again with
// the correction and its back-propagation.
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "apm_internal.cuh"

namespace apm {

constexpr int kFwTail = 9;   // elements expanded breadth first
constexpr int kFwWarps = 4;  // warps per CTA
constexpr int kFwMaxN = 16;

// Tail level J (J = 0..S-4) holds 2^J nodes of size S-J; even levels in bufE,
// odd in bufO. S = 9: bufE 81, 196, 400; bufO 128, 288, 512.
__host__ __device__ constexpr int fw_level_entries(int S, int J) { return (1 << J) * (S - J) * (S - J); }
__host__ __device__ constexpr int fw_buf_entries(int S, int parity) {
    int b = 0;
    for (int J = parity; J <= S - 4; J += 2) b = b > fw_level_entries(S, J) ? b : fw_level_entries(S, J);
    return b;
}
constexpr int kFwBufE = fw_buf_entries(kFwTail, 0);
constexpr int kFwBufO = fw_buf_entries(kFwTail, 1);
static_assert(kFwBufE == 400 && kFwBufO == 512, "9-element tail");
// row factors: one per row of every kept child (2^J (S-J-1), at most 16 x 4), or
// of one depth-first step (at most 15)
constexpr int kFwFac = 64;

struct alignas(16) FwWarpSmem {
    double bufE[kFwBufE];
    double bufO[kFwBufO];
    double f[kFwFac];
    double inv[1 << (kFwTail - 5)];  // reciprocal pivots of one level (at most 16 nodes)
    double nd[2][1 << (kFwTail - 4)];  // node minors of the current and the next level
    double pdet[kFwMaxN + 1];
    const double *vp[kFwMaxN + 1];  // depth-first views: first element and row stride
    int vs[kFwMaxN + 1];
};
static_assert(sizeof(FwWarpSmem) % 16 == 0, "per-warp blocks stay 16-byte aligned");

// stack entries (doubles) for order n: the kept-pivot matrices of depths 1..D-1 (D = n - 9)
__host__ __device__ constexpr size_t fw_stack_entries(int n) {
    const int D = n > kFwTail ? n - kFwTail : 0;
    size_t t = 0;
    for (int d = 1; d < D; ++d) t += static_cast<size_t>(n - d) * (n - d);
    return t;
}

// 1/p for a pivot (flags a zero or non-finite one) and whether |p| <= thrA
__device__ __forceinline__ double fw_inv(double p, double thrA, int &bad, int &small) {
    const long long bits = __double_as_longlong(p);
    if ((bits << 1) == 0 || ((bits >> 52) & 0x7ff) == 0x7ff) bad = 1;
    small |= fabs(p) <= thrA;
    return rcp_nr(p);
}

// One breadth-first level J of the tail: 2^J nodes of size k = S-J in cur give
// 2^(J+1) children of size k-1 in nxt.
template <int S, int J>
__device__ __forceinline__ void fw_tail_level(const double *cur, double *nxt, FwWarpSmem &w, int lane, double thrA,
                                              int &bad, int &small) {
    constexpr int k = S - J, k1 = k - 1, kk = k * k, kk1 = k1 * k1, nodes = 1 << J;
    const double *ndc = w.nd[J & 1];
    double *ndn = w.nd[(J + 1) & 1];
    for (int i = lane; i < nodes; i += 32) {
        const double p = cur[i * kk + k1 * k + k1];
        w.inv[i] = fw_inv(p, thrA, bad, small);
        ndn[2 * i] = ndc[i];
        ndn[2 * i + 1] = ndc[i] * p;
    }
    __syncwarp();
    for (int idx = lane; idx < nodes * k1; idx += 32) {
        const int i = idx / k1, r = idx - i * k1;
        w.f[idx] = cur[i * kk + r * k + k1] * w.inv[i];
    }
    __syncwarp();
    for (int e = lane; e < nodes * kk1; e += 32) {
        const int i = e / kk1, rem = e - i * kk1, r = rem / k1, q = rem - r * k1;
        const double *P = cur + i * kk;
        const double v = P[r * k + q];
        nxt[(2 * i) * kk1 + rem] = v;
        nxt[(2 * i + 1) * kk1 + rem] = fma(-w.f[i * k1 + r], P[k1 * k + q], v);
    }
    __syncwarp();
}

// The 16 principal minors of every 4 x 4 node i (node minor d = nd[i]) in
// closed form, out[16 i + X] for X within {0,1,2,3}: with s_jk the 2 x 2 minors
// of rows 0,1 and c_jk those of rows 2,3 on columns j,k, the triples by
// expansion along their third row and the whole by Laplace expansion along rows
// 0,1. Row 0 is scaled by d first, so that every minor holding element 0 comes
// out scaled; the other seven are multiplied by d. No pivot, no division.
template <int S>
__device__ __forceinline__ void fw_bottom(const double *cur, const double *nd, double *out, int lane) {
    constexpr int nodes = 1 << (S - 4);
    for (int i = lane; i < nodes; i += 32) {
        const double *M = cur + 16 * i;
        const double d = nd[i];
        const double a0 = d * M[0], a1 = d * M[1], a2 = d * M[2], a3 = d * M[3];
        const double s01 = fma(a0, M[5], -a1 * M[4]), s02 = fma(a0, M[6], -a2 * M[4]);
        const double s03 = fma(a0, M[7], -a3 * M[4]), s12 = fma(a1, M[6], -a2 * M[5]);
        const double s13 = fma(a1, M[7], -a3 * M[5]), s23 = fma(a2, M[7], -a3 * M[6]);
        const double c01 = fma(M[8], M[13], -M[9] * M[12]), c02 = fma(M[8], M[14], -M[10] * M[12]);
        const double c03 = fma(M[8], M[15], -M[11] * M[12]), c12 = fma(M[9], M[14], -M[10] * M[13]);
        const double c13 = fma(M[9], M[15], -M[11] * M[13]), c23 = fma(M[10], M[15], -M[11] * M[14]);
        const double p02 = fma(a0, M[10], -a2 * M[8]), p03 = fma(a0, M[15], -a3 * M[12]);
        const double p12 = fma(M[5], M[10], -M[6] * M[9]), p13 = fma(M[5], M[15], -M[7] * M[13]);
        const double t012 = fma(M[10], s01, fma(-M[9], s02, M[8] * s12));
        const double t013 = fma(M[15], s01, fma(-M[13], s03, M[12] * s13));
        const double t023 = fma(a0, c23, fma(-a2, c03, a3 * c02));
        const double t123 = fma(M[5], c23, fma(-M[6], c13, M[7] * c12));
        double q = s01 * c23;
        q = fma(-s02, c13, q);
        q = fma(s03, c12, q);
        q = fma(s12, c03, q);
        q = fma(-s13, c02, q);
        q = fma(s23, c01, q);
        double2 *o = reinterpret_cast<double2 *>(out + 16 * i);
        o[0] = make_double2(d, a0);
        o[1] = make_double2(d * M[5], s01);
        o[2] = make_double2(d * M[10], p02);
        o[3] = make_double2(d * p12, t012);
        o[4] = make_double2(d * M[15], p03);
        o[5] = make_double2(d * p13, t013);
        o[6] = make_double2(d * c23, t023);
        o[7] = make_double2(d * t123, q);
    }
}

template <int S, int J>
__device__ __forceinline__ void fw_tail_levels(double *cur, double *nxt, double *out, FwWarpSmem &w, int lane,
                                               double thrA, int &bad, int &small) {
    if constexpr (J <= S - 5) {
        fw_tail_level<S, J>(cur, nxt, w, lane, thrA, bad, small);
        fw_tail_levels<S, J + 1>(nxt, cur, out, w, lane, thrA, bad, small);
    } else {
        fw_bottom<S>(cur, w.nd[J & 1], out, lane);
    }
}

// One matrix of order n (9..16), whole warp: its 2^n minors, each times pre,
// into out. Returns 1 when a pivot is below thrA or zero (the fused kernel
// redoes the matrix) or the input is not finite (the fused kernel then sets the
// status and NaN).
__device__ __forceinline__ int fw_matrix(const double *A, int n, double *out, double thr, double pre, double *stack,
                                         FwWarpSmem &w, int lane) {
    const int D = n - kFwTail;
    int bad = 0, small = 0, nonfin = 0;
    double amax = 0.0;
    for (int e = lane; e < n * n; e += 32) {
        const double x = A[e];
        if (!isfinite(x)) nonfin = 1;
        amax = fmax(amax, fabs(x));
    }
    nonfin = __any_sync(0xffffffffu, nonfin);
    if (nonfin) return 1;
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    const double thrA = thr * (amax > 0.0 ? amax : 1.0);
    if (lane == 0) {
        w.vp[0] = A;
        w.vs[0] = n;
        w.pdet[0] = pre;
    }
    __syncwarp();
    for (int64_t t = 0; t < (int64_t(1) << D); ++t) {
        // first depth whose decision changed from t-1 to t (element n-1 <-> top bit)
        const int d0 = t == 0 ? 0 : D - __ffsll(t);
        for (int d = d0; d < D; ++d) {
            const int keep = static_cast<int>((t >> (D - 1 - d)) & 1);
            const double *P = w.vp[d];
            const int st = w.vs[d], k = n - d, k1 = k - 1;
            double *dst = w.bufE;
            if (d + 1 < D) {  // stack slot of depth d+1
                size_t off = 0;
                for (int j = 1; j <= d; ++j) off += static_cast<size_t>(n - j) * (n - j);
                dst = stack + off;
            }
            if (keep) {
                const double piv = P[k1 * st + k1];
                const double iv = fw_inv(piv, thrA, bad, small);
                for (int r = lane; r < k1; r += 32) w.f[r] = P[r * st + k1] * iv;
                __syncwarp();
                for (int e = lane; e < k1 * k1; e += 32) {
                    const int r = e / k1, q = e - r * k1;
                    dst[e] = fma(-w.f[r], P[k1 * st + q], P[r * st + q]);
                }
                __syncwarp();
                if (lane == 0) {
                    w.vp[d + 1] = dst;
                    w.vs[d + 1] = k1;
                    w.pdet[d + 1] = w.pdet[d] * piv;
                }
            } else {
                if (d + 1 == D) {  // the tail root must be dense
                    for (int e = lane; e < k1 * k1; e += 32) {
                        const int r = e / k1, q = e - r * k1;
                        w.bufE[e] = P[r * st + q];
                    }
                }
                if (lane == 0) {
                    w.vp[d + 1] = d + 1 == D ? w.bufE : P;
                    w.vs[d + 1] = d + 1 == D ? k1 : st;
                    w.pdet[d + 1] = w.pdet[d];
                }
            }
            __syncwarp();
        }
        if (D == 0) {  // the whole matrix is the tail root
            for (int e = lane; e < n * n; e += 32) w.bufE[e] = A[e];
        }
        if (lane == 0) w.nd[0][0] = w.pdet[D];
        __syncwarp();
        fw_tail_levels<kFwTail, 0>(w.bufE, w.bufO, out + (t << kFwTail), w, lane, thrA, bad, small);
        __syncwarp();
    }
    return __any_sync(0xffffffffu, bad | small);
}

// Every matrix; redo[b] = 1 where the fused kernel must compute it again. pre
// (or NULL for 1): a factor per matrix on all its minors.
__global__ void __launch_bounds__(kFwWarps * 32, 4) fpm_warp_kernel(const double *__restrict__ A, int n,
                                                                  int64_t batch, double *minors, double thr,
                                                                  const double *__restrict__ pre, uint32_t *redo,
                                                                  uint32_t *status, double *stack_base,
                                                                  size_t stack_per_warp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    FwWarpSmem &w = reinterpret_cast<FwWarpSmem *>(smem_raw)[wid];
    const int64_t gw = static_cast<int64_t>(blockIdx.x) * kFwWarps + wid;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * kFwWarps;
    double *stack = stack_base ? stack_base + gw * stack_per_warp : nullptr;
    const int64_t nn = static_cast<int64_t>(n) * n, N = int64_t(1) << n;
    for (int64_t b = gw; b < batch; b += nw) {
        const int r = fw_matrix(A + b * nn, n, minors + b * N, thr, pre ? pre[b] : 1.0, stack, w, lane);
        if (lane == 0) {
            redo[b] = static_cast<uint32_t>(r);
            if (status && !r) status[b] = 0u;
        }
    }
}

int fpm_warp_grid(int64_t batch, int *err) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = kFwWarps * sizeof(FwWarpSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fpm_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fpm_warp_kernel, kFwWarps * 32, smem);
    if (e != cudaSuccess || per_sm < 1) {
        *err = e != cudaSuccess ? static_cast<int>(e) : static_cast<int>(cudaErrorInvalidConfiguration);
        return 0;
    }
    *err = 0;
    const int64_t need = (batch + kFwWarps - 1) / kFwWarps;
    int64_t g = static_cast<int64_t>(sms) * per_sm;
    if (need < g) g = need;
    return static_cast<int>(g < 1 ? 1 : g);
}

// Workspace: per resident warp the depth-first stack, one redo flag per
// matrix, and for n > 12 the fused kernel's global scratch (its redo launch).
struct FwPlan {
    size_t stack, redo, fused, total;
};
static int fw_plan(int n, int64_t batch, FwPlan *p, int *grid) {
    int err = 0;
    *grid = fpm_warp_grid(batch, &err);
    if (err) return err;
    auto al = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
    p->stack = al(static_cast<size_t>(*grid) * kFwWarps * fw_stack_entries(n) * sizeof(double));
    p->redo = al(static_cast<size_t>(batch) * sizeof(uint32_t));
    p->fused = 0;
    if (n > cdet_smem_max_n(false)) {
        const int g = cdet_grid(n, batch, false, false, &err);
        if (err) return err;
        p->fused = al(static_cast<size_t>(g) * cdet_slot_doubles(n) * sizeof(double));
    }
    p->total = p->stack + p->redo + p->fused;
    return 0;
}

size_t fpm_warp_workspace_bytes(int n, int64_t batch, int *err) {
    *err = 0;
    if (batch == 0) return 0;
    FwPlan p;
    int grid = 0;
    *err = fw_plan(n, batch, &p, &grid);
    return *err ? 0 : p.total;
}

int launch_fpm_warp(const double *A, int n, int64_t batch, double *minors, double thr, double shf,
                    uint32_t *status, void *workspace, cudaStream_t s, const double *pre, uint32_t **redo_out) {
    FwPlan plan;
    int grid = 0;
    int err = fw_plan(n, batch, &plan, &grid);
    if (err) return err;
    const size_t smem = kFwWarps * sizeof(FwWarpSmem);
    const size_t per = fw_stack_entries(n);
    char *ws = static_cast<char *>(workspace);
    double *stack = per ? reinterpret_cast<double *>(ws) : nullptr;
    uint32_t *redo = reinterpret_cast<uint32_t *>(ws + plan.stack);
    double *fused = plan.fused ? reinterpret_cast<double *>(ws + plan.stack + plan.redo) : nullptr;
    if (redo_out) *redo_out = redo;
    fpm_warp_kernel<<<grid, kFwWarps * 32, smem, s>>>(A, n, batch, minors, thr, pre, redo, status, stack, per);
    err = static_cast<int>(cudaGetLastError());
    if (err) return err;
    // the flagged matrices again, by the fused kernel with the pivot correction
    // (without the factor pre: the caller scales those rows)
    CdetArgs a = {};
    a.A_up = A;
    a.minors_out = minors;
    a.status = status;
    a.batch = batch;
    a.n = n;
    a.mode = kModeMinors;
    a.piv_thr = thr;
    a.piv_shift = shf;
    a.redo = redo;
    a.gscratch = fused;
    return launch_fpm_cdet(a, s);
}

}  // namespace apm
