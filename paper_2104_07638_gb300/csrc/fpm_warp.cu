// All principal minors, one warp per matrix (orders 9..16, minors only).
//
// Paper: Section II (Eq. minor, Alg. 1): the minor of a kept set is the minor
// of the set without its last decided element times the pivot of the Schur
// complement reached on its tree path.
//
// The fused minors / connected-sum kernel runs one matrix per CTA, which pays
// when the recursion follows; for the minors alone its tree levels, one CTA
// barrier each, leave the SM waiting. Here a warp takes a matrix, as in the
// XNOR and NAND kernels, and elements are decided from the last one down. The
// FP64 pipe is the bound (one warp instruction per 16 SM cycles), and it is
// charged for a whole warp instruction whatever the number of active lanes, so
// the tree is laid out to keep the lanes busy:
//   * above the last T = min(n, 12) elements, depth first (the matrices of kept
//     pivots on a per-warp stack in caller scratch);
//   * the first 5 levels of the T-element tail breadth first in shared memory
//     (a node of level J holds the Schur complement on elements 0 .. T-1-J of
//     the elements kept on its path; child 2i drops element T-1-J, the leading
//     block; child 2i+1 keeps it, the leading block less the rank-1 term over
//     the pivot), which leaves 32 nodes of order L = T - 5;
//   * lane i then takes node i and finishes its whole subtree in registers:
//     fully unrolled Schur steps down to order 3, and the 8 principal minors of
//     each 3 x 3 node in closed form (row 0 scaled by the node minor first, the
//     whole by expansion along row 0; no pivot, no division).
// Node i of the lane level carries element e's decision in bit e - L, so lane i
// writes the minors of the sets (i << L) | X, X within 0 .. L-1, contiguously.
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

constexpr int kFwTail = 12;   // elements below the depth-first part
constexpr int kFwBfs = 5;     // tail levels expanded breadth first (32 nodes after them)
constexpr int kFwWarps = 4;   // warps per CTA
constexpr int kFwMaxN = 16;

// Tail level J (J = 0..kFwBfs) holds 2^J nodes of size T-J; even levels in
// bufE, odd in bufO. T = 12: bufE 144, 400, 1024; bufO 242, 648, 1568.
__host__ __device__ constexpr int fw_level_entries(int T, int J) { return (1 << J) * (T - J) * (T - J); }
__host__ __device__ constexpr int fw_buf_entries(int T, int parity) {
    int b = 0;
    for (int J = parity; J <= kFwBfs; J += 2) b = b > fw_level_entries(T, J) ? b : fw_level_entries(T, J);
    return b;
}
constexpr int kFwBufE = fw_buf_entries(kFwTail, 0);
constexpr int kFwBufO = fw_buf_entries(kFwTail, 1);
static_assert(kFwBufE == 1024 && kFwBufO == 1568, "12-element tail");
// row factors of one breadth-first level (2^J (T-J-1), at most 16 x 7), or of
// one depth-first step (at most 15)
constexpr int kFwFac = 112;

struct alignas(16) FwWarpSmem {
    double bufE[kFwBufE];
    double bufO[kFwBufO];
    double f[kFwFac];
    double inv[1 << (kFwBfs - 1)];  // reciprocal pivots of one level (at most 16 nodes)
    double nd[2][1 << kFwBfs];      // node minors of the current and the next level
    double pdet[kFwMaxN + 1];
    const double *vp[kFwMaxN + 1];  // depth-first views: first element and row stride
    int vs[kFwMaxN + 1];
};
static_assert(sizeof(FwWarpSmem) % 16 == 0, "per-warp blocks stay 16-byte aligned");

// stack entries (doubles) for order n: the kept-pivot matrices of depths 1..D-1 (D = n - 12)
__host__ __device__ constexpr size_t fw_stack_entries(int n) {
    const int D = n > kFwTail ? n - kFwTail : 0;
    size_t t = 0;
    for (int d = 1; d < D; ++d) t += static_cast<size_t>(n - d) * (n - d);
    return t;
}

// 1/p for a pivot; fl gets 1 for a zero or non-finite one and where |p| <= thrA
// (thrA >= 0), tested on the high words in integer arithmetic (off the FP64
// pipe): it also flags pivots up to 2^-20 (relative) above thrA, which only
// sends such a matrix to the fused kernel, whose own test is exact. One flag
// for both (the caller only needs to know whether to redo the matrix) keeps
// the order-7 lane subtree within 255 registers without a spill.
__device__ __forceinline__ double fw_inv(double p, double thrA, int &fl) {
    const long long bits = __double_as_longlong(p);
    fl |= ((bits << 1) == 0) | (((bits >> 52) & 0x7ff) == 0x7ff) |
          ((static_cast<unsigned>(__double2hiint(p)) & 0x7fffffffu) <= static_cast<unsigned>(__double2hiint(thrA)));
    return rcp_nr(p);
}

// One breadth-first level J of a T-element tail: 2^J nodes of size k = T-J in
// cur give 2^(J+1) children of size k-1 in nxt.
template <int T, int J>
__device__ __forceinline__ void fw_tail_level(const double *cur, double *nxt, FwWarpSmem &w, int lane, double thrA,
                                              int &fl) {
    constexpr int k = T - J, k1 = k - 1, kk = k * k, kk1 = k1 * k1, nodes = 1 << J;
    const double *ndc = w.nd[J & 1];
    double *ndn = w.nd[(J + 1) & 1];
    if (lane < nodes) {
        const double p = cur[lane * kk + k1 * k + k1];
        w.inv[lane] = fw_inv(p, thrA, fl);
        ndn[2 * lane] = ndc[lane];
        ndn[2 * lane + 1] = ndc[lane] * p;
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

// The 8 principal minors of a 3 x 3 node C with node minor d, out[X] for X
// within {0,1,2}: row 0 scaled by d first, so that the four minors holding
// element 0 come out scaled; the 2 x 2 minors directly; the whole by expansion
// along row 0. 19 FP64 operations, no division.
__device__ __forceinline__ void fw_cf3(const double (&C)[3][3], double d, double *out) {
    const double a0 = d * C[0][0], a1 = d * C[0][1], a2 = d * C[0][2];
    const double m12 = fma(C[1][1], C[2][2], -C[1][2] * C[2][1]);
    const double m02 = fma(C[1][0], C[2][2], -C[1][2] * C[2][0]);
    const double m01 = fma(C[1][0], C[2][1], -C[1][1] * C[2][0]);
    const double s01 = fma(a0, C[1][1], -a1 * C[1][0]);
    const double s02 = fma(a0, C[2][2], -a2 * C[2][0]);
    const double t = fma(a0, m12, fma(-a1, m02, a2 * m01));
    double2 *o = reinterpret_cast<double2 *>(out);
    o[0] = make_double2(d, a0);
    o[1] = make_double2(d * C[1][1], s01);
    o[2] = make_double2(d * C[2][2], s02);
    o[3] = make_double2(d * m12, t);
}

// All 2^K principal minors of a K x K node M in registers (node minor d) into
// out[0 .. 2^K): the last element's pivot gives the kept child (the Schur
// complement) at out + 2^(K-1), the leading block the dropped one at out.
template <int K>
__device__ __forceinline__ void fw_lane_tree(const double (&M)[K][K], double d, double *out, double thrA, int &fl) {
    if constexpr (K == 3) {
        fw_cf3(M, d, out);
    } else {
        constexpr int K1 = K - 1;
        const double p = M[K1][K1];
        const double iv = fw_inv(p, thrA, fl);
        double S[K1][K1];
#pragma unroll
        for (int r = 0; r < K1; ++r) {
            const double f = M[r][K1] * iv;
#pragma unroll
            for (int q = 0; q < K1; ++q) S[r][q] = fma(-f, M[K1][q], M[r][q]);
        }
        fw_lane_tree<K1>(S, d * p, out + (1 << K1), thrA, fl);
        double Lb[K1][K1];
#pragma unroll
        for (int r = 0; r < K1; ++r)
#pragma unroll
            for (int q = 0; q < K1; ++q) Lb[r][q] = M[r][q];
        fw_lane_tree<K1>(Lb, d, out, thrA, fl);
    }
}

// A lane's node of size K, read from shared memory (row-major), node minor d:
// its kept child is formed in registers; its dropped child, the leading block,
// is read again from shared memory, so that the two need not be live at once.
template <int K>
__device__ __forceinline__ void fw_lane_root(const double *P, double d, double *out, double thrA, int &fl) {
    constexpr int K1 = K - 1;
    const double p = P[K1 * K + K1];
    const double iv = fw_inv(p, thrA, fl);
    {
        double S[K1][K1];
#pragma unroll
        for (int r = 0; r < K1; ++r) {
            const double f = P[r * K + K1] * iv;
#pragma unroll
            for (int q = 0; q < K1; ++q) S[r][q] = fma(-f, P[K1 * K + q], P[r * K + q]);
        }
        fw_lane_tree<K1>(S, d * p, out + (1 << K1), thrA, fl);
    }
    double Lb[K1][K1];
#pragma unroll
    for (int r = 0; r < K1; ++r)
#pragma unroll
        for (int q = 0; q < K1; ++q) Lb[r][q] = P[r * K + q];
    fw_lane_tree<K1>(Lb, d, out, thrA, fl);
}

template <int T, int J>
__device__ __forceinline__ void fw_tail_levels(double *cur, double *nxt, double *out, FwWarpSmem &w, int lane,
                                               double thrA, int &fl) {
    if constexpr (J < kFwBfs) {
        fw_tail_level<T, J>(cur, nxt, w, lane, thrA, fl);
        fw_tail_levels<T, J + 1>(nxt, cur, out, w, lane, thrA, fl);
    } else {
        constexpr int L = T - kFwBfs;
        fw_lane_root<L>(cur + lane * L * L, w.nd[J & 1][lane], out + (lane << L), thrA, fl);
    }
}

// The tail of T elements whose root matrix is in w.bufE (node minor w.nd[0][0]).
template <int T>
__device__ __forceinline__ void fw_tail(double *out, FwWarpSmem &w, int lane, double thrA, int &fl) {
    fw_tail_levels<T, 0>(w.bufE, w.bufO, out, w, lane, thrA, fl);
}

// One matrix of order n (9..16), whole warp: its 2^n minors, each times pre,
// into out. Returns 1 when a pivot is below thrA or zero (the fused kernel
// redoes the matrix) or the input is not finite (the fused kernel then sets the
// status and NaN).
template <int T>
__device__ __forceinline__ int fw_matrix(const double *A, int n, double *out, double thr, double pre,
                                         const double *anorm, double *stack, FwWarpSmem &w, int lane) {
    const int D = n - T;
    int fl = 0, nonfin = 0;
    // ||A||max and the finiteness test on the bit patterns of |x| (integer
    // order is the order of non-negative doubles), off the FP64 pipe
    unsigned long long am = 0;
    for (int e = lane; e < n * n; e += 32) {
        const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(A[e])) & 0x7fffffffffffffffull;
        nonfin |= b >= 0x7ff0000000000000ull;
        am = b > am ? b : am;
    }
    nonfin = __any_sync(0xffffffffu, nonfin);
    if (nonfin) return 1;
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, am, o);
        am = y > am ? y : am;
    }
    double amax = __longlong_as_double(static_cast<long long>(am));
    if (anorm) amax = *anorm;
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
                const double iv = fw_inv(piv, thrA, fl);
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
        fw_tail<T>(out + (t << T), w, lane, thrA, fl);
        __syncwarp();
    }
    return __any_sync(0xffffffffu, fl);
}

// Every matrix; b is appended to redo_list (*redo_count entries, zeroed
// before) where the fused kernel must compute it again. pre
// (or NULL for 1): a factor per matrix on all its minors; anorm (or NULL): the
// scale of the threshold, anorm[b >> anorm_shift], in place of the matrix's own
// ||A||max (the leaves of a larger matrix take its norm). T = min(n, 12), one
// instantiation each, so that the register allocation of the largest lane
// subtree does not burden the others. Shared memory (90 KB per CTA) admits two
// CTAs per SM, so each thread may use up to 255 registers.
template <int T>
__global__ void __launch_bounds__(kFwWarps * 32, 2) fpm_warp_kernel(const double *__restrict__ A, int n,
                                                                  int64_t batch, double *minors, double thr,
                                                                  const double *__restrict__ pre,
                                                                  uint32_t *redo_list, unsigned *redo_count,
                                                                  uint32_t *status, double *stack_base,
                                                                  size_t stack_per_warp,
                                                                  const double *__restrict__ anorm,
                                                                  int anorm_shift) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    FwWarpSmem &w = reinterpret_cast<FwWarpSmem *>(smem_raw)[wid];
    const int64_t gw = static_cast<int64_t>(blockIdx.x) * kFwWarps + wid;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * kFwWarps;
    double *stack = stack_base ? stack_base + gw * stack_per_warp : nullptr;
    const int64_t nn = static_cast<int64_t>(n) * n, N = int64_t(1) << n;
    for (int64_t b = gw; b < batch; b += nw) {
        const int r = fw_matrix<T>(A + b * nn, n, minors + b * N, thr, pre ? pre[b] : 1.0,
                                   anorm ? anorm + (b >> anorm_shift) : nullptr, stack, w, lane);
        if (lane == 0) {
            if (r) redo_list[atomicAdd(redo_count, 1u)] = static_cast<uint32_t>(b);
            if (status && !r) status[b] = 0u;
        }
    }
}

// The minors of the connected-sum paths at orders 13..16 (fpm_cdet.cu reads
// them back unless a matrix is flagged): matrix b's minors go to
// out + b * 2^n, or, with an item list (order != NULL), the items
// order[*first + i], i < *count, of an uneven batch, matrix A + a_off[b] and
// minors out + o_off[b]. flag[b] = 1 where the fused kernel must compute the
// matrix itself (a pivot at or below the threshold, a non-finite entry), else 0
// with status[b] = 0. Orders above 12 only (tail of 12 elements).
__global__ void __launch_bounds__(kFwWarps * 32, 2) fpm_warp_route_kernel(
    const double *__restrict__ A, int n, int64_t batch, double *out, double thr, uint8_t *flag,
    uint32_t *status, double *stack_base, size_t stack_per_warp, const int *__restrict__ order,
    const int64_t *__restrict__ a_off, const int64_t *__restrict__ o_off, const unsigned *first,
    const unsigned *count) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    FwWarpSmem &w = reinterpret_cast<FwWarpSmem *>(smem_raw)[wid];
    const int64_t gw = static_cast<int64_t>(blockIdx.x) * kFwWarps + wid;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * kFwWarps;
    double *stack = stack_base ? stack_base + gw * stack_per_warp : nullptr;
    const int64_t nn = static_cast<int64_t>(n) * n, N = int64_t(1) << n;
    const int64_t items = order ? static_cast<int64_t>(*count) : batch;
    const int64_t i0 = order ? static_cast<int64_t>(*first) : 0;
    for (int64_t i = gw; i < items; i += nw) {
        const int64_t b = order ? order[i0 + i] : i;
        const double *Ab = order ? A + a_off[b] : A + b * nn;
        double *ob = order ? out + o_off[b] : out + b * N;
        const int r = fw_matrix<kFwTail>(Ab, n, ob, thr, 1.0, nullptr, stack, w, lane);
        if (lane == 0) {
            flag[b] = static_cast<uint8_t>(r);
            if (status && !r) status[b] = 0u;
        }
    }
}

using FwKernel = void (*)(const double *, int, int64_t, double *, double, const double *, uint32_t *, unsigned *,
                         uint32_t *, double *, size_t, const double *, int);
static FwKernel fw_kernel_for(int n) {
    switch (n < kFwTail ? n : kFwTail) {
        case 9: return fpm_warp_kernel<9>;
        case 10: return fpm_warp_kernel<10>;
        case 11: return fpm_warp_kernel<11>;
        default: return fpm_warp_kernel<12>;
    }
}

static int fpm_warp_grid(int n, int64_t batch, int *err) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = kFwWarps * sizeof(FwWarpSmem);
    const FwKernel kern = fw_kernel_for(n);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kFwWarps * 32, smem);
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

// Workspace: per resident warp the depth-first stack, the redo list (a
// counter, then up to one entry per matrix), and for n > 12 the fused kernel's
// global scratch (its redo launch).
struct FwPlan {
    size_t stack, list, fused, total;
};
static int fw_plan(int n, int64_t batch, FwPlan *p, int *grid) {
    int err = 0;
    *grid = fpm_warp_grid(n, batch, &err);
    if (err) return err;
    auto al = [](size_t x) { return (x + 255) & ~static_cast<size_t>(255); };
    p->stack = al(static_cast<size_t>(*grid) * kFwWarps * fw_stack_entries(n) * sizeof(double));
    p->list = 256 + al(static_cast<size_t>(batch) * sizeof(uint32_t));
    p->fused = 0;
    if (n > cdet_smem_max_n(false)) {
        const int g = cdet_grid(n, batch, false, false, &err);
        if (err) return err;
        p->fused = al(static_cast<size_t>(g) * cdet_slot_doubles(n) * sizeof(double));
    }
    p->total = p->stack + p->list + p->fused;
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
                    uint32_t *status, void *workspace, cudaStream_t s, const double *pre,
                    const double *anorm_in, int anorm_shift) {
    FwPlan plan;
    int grid = 0;
    int err = fw_plan(n, batch, &plan, &grid);
    if (err) return err;
    const size_t smem = kFwWarps * sizeof(FwWarpSmem);
    const size_t per = fw_stack_entries(n);
    char *ws = static_cast<char *>(workspace);
    double *stack = per ? reinterpret_cast<double *>(ws) : nullptr;
    unsigned *count = reinterpret_cast<unsigned *>(ws + plan.stack);
    uint32_t *list = reinterpret_cast<uint32_t *>(ws + plan.stack + 256);
    double *fused = plan.fused ? reinterpret_cast<double *>(ws + plan.stack + plan.list) : nullptr;
    err = static_cast<int>(cudaMemsetAsync(count, 0, sizeof(unsigned), s));
    if (err) return err;
    fw_kernel_for(n)<<<grid, kFwWarps * 32, smem, s>>>(A, n, batch, minors, thr, pre, list, count, status, stack,
                                                        per, anorm_in, anorm_shift);
    err = static_cast<int>(cudaGetLastError());
    if (err) return err;
    // the flagged matrices again, by the fused kernel with the pivot correction
    // (pre as the root minor of their trees too)
    CdetArgs a = {};
    a.A_up = A;
    a.minors_out = minors;
    a.status = status;
    a.batch = batch;
    a.n = n;
    a.mode = kModeMinors;
    a.piv_thr = thr;
    a.piv_shift = shf;
    a.redo_list = list;
    a.redo_count = count;
    a.gscratch = fused;
    a.anorm_in = anorm_in;
    a.anorm_shift = anorm_shift;
    a.pre = pre;
    return launch_fpm_cdet(a, s);
}

static int fw_route_grid(int64_t batch, int *err) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = kFwWarps * sizeof(FwWarpSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fpm_warp_route_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fpm_warp_route_kernel, kFwWarps * 32, smem);
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

size_t fpm_warp_route_stack_bytes(int n, int64_t batch, int *err) {
    *err = 0;
    if (batch == 0 || n <= kFwTail) return 0;
    const int grid = fw_route_grid(batch, err);
    if (*err) return 0;
    return static_cast<size_t>(grid) * kFwWarps * fw_stack_entries(n) * sizeof(double);
}

int launch_fpm_warp_route(const double *A, int n, int64_t batch, double *out, double thr, uint8_t *flag,
                          uint32_t *status, double *stack, const int *order, const int64_t *a_off,
                          const int64_t *o_off, const unsigned *first, const unsigned *count, cudaStream_t s) {
    if (n <= kFwTail || n > kFwMaxN) return static_cast<int>(cudaErrorInvalidValue);
    int err = 0;
    const int grid = fw_route_grid(batch, &err);
    if (err) return err;
    fpm_warp_route_kernel<<<grid, kFwWarps * 32, kFwWarps * sizeof(FwWarpSmem), s>>>(
        A, n, batch, out, thr, flag, status, stack, fw_stack_entries(n), order, a_off, o_off, first, count);
    return static_cast<int>(cudaGetLastError());
}

}  // namespace apm
