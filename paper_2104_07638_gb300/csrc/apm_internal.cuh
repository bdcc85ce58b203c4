// Internal declarations shared by the translation units of libapm.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/apm.h"

namespace apm {

// 1/d. Where d and 1/d are normal numbers (biased exponent of |d| in 3..2044):
// the hardware approximation x (rcp.approx.ftz.f64; its relative error
// e = 1 - d x measured at most 2^-19.9 over all 2^22 leading mantissa bits at
// several exponents) refined by one step of the cubic iteration
// x <- x (1 + e + e^2), the truncated geometric series of 1/(1 - e), which
// leaves the relative error e^3 < 2^-59 plus the rounding of the last FMA
// (three FMAs instead of the four of two Newton-Raphson steps).
// Elsewhere (zero, subnormal, huge, inf, NaN): the IEEE division.
__device__ __forceinline__ double rcp_nr(double d) {
    const unsigned ex = (static_cast<unsigned>(__double2hiint(d)) >> 20) & 0x7ffu;
    if (ex - 3u < 2042u) {
        double x;
        asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(x) : "d"(d));
        const double e = fma(-d, x, 1.0);
        return fma(x, fma(e, e, e), x);
    }
    return 1.0 / d;
}

// Asynchronous global -> shared copies of 8 or 16 bytes (cp.async): a thread
// issues all of its copies of a staging step back to back, without holding the
// values in registers, and waits once for all of them, so that one memory
// latency is exposed per step instead of one per unrolled group of loads.
// Both addresses must be aligned to the copy size. After cp_async_wait_all the
// data is visible to the issuing thread; a barrier makes it visible to the
// others.
__device__ __forceinline__ void cp_async8(double *dst, const double *src) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(double *dst, const double *src) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

// Threads per CTA of the minor / connected-sum kernels.
constexpr int kCdetThreads = 256;
// Capacity of the per-matrix pivot-correction log.
constexpr int kCorrCap = 256;

// Largest order whose a[] and c[] arrays stay in shared memory.
int cdet_smem_max_n(bool two_mats);

// Bytes of dynamic shared memory of the minor / connected-sum kernel.
size_t cdet_smem_bytes(int n, bool two_mats, bool smem_arrays);

// Grid size used for a fixed-order launch (also sizes the workspace).
int cdet_grid(int n, int64_t batch, bool two_mats, bool smem_arrays, int *err);

// Doubles of global scratch one CTA uses when the arrays do not fit on chip.
size_t cdet_slot_doubles(int n);

enum CdetMode : int { kModeMinors = 0, kModeCdet = 1, kModeWeights = 2 };

struct CdetArgs {
    const double *A_up;
    const double *A_dn;
    const double *a_in;
    double *minors_out;
    double *c_out;
    uint32_t *status;
    double *gscratch;
    int64_t batch;
    int n;
    int mode;
    int single_det;
    int two_mats;
    double piv_thr;
    double piv_shift;
    int fsc_from_n;  // orders >= this (0: none) leave the weights a[] in c for the fast subset convolution
    // fixed-order launch: if set, only the matrices redo_list[0 .. *redo_count - 1]
    // (in any order: each is computed on its own)
    const uint32_t *redo_list;
    const unsigned *redo_count;
    // fixed-order minors launch (kModeMinors, one matrix): if set, matrix b's
    // tree starts from the root minor pre[b] instead of 1, so that all its
    // minors come out times pre[b]
    const double *pre;
    // fixed-order launch: if set, matrix b scales its pivot threshold and shift
    // by anorm_in[b >> anorm_shift] instead of its own ||A||max (the leaves of
    // a larger matrix take that matrix's norm)
    const double *anorm_in;
    int anorm_shift;
    // connected sums of one matrix per item at orders >= warp_from_n (0: none):
    // the warp-per-matrix minors kernel ran first and left each item's minors
    // in its minors_out row (its c row when minors_out is NULL); the fused
    // kernel reads them back and only computes the tree itself where
    // wflag[b] != 0 (b: the item's batch index)
    uint8_t *wflag;
    int warp_from_n;
};

// Orders whose connected sums apm_cdet_connected and its uneven-batch form take
// through the fast subset convolution by default (faster than the recursion
// from here on, as measured); apm_tune_options_set moves the hand-off within
// kFscMinFrom .. 17 (17: never).
constexpr int kFscFromN = 16;
constexpr int kFscMinFrom = 13;
int cdet_fsc_from_n();
// tuned knobs of the uneven-batch launches (0: the default)
int cdet_varlen_ctas_per_sm();
int keldysh_varlen_warps();
void keldysh_varlen_warps_set(int w);
void cdet_tune_options_set(int fsc_from_n, int cdet_ctas_per_sm);

// Launches the fused minors / connected-sum kernel. Returns a cudaError_t.
int launch_fpm_cdet(const CdetArgs &a, cudaStream_t s);

// All principal minors for orders 9..16 (minors only), one warp per matrix;
// matrices with a small pivot are redone by the fused kernel (fpm_warp.cu).
constexpr int kWarpMinorsFromN = 9;
size_t fpm_warp_workspace_bytes(int n, int64_t batch, int *err);
// pre (or NULL): a factor per matrix on all its minors (the root minor of its
// tree, in the redone matrices too). anorm_in (or NULL): per matrix b the scale
// anorm_in[b >> anorm_shift] of the pivot threshold and shift instead of the
// matrix's own ||A||max.
int launch_fpm_warp(const double *A, int n, int64_t batch, double *minors, double thr, double shf,
                    uint32_t *status, void *workspace, cudaStream_t s, const double *pre = nullptr,
                    const double *anorm_in = nullptr, int anorm_shift = 0);

// The minors of the connected-sum paths at orders 13..16, one warp per matrix:
// fixed order (order == NULL: matrix b at A + b n^2, minors at out + b 2^n) or
// the items order[*first + i], i < *count, of an uneven batch (A + a_off[b],
// out + o_off[b]); flag[b] = 1 where the fused kernel must compute the tree
// itself. The stack is caller scratch of fpm_warp_route_stack_bytes(n_max, batch).
constexpr int kWarpRouteFromN = 13;
size_t fpm_warp_route_stack_bytes(int n, int64_t batch, int *err);
int launch_fpm_warp_route(const double *A, int n, int64_t batch, double *out, double thr, uint8_t *flag,
                          uint32_t *status, double *stack, const int *order, const int64_t *a_off,
                          const int64_t *o_off, const unsigned *first, const unsigned *count, cudaStream_t s);

// All principal minors for orders 17..24: the upper levels of the tree breadth
// first, the 12 x 12 leaves by the fused kernel (fpm_big.cu).
size_t fpm_big_workspace_bytes(int n, int64_t batch, int *err);
int launch_fpm_big(const double *A, int n, int64_t batch, double *minors, double thr, double shf,
                   uint32_t *status, void *workspace, cudaStream_t s);

// Uploads the popcount-ordered mask table on the current device (idempotent).
int ensure_tables();

// Per-layer lane-group sizes (log2) chosen by the cost model for order n.
void cdet_group_table(int n, int threads, uint8_t *gsel /*[17]*/);

// Fixed-order Keldysh launch layout: grid, chunks per matrix (log2) and the
// workspace parts (depth-first stacks, chunk slots, chunk flags, counters).
struct KeldyshPlan {
    int grid;
    int kc;
    size_t stack_bytes, slot_bytes, flag_bytes, ctr_bytes, total;
};
int keldysh_plan(int n, int64_t batch, KeldyshPlan *p);
int launch_keldysh(const double *Mt, int n, int64_t batch, int sgn, double *sum, double *partial,
                   uint32_t *status, void *workspace, cudaStream_t s);
int keldysh_grid(int64_t batch, int *err);
int keldysh_warps_per_block();
size_t keldysh_stack_entries(int n);

int launch_ppm(const double *A, int n, int64_t batch, double *perms, cudaStream_t s);

// XNOR minors of 2n x 2n block matrices (one warp per matrix).
int xnor_grid(int64_t batch, int *err);
size_t xnor_workspace_bytes(int n, int64_t batch, int *err);
int launch_xnor(const double *M, int n, int64_t batch, double *minors, uint32_t *status, void *workspace,
                cudaStream_t s);

// Two-spin Keldysh sums (one warp per matrix pair).
int keldysh2_grid(int64_t batch, int *err);
size_t keldysh2_workspace_bytes(int n, int64_t batch, int *err);
int launch_keldysh2(const double *Mu, const double *Md, int n, int64_t batch, int sgn, double *sum,
                    double *partial, uint32_t *status, void *workspace, cudaStream_t s);

// NAND minors (type_sums = false: all 3^n per matrix) or their sums over the
// two vertex types (type_sums = true: 2^n per matrix); one warp per matrix.
int nand_grid(int64_t batch, int *err);
size_t nand_workspace_bytes(int n, int64_t batch, int *err);
int launch_nand(const double *M, int n, int64_t batch, double *out, bool type_sums, double thr, double shf,
                uint32_t *status, void *workspace, cudaStream_t s);

// connected sums by the fast subset convolution (from weights)
int fsc_grid(int n, int64_t batch, int *err);
size_t fsc_workspace_bytes(int n, int64_t batch, int *err);
int launch_fsc(const double *a, int n, int64_t batch, double *c, void *workspace, cudaStream_t s);
// in place on the rows c + c_off[order[*first + i]] (2^n doubles: weights in,
// connected sums out) for i < *count (device values, count at most max_items)
int launch_fsc_items(double *c, const int64_t *c_off, const int *order, const unsigned *first,
                     const unsigned *count, int64_t max_items, int n, void *workspace, cudaStream_t s);

// uneven batches
unsigned long long cdet_gsel_packed(int n);
void cdet_tune_set(const unsigned long long *table);
size_t cdet_varlen_workspace(int n_max, int64_t batch, bool two_mats, int *err);
int launch_cdet_varlen(const CdetArgs &a, const int64_t *a_off, const int *n_arr, const int64_t *c_off,
                       int n_max, void *workspace, cudaStream_t s);
// Counting sort by decreasing order into `order`; ctr[0] = 0 (work counter),
// ctr[1] = the items of orders >= fsc_from_n, and for each order m the first
// index and the count of its items at ctr[2 + 2m], ctr[3 + 2m].
int launch_order(const int *n_arr, int64_t batch, int n_max, int *order, unsigned *ctr, cudaStream_t s,
                 int fsc_from_n = kFscFromN);
int launch_keldysh_varlen(const double *Mt, const int64_t *m_off, const int *n_arr, int64_t batch, int n_max,
                          int sgn, double *sum, double *partial, uint32_t *status, void *stack,
                          const int *order, unsigned *ctr, cudaStream_t s);

// surrogate network
constexpr int kMlpIn = 64, kMlpH = 256;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpH * kMlpIn;
constexpr int kOffW2 = kOffB1 + kMlpH;
constexpr int kOffB2 = kOffW2 + kMlpH * kMlpH;
constexpr int kOffW3 = kOffB2 + kMlpH;
constexpr int kOffB3 = kOffW3 + kMlpH * kMlpH;
constexpr int kOffW4 = kOffB3 + kMlpH;
constexpr int kOffB4 = kOffW4 + kMlpH;
constexpr int kMlpParams = kOffB4 + 8;
static_assert(kMlpParams == APM_MLP_PARAMS, "parameter count");
}  // namespace apm
#include <cuda_bf16.h>
namespace apm {
struct MlpParams {
    float *param, *grad, *m, *v;
    __nv_bfloat16 *pb;
    const __nv_bfloat16 *w1b, *w2b, *w3b, *w4b;
    const float *b1, *b2, *b3, *b4;
};
struct MlpWork {
    uint32_t *err;  // bit 0: a bounded wait of the tensor-core GEMM gave up
    float *part;    // split-K partial tiles
    __nv_bfloat16 *h1, *h2, *h3, *dzb, *t1, *t2, *wt;
    float *y, *dy, *dz32, *dh32;
    float *pcol, *pcol2, *pvec, *pvec2;  // per-block partial column sums of the backward pass
};
// C = A * Bt^T (+ bias) (ReLU) on the tensor cores; part (part_floats) holds
// split-K partials when K is long next to M x N
size_t tc_gemm_split_floats();
int launch_tc_gemm_tn(const __nv_bfloat16 *A, const __nv_bfloat16 *Bt, const float *bias, float *C32,
                      __nv_bfloat16 *Cb, int M, int N, int K, int relu, float *part, size_t part_floats,
                      uint32_t *err, cudaStream_t s);
size_t mlp_workspace_bytes(int Bp);
void mlp_bind(const apm_mlp *net, MlpParams &P);
void mlp_work(void *ws, int Bp, MlpWork &w);
int mlp_forward(const MlpParams &P, const __nv_bfloat16 *X, int Bp, float *y, MlpWork &w, cudaStream_t s);
int mlp_train_step(MlpParams &P, const __nv_bfloat16 *X, const float *target, int Bp, int B_valid, MlpWork &w,
                   float lr, int step, float *loss_acc, cudaStream_t s);
int mlp_refresh_bf16(MlpParams &P, cudaStream_t s);
int mlp_gradient(MlpParams &P, const __nv_bfloat16 *X, const float *target, int Bp, int B_valid, MlpWork &w,
                 float *loss_acc, cudaStream_t s);
int mlp_adam(MlpParams &P, float lr, int step, cudaStream_t s);

int launch_fp64_probe(double *sink, int blocks, int threads, int iters, cudaStream_t s);

}  // namespace apm
