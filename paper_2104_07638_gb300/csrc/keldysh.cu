// Real-time Keldysh sum as the sum of XOR principal minors (complex128).
//
// Paper: Section III.D (XOR minors: of each pair (2l+1, 2l+2) exactly one row
// and column is kept; only the two Schur-complement branches of the ternary
// tree remain, a binary tree with O(2^n) nodes, no pivot correction possible)
// and Section V.D (the sum over all 2^n Keldysh index assignments equals the
// sum of those minors of the 2n x 2n block matrix; the per-depth sums are the
// lower orders obtained on the way).
//
// Tree: the node at depth d fixes the indices alpha_0..alpha_{d-1}; it holds
// the Schur complement of the block matrix with respect to the kept rows and
// columns {(i, alpha_i), i < d}, restricted to the rows/columns of vertices
// d..n-1 (size 2(n-d)). Child alpha: pivot p = entry (d,alpha),(d,alpha); the
// partner row/column (d, 1-alpha) is dropped and the rest is Schur-complemented
// with respect to p; det(child) = det(node) * p (times -1 for alpha = - when
// the assignments are sign-weighted).
//
// Mapping: one warp per matrix. The upper vertices 0..D-1 (D = n - S, S = 7)
// are walked depth first; each Schur step is spread over the 32 lanes and its
// result goes to a per-warp stack in caller scratch (global memory, L1/L2
// resident). Of the last min(n,S) vertices, all but three are expanded breadth
// first in shared memory (one child entry per lane step); the 6x6 nodes that
// remain are summed in closed form: the sum over the 8 assignments of the last
// three vertices is a sum of 3x3 determinants, four lanes per node, two
// determinants per lane, with no pivots. The running sums stay in per-lane
// registers for the whole matrix and are reduced over the warp once at its end.
//
// Cost model: an FP64 warp instruction occupies the SM sub-partition's FP64
// unit for the same time whatever the number of active lanes, so the design
// counts warp instructions: the closed form replaces two tree levels (with
// their reciprocals, issued on 16 and fewer lanes) and the leaf level, and a
// tail of 7 rather than 6 vertices halves the depth-first steps per leaf and
// doubles the nodes that share each breadth-first level's reciprocal step
// (measured 0.87 against 0.68 TFLOP/s at n = 12).
#include <cuda_runtime.h>
#include <stdint.h>

#include "apm_internal.cuh"
#include "complex_ops.cuh"

// x is infinite or NaN: the exponent bits all set, tested on the high word in
// integer arithmetic (no FP64 compare)
__device__ __forceinline__ bool nonfinite_bits(double x) {
    return (static_cast<unsigned>(__double2hiint(x)) & 0x7ff00000u) == 0x7ff00000u;
}
namespace apm {

// Tail size S (vertices expanded breadth first in shared memory) and warps per
// CTA; S = 7 needs 17.3 KB of shared memory per warp, so its CTA holds the 12
// warps that fit on one SM (13 would fit the shared memory but not the
// registers, 168 per thread).
#ifndef APM_KEL_TAIL
#define APM_KEL_TAIL 7
#endif
constexpr int kKelTail = APM_KEL_TAIL;
static_assert(kKelTail == 6 || kKelTail == 7, "tail of 6 or 7 vertices");
constexpr int kKelWarps = kKelTail == 6 ? 4 : 12;
// Tail nodes are stored without the off-diagonal entries of the 2 x 2 blocks:
// an XOR minor keeps one row and column of a block, and a Schur update of
// entry (r, q) reads only (r, q), (r, p), (p, q) and (p, p) with the pivot p in
// another block, so entries (2i, 2i+1) and (2i+1, 2i) are never read. Row r of
// a node of size m holds its m - 1 columns q != r ^ 1 in order (compact column
// c <-> q = c + (c >= (r ^ 1))); entry (r+2, q+2) of a node has the compact
// column of (r, q) in its child, plus 2.
// Tail of S vertices: the root (2S x 2S) and the outputs of the odd levels sit
// in bufE, the outputs of the even levels in bufO; level J (J = 0..S-4) makes
// 2^(J+1) nodes of size m = 2(S-J-1), m(m-1) entries each. S = 6: bufE 132,
// 224; bufO 180, 240. S = 7: bufE 182, 360, 480; bufO 264, 448.
__host__ __device__ constexpr int kel_level_entries(int S, int J) {
    return (2 << J) * (2 * (S - J - 1)) * (2 * (S - J - 1) - 1);
}
__host__ __device__ constexpr int kel_buf_entries(int S, int first) {
    int b = first == 1 ? 2 * S * (2 * S - 1) : 0;
    for (int J = first; J <= S - 4; J += 2) b = b > kel_level_entries(S, J) ? b : kel_level_entries(S, J);
    return b;
}
// row factors: nchild * (m - 2) at level J, and up to 30 for a depth-first step
__host__ __device__ constexpr int kel_fac_entries(int S) {
    int b = 32;
    for (int J = 0; J <= S - 4; ++J) {
        const int f = (2 << J) * (2 * (S - J) - 2);
        b = b > f ? b : f;
    }
    return b;
}
constexpr int kKelBufE = kel_buf_entries(kKelTail, 1);
constexpr int kKelBufO = kel_buf_entries(kKelTail, 0);
constexpr int kKelFac = kel_fac_entries(kKelTail);
static_assert(kKelTail != 6 || (kKelBufE == 224 && kKelBufO == 240 && kKelFac == 48), "6-vertex tail");
static_assert(kKelTail != 7 || (kKelBufE == 480 && kKelBufO == 448 && kKelFac == 96), "7-vertex tail");

struct KelWarpSmem {
    double2 bufE[kKelBufE];
    double2 bufO[kKelBufO];
    double2 fac[kKelFac];
    double2 inv[16];
    double2 ndet[2][16];
    double2 part[17];
    double2 pdet[17];
    int bad;
    int flags;
};
// CTAs per SM that the shared memory allows (228 KB per SM, 1 KB reserved per CTA)
constexpr int kKelMinBlocks = static_cast<int>((228 * 1024) / (kKelWarps * sizeof(KelWarpSmem) + 1024));
static_assert(kKelMinBlocks >= 1, "tail buffers exceed shared memory");


// double2 entries of the per-warp stack for order n: depths 1..D-1
__host__ __device__ constexpr size_t kel_stack_entries(int n) {
    const int D = n > kKelTail ? n - kKelTail : 0;
    size_t t = 0;
    for (int d = 1; d < D; ++d) t += static_cast<size_t>(2 * (n - d)) * (2 * (n - d));
    return t;
}

// One Schur step of the depth-first part: src (m x m, dense) -> dst ((m-2) x
// (m-2)): the entries a minor can read, dense on the stack (the blocks'
// off-diagonal entries left unwritten) or compact in the tail root.
__device__ __forceinline__ void kel_schur(const double2 *src, int m, int alpha, double2 *dst, bool root,
                                          KelWarpSmem &w, int lane, double2 &piv, int &bad) {
    piv = src[alpha * m + alpha];
    const double2 iv = crcp(piv, bad);
    const int m2 = m - 2;
    for (int r = lane; r < m2; r += 32) w.fac[r] = cmul(src[(r + 2) * m + alpha], iv);
    __syncwarp();
    for (int e = lane; e < m2 * (m2 - 1); e += 32) {
        const int r = e / (m2 - 1), c = e - r * (m2 - 1), q = c + (c >= (r ^ 1));
        dst[root ? e : r * m2 + q] = cfms(w.fac[r], src[alpha * m + q + 2], src[(r + 2) * m + q + 2]);
    }
    __syncwarp();
}

// Per-lane running sums of one matrix, indexed by r = n - depth: r = 0 is the
// full sum, r >= 1 the lower-order partial sums found in the tail. Reduced over
// the warp once per matrix.
struct KelAcc {
    double2 v[kKelTail];
};

// One breadth-first level J of a tail over S vertices: the 2^J nodes of size
// m = 2(S-J) in cur give 2^(J+1) children of size m-2 in nxt (compact layout:
// the pivot (alpha, alpha) is compact column 0 of row alpha, entry (r+2, alpha)
// column alpha of row r+2, entry (alpha, q+2) column q+1 of row alpha).
template <int S, int J>
__device__ __forceinline__ void kel_tail_level(const double2 *cur, double2 *nxt, bool want_part, bool sgn,
                                               KelWarpSmem &w, int lane, int &bad, KelAcc &acc) {
    constexpr int m = 2 * (S - J), m2 = m - 2, rl = m - 1, rl2 = m2 - 1, mm = m * rl, mm2 = m2 * rl2;
    constexpr int nchild = 2 << J;
    if (lane < nchild) {
        const int alpha = lane & 1;
        const double2 *P = cur + (lane >> 1) * mm;
        const double2 piv = P[alpha * rl];
        w.inv[lane] = crcp(piv, bad);
        const double2 nd = cneg_if(cmul(w.ndet[J & 1][lane >> 1], piv), sgn && alpha);
        w.ndet[(J + 1) & 1][lane] = nd;
        if (want_part) acc.v[S - 1 - J] = cadd(acc.v[S - 1 - J], nd);
    }
    __syncwarp();
    for (int idx = lane; idx < nchild * m2; idx += 32) {
        const int c = idx / m2, r = idx - c * m2, alpha = c & 1;
        const double2 *P = cur + (c >> 1) * mm;
        w.fac[idx] = cmul(P[(r + 2) * rl + alpha], w.inv[c]);
    }
    __syncwarp();
    for (int e = lane; e < nchild * mm2; e += 32) {
        const int c = e / mm2, rem = e - c * mm2, r = rem / rl2, cc = rem - r * rl2, alpha = c & 1;
        const int q = cc + (cc >= (r ^ 1));
        const double2 *P = cur + (c >> 1) * mm;
        nxt[e] = cfms(w.fac[c * m2 + r], P[alpha * rl + q + 1], P[(r + 2) * rl + cc + 2]);
    }
    __syncwarp();
}

// Closed form for the last three vertices of NODES nodes (6 x 6 each, compact
// rows of 5, node determinants nd[]): four lanes per node, lane (a0, a1) forms
// the two 3 x 3 XOR minors with rows/columns (0,a0), (1,a1), (2,a2), a2 = 0, 1,
// by expansion along the last row; the leading 2 x 2 cofactor and the leading
// entry are the node's contributions to the two orders below. No pivots, no
// divisions. Entry (i, j) of another block than i's is at compact column
// j - (j > i), the diagonal entry (i, i) at column i & ~1.
template <int NODES>
__device__ __forceinline__ void kel_closed3(const double2 *cur, const double2 *nd, bool want_part, bool sgn,
                                            int lane, KelAcc &acc) {
    for (int idx = lane; idx < 4 * NODES; idx += 32) {
        const int k = idx >> 2, a0 = idx & 1, a1 = (idx >> 1) & 1;
        const double2 *M = cur + k * 30;
        const int r0 = a0, r1 = 2 + a1;
        const double2 A = M[r0 * 5], B = M[r0 * 5 + r1 - 1];
        const double2 Dv = M[r1 * 5 + r0], E = M[r1 * 5 + 2];
        const double2 C2 = cfms(B, Dv, cmul(A, E));  // A E - B D
        double2 tot = make_double2(0.0, 0.0);
#pragma unroll
        for (int a2 = 0; a2 < 2; ++a2) {
            const int r2 = 4 + a2;
            const double2 C = M[r0 * 5 + r2 - 1], F = M[r1 * 5 + r2 - 1];
            const double2 G = M[r2 * 5 + r0], H = M[r2 * 5 + r1], Iv = M[r2 * 5 + 4];
            const double2 u = cfms(C, E, cmul(B, F));   // B F - C E
            const double2 v = cfms(C, Dv, cmul(A, F));  // A F - C D
            const double2 det = cfma(Iv, C2, cfms(H, v, cmul(G, u)));
            tot = a2 == 0 ? det : (sgn ? csub(tot, det) : cadd(tot, det));
        }
        const double2 dk = cneg_if(nd[k], sgn && (a0 ^ a1));
        acc.v[0] = cfma(dk, tot, acc.v[0]);
        if (want_part) {
            acc.v[1] = cfma(dk, C2, acc.v[1]);
            if (a1 == 0) acc.v[2] = cfma(dk, A, acc.v[2]);
        }
    }
}

// Orders 1 and 2 (one node, the whole matrix; compact rows of 3 and 1).
__device__ __forceinline__ void kel_closed2(const double2 *M, double2 det0, bool want_part, bool sgn, int lane,
                                            KelAcc &acc) {
    if (lane < 4) {
        const int a0 = lane & 1, a1 = lane >> 1;
        const double2 A = M[a0 * 3], B = M[a0 * 3 + 1 + a1];
        const double2 Dv = M[(2 + a1) * 3 + a0], E = M[(2 + a1) * 3 + 2];
        const double2 dk = cneg_if(det0, sgn && (a0 ^ a1));
        acc.v[0] = cfma(dk, cfms(B, Dv, cmul(A, E)), acc.v[0]);
        if (want_part && a1 == 0) acc.v[1] = cfma(dk, A, acc.v[1]);
    }
}
__device__ __forceinline__ void kel_closed1(const double2 *M, double2 det0, bool sgn, int lane, KelAcc &acc) {
    if (lane == 0) acc.v[0] = cfma(det0, sgn ? csub(M[0], M[1]) : cadd(M[0], M[1]), acc.v[0]);
}

template <int S, int J>
__device__ __forceinline__ void kel_tail_levels(double2 *cur, double2 *nxt, double2 det0, bool want_part,
                                                bool sgn, KelWarpSmem &w, int lane, int &bad, KelAcc &acc) {
    if constexpr (S <= 2) {
        if constexpr (S == 2) kel_closed2(cur, det0, want_part, sgn, lane, acc);
        else kel_closed1(cur, det0, sgn, lane, acc);
    } else if constexpr (J < S - 3) {
        kel_tail_level<S, J>(cur, nxt, want_part, sgn, w, lane, bad, acc);
        kel_tail_levels<S, J + 1>(nxt, cur, det0, want_part, sgn, w, lane, bad, acc);
    } else {
        kel_closed3<(1 << J)>(cur, w.ndet[J & 1], want_part, sgn, lane, acc);
    }
}

// Breadth-first tail over the last S vertices; the root (2S x 2S) is in bufE
// with determinant det0. Adds its leaf sum and (if want_part) the node sums of
// the S lowest depths into the lane accumulators.
template <int S>
__device__ __forceinline__ void kel_tail(double2 det0, bool want_part, bool sgn, KelWarpSmem &w, int lane,
                                         int &bad, KelAcc &acc) {
    if (lane == 0) w.ndet[0][0] = det0;
    __syncwarp();
    kel_tail_levels<S, 0>(w.bufE, w.bufO, det0, want_part, sgn, w, lane, bad, acc);
    __syncwarp();
}

// Whole matrix of order n <= S as one tail (root determinant 1).
template <int S>
__device__ __forceinline__ void kel_tail_order(int n, bool want_part, bool sgn, KelWarpSmem &w, int lane,
                                               int &bad, KelAcc &acc) {
    if constexpr (S >= 1) {
        if (n == S) kel_tail<S>(make_double2(1.0, 0.0), want_part, sgn, w, lane, bad, acc);
        else kel_tail_order<S - 1>(n, want_part, sgn, w, lane, bad, acc);
    }
}

// Depth-first leaves t0 <= t < t1 of one matrix of order n (whole warp; all
// 2^(n-S) leaves, or one chunk of them). Leaves the sums in w.part[0..n]
// (part[0] = 1) and sets bad / nonfin. A node's determinant is added to the
// partial sum of its depth at the node's first leaf only, so chunks of one
// matrix never count a node twice.
__device__ __forceinline__ void kel_matrix(const double2 *A, int n, bool sgn, bool want_part, int64_t t0,
                                           int64_t t1, double2 *stack, KelWarpSmem &w, int lane, int &bad,
                                           int &nonfin) {
    const int s = n < kKelTail ? n : kKelTail;
    const int D = n - s;
    const int m0 = 2 * n;
    bad = 0;
    nonfin = 0;
    for (int e = lane; e < m0 * m0; e += 32) {
        const double2 v = A[e];
        nonfin |= nonfinite_bits(v.x) | nonfinite_bits(v.y);
    }
    nonfin = __any_sync(0xffffffffu, nonfin);
    KelAcc acc;
#pragma unroll
    for (int r = 0; r < kKelTail; ++r) acc.v[r] = make_double2(0.0, 0.0);
    if (lane <= n) w.part[lane] = make_double2(lane == 0 ? 1.0 : 0.0, 0.0);
    if (lane == 0) w.pdet[0] = make_double2(1.0, 0.0);
    __syncwarp();
    if (D == 0) {
        for (int e = lane; e < m0 * (m0 - 1); e += 32) {  // compact tail root
            const int r = e / (m0 - 1), c = e - r * (m0 - 1);
            w.bufE[e] = A[r * m0 + c + (c >= (r ^ 1))];
        }
        __syncwarp();
        kel_tail_order<kKelTail>(n, want_part, sgn, w, lane, bad, acc);
    } else {
        for (int64_t t = t0; t < t1; ++t) {
            // first depth whose index changed from t-1 to t (vertex 0 <-> top
            // bit); the first leaf of a chunk builds its whole path
            const int d0 = t == t0 ? 0 : D - __ffsll(t);
            size_t off = 0;  // stack offset of depth d0 (depths 1..D-1 are stacked)
            for (int d = 1; d < d0; ++d) off += static_cast<size_t>(2 * (n - d)) * (2 * (n - d));
            for (int d = d0; d < D; ++d) {
                const int alpha = static_cast<int>((t >> (D - 1 - d)) & 1);
                const int m = 2 * (n - d);
                const double2 *src = d == 0 ? A : stack + off;
                if (d > 0) off += static_cast<size_t>(m) * m;
                double2 *dst = (d + 1 == D) ? w.bufE : stack + off;
                double2 piv;
                kel_schur(src, m, alpha, dst, d + 1 == D, w, lane, piv, bad);
                if (lane == 0) {
                    const double2 pd = cneg_if(cmul(w.pdet[d], piv), sgn && alpha);
                    w.pdet[d + 1] = pd;
                    const bool first_leaf = (t & ((int64_t(1) << (D - 1 - d)) - 1)) == 0;
                    if (want_part && first_leaf) w.part[d + 1] = cadd(w.part[d + 1], pd);
                }
                __syncwarp();
            }
            kel_tail<kKelTail>(w.pdet[D], want_part, sgn, w, lane, bad, acc);
        }
    }
#pragma unroll
    for (int r = 0; r < kKelTail; ++r) {
        if (r == 0 || want_part) {
            const double2 v = warp_csum(acc.v[r]);
            if (lane == 0 && n - r >= 1) w.part[n - r] = cadd(w.part[n - r], v);
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    __syncwarp();
}

// Final results of one matrix from w.part: sum[2], partial[(n+1)*2] (if not
// NULL) and the status word; NaN where a pivot failed or the input is not finite.
__device__ __forceinline__ void kel_store(int n, int bad, int nonfin, double *sum_out, double *partial_out,
                                          uint32_t *status_out, const KelWarpSmem &w, int lane) {
    const double nanv = __longlong_as_double(0x7ff8000000000000ll);
    if (lane == 0) {
        const double2 r = (bad || nonfin) ? make_double2(nanv, nanv) : w.part[n];
        sum_out[0] = r.x;
        sum_out[1] = r.y;
        if (status_out) *status_out = (bad ? APM_ST_ZERO_PIVOT : 0u) | (nonfin ? APM_ST_NONFINITE_INPUT : 0u);
    }
    if (partial_out && lane <= n) {
        const double2 r = (bad || nonfin) ? make_double2(nanv, nanv) : w.part[lane];
        partial_out[2 * lane] = r.x;
        partial_out[2 * lane + 1] = r.y;
    }
    __syncwarp();
}

// Fixed order n. Work items are (matrix, chunk) pairs: 2^kc chunks of 2^(D-kc)
// consecutive depth-first leaves per matrix (kc = 0: whole matrices). With
// kc > 0 every chunk writes its sums and flags to a slot and counts itself in
// ctr[b]; the warp that completes the count adds the slots in chunk order
// (fixed, so the result does not depend on which warp finishes last) and
// stores the matrix's results. ctr must be zero at launch.
__global__ void __launch_bounds__(kKelWarps * 32, kKelMinBlocks) keldysh_kernel(
    const double2 *__restrict__ Mt, int n, int64_t batch, int sgn_flag, double *sum, double *partial,
    uint32_t *status, double2 *stack_base, size_t stack_per_warp, int kc, double2 *slots,
    uint32_t *slot_flags, unsigned *ctr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    KelWarpSmem &w = reinterpret_cast<KelWarpSmem *>(smem_raw)[wid];
    const int64_t gw = static_cast<int64_t>(blockIdx.x) * kKelWarps + wid;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * kKelWarps;
    double2 *stack = stack_base ? stack_base + gw * stack_per_warp : nullptr;
    const int64_t m0 = 2 * n;
    const int D = n > kKelTail ? n - kKelTail : 0;
    const int64_t nchunk = int64_t(1) << kc, leaves = int64_t(1) << (D - kc);
    const bool want_part = partial != nullptr;
    for (int64_t it = gw; it < (batch << kc); it += nw) {
        const int64_t b = it >> kc, c = it & (nchunk - 1);
        int bad, nonfin;
        kel_matrix(Mt + b * m0 * m0, n, sgn_flag != 0, want_part, c * leaves, (c + 1) * leaves, stack, w, lane,
                   bad, nonfin);
        double *sum_b = sum + 2 * b;
        double *part_b = want_part ? partial + b * (n + 1) * 2 : nullptr;
        uint32_t *st_b = status ? status + b : nullptr;
        if (kc == 0) {
            kel_store(n, bad, nonfin, sum_b, part_b, st_b, w, lane);
            continue;
        }
        double2 *slot = slots + it * (n + 1);
        if (lane <= n) slot[lane] = w.part[lane];
        if (lane == 0) slot_flags[it] = (bad ? 1u : 0u) | (nonfin ? 2u : 0u);
        __threadfence();
        __syncwarp();
        unsigned prev = 0;
        if (lane == 0) prev = atomicAdd(ctr + b, 1u);
        prev = __shfl_sync(0xffffffffu, prev, 0);
        if (prev != static_cast<unsigned>(nchunk - 1)) continue;
        __threadfence();
        double2 v = make_double2(0.0, 0.0);
        uint32_t fl = 0;
        const double2 *slot_b = slots + (b << kc) * (n + 1);
        for (int64_t cc = 0; cc < nchunk; ++cc) {
            if (lane <= n) v = cadd(v, __ldcg(slot_b + cc * (n + 1) + lane));
            fl |= __ldcg(slot_flags + (b << kc) + cc);
        }
        if (lane <= n) w.part[lane] = lane == 0 ? make_double2(1.0, 0.0) : v;
        __syncwarp();
        kel_store(n, (fl & 1u) ? 1 : 0, (fl & 2u) ? 1 : 0, sum_b, part_b, st_b, w, lane);
    }
}

// Uneven batch: warps take matrices longest-first from `order` through a
// global counter. partial rows have 17 complex entries per matrix. The CTA has
// blockDim.x / 32 warps (at most kKelWarps: a tuned launch may take fewer, and
// then more CTAs fit on an SM).
__global__ void __launch_bounds__(kKelWarps * 32, kKelMinBlocks) keldysh_varlen_kernel(
    const double2 *__restrict__ Mt, const int64_t *__restrict__ m_off, const int *__restrict__ n_arr,
    int64_t batch, int n_max, int sgn_flag, double *sum, double *partial, uint32_t *status,
    double2 *stack_base, size_t stack_per_warp, const int *__restrict__ order, unsigned *ctr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    KelWarpSmem &w = reinterpret_cast<KelWarpSmem *>(smem_raw)[wid];
    const int64_t gw = static_cast<int64_t>(blockIdx.x) * (blockDim.x >> 5) + wid;
    double2 *stack = stack_base ? stack_base + gw * stack_per_warp : nullptr;
    while (true) {
        int item = 0;
        if (lane == 0) item = static_cast<int>(atomicAdd(ctr, 1u));
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= batch) break;
        const int b = order[item];
        const int n = n_arr[b];
        if (n < 1 || n > n_max) {
            if (lane == 0 && status) status[b] = APM_ST_BAD_ORDER;
            continue;
        }
        const int D = n > kKelTail ? n - kKelTail : 0;
        int bad, nonfin;
        kel_matrix(Mt + m_off[b], n, sgn_flag != 0, partial != nullptr, 0, int64_t(1) << D, stack, w, lane, bad,
                   nonfin);
        kel_store(n, bad, nonfin, sum + 2 * static_cast<int64_t>(b),
                  partial ? partial + static_cast<int64_t>(b) * 17 * 2 : nullptr, status ? status + b : nullptr, w,
                  lane);
    }
}

// Warps per CTA of the uneven-batch launch (apm_tune_options_set; 0: kKelWarps).
static int g_kel_varlen_warps = 0;
int keldysh_varlen_warps() { return g_kel_varlen_warps; }
void keldysh_varlen_warps_set(int w) { g_kel_varlen_warps = w; }

int launch_keldysh_varlen(const double *Mt, const int64_t *m_off, const int *n_arr, int64_t batch, int n_max,
                          int sgn, double *sum, double *partial, uint32_t *status, void *stack,
                          const int *order, unsigned *ctr, cudaStream_t s) {
    int err = 0;
    // the workspace holds a stack for every warp of the default launch
    // (keldysh_grid(batch) CTAs of kKelWarps warps, as apm_workspace_size sizes it)
    const int full = keldysh_grid(batch, &err);
    if (err) return err;
    const int warps = g_kel_varlen_warps > 0 ? g_kel_varlen_warps : kKelWarps;
    const size_t smem = static_cast<size_t>(warps) * sizeof(KelWarpSmem);
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, keldysh_varlen_kernel, warps * 32, smem);
    if (e != cudaSuccess || per_sm < 1) return e != cudaSuccess ? static_cast<int>(e) : 1;
    int64_t grid = static_cast<int64_t>(sms) * per_sm;
    const int64_t slots = static_cast<int64_t>(full) * kKelWarps;  // stacks in the workspace
    if (grid * warps > slots) grid = slots / warps;
    const int64_t need = (batch + warps - 1) / warps;
    if (grid > need) grid = need;
    keldysh_varlen_kernel<<<static_cast<int>(grid < 1 ? 1 : grid), warps * 32, smem, s>>>(
        reinterpret_cast<const double2 *>(Mt), m_off, n_arr, batch, n_max, sgn, sum, partial, status,
        static_cast<double2 *>(stack), kel_stack_entries(n_max), order, ctr);
    return static_cast<int>(cudaGetLastError());
}

size_t keldysh_stack_entries(int n) { return kel_stack_entries(n); }

int keldysh_grid(int64_t batch, int *err) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = kKelWarps * sizeof(KelWarpSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(keldysh_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(keldysh_varlen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, keldysh_kernel, kKelWarps * 32, smem);
    if (e != cudaSuccess || per_sm < 1) {
        *err = e != cudaSuccess ? static_cast<int>(e) : static_cast<int>(cudaErrorInvalidConfiguration);
        return 0;
    }
    *err = 0;
    const int64_t need = (batch + kKelWarps - 1) / kKelWarps;
    int64_t g = static_cast<int64_t>(sms) * per_sm;
    if (need < g) g = need;
    return static_cast<int>(g < 1 ? 1 : g);
}

int keldysh_warps_per_block() { return kKelWarps; }

// Chunks per matrix for a fixed-order launch: the smallest power of two whose
// (matrix, chunk) items fill at least 90 % of the warps' last round (chunks of
// at least 4 depth-first leaves), else the best fill among those allowed.
static int keldysh_chunk_log2(int n, int64_t batch, int64_t warps) {
    const int D = n > kKelTail ? n - kKelTail : 0;
    const int kmax = D > 2 ? D - 2 : 0;
    int best = 0;
    double best_fill = 0.0;
    for (int k = 0; k <= kmax; ++k) {
        const int64_t items = batch << k;
        const int64_t rounds = (items + warps - 1) / warps;
        const double fill = static_cast<double>(items) / static_cast<double>(rounds * warps);
        if (fill >= 0.9) return k;
        if (fill > best_fill + 1e-12) {
            best_fill = fill;
            best = k;
        }
    }
    return best;
}

int keldysh_plan(int n, int64_t batch, KeldyshPlan *p) {
    int err = 0;
    const int full = keldysh_grid(INT64_MAX / 64, &err);  // all resident CTAs
    if (err) return err;
    const int64_t warps = static_cast<int64_t>(full) * kKelWarps;
    p->kc = keldysh_chunk_log2(n, batch, warps);
    const int64_t items = batch << p->kc;
    const int64_t need = (items + kKelWarps - 1) / kKelWarps;
    p->grid = static_cast<int>(need < full ? (need < 1 ? 1 : need) : full);
    p->stack_bytes = static_cast<size_t>(p->grid) * kKelWarps * kel_stack_entries(n) * sizeof(double2);
    if (p->kc == 0) {
        p->slot_bytes = p->flag_bytes = p->ctr_bytes = 0;
    } else {
        p->slot_bytes = static_cast<size_t>(items) * (n + 1) * sizeof(double2);
        p->flag_bytes = (static_cast<size_t>(items) * sizeof(uint32_t) + 15) & ~size_t(15);
        p->ctr_bytes = (static_cast<size_t>(batch) * sizeof(unsigned) + 15) & ~size_t(15);
    }
    p->total = p->stack_bytes + p->slot_bytes + p->flag_bytes + p->ctr_bytes;
    return 0;
}

int launch_keldysh(const double *Mt, int n, int64_t batch, int sgn, double *sum, double *partial,
                   uint32_t *status, void *workspace, cudaStream_t s) {
    KeldyshPlan p;
    const int err = keldysh_plan(n, batch, &p);
    if (err) return err;
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    double2 *stack = p.stack_bytes ? reinterpret_cast<double2 *>(ws) : nullptr;
    double2 *slots = nullptr;
    uint32_t *slot_flags = nullptr;
    unsigned *ctr = nullptr;
    if (p.kc > 0) {
        slots = reinterpret_cast<double2 *>(ws + p.stack_bytes);
        slot_flags = reinterpret_cast<uint32_t *>(ws + p.stack_bytes + p.slot_bytes);
        ctr = reinterpret_cast<unsigned *>(ws + p.stack_bytes + p.slot_bytes + p.flag_bytes);
        const cudaError_t e = cudaMemsetAsync(ctr, 0, static_cast<size_t>(batch) * sizeof(unsigned), s);
        if (e != cudaSuccess) return static_cast<int>(e);
    }
    const size_t smem = kKelWarps * sizeof(KelWarpSmem);
    keldysh_kernel<<<p.grid, kKelWarps * 32, smem, s>>>(reinterpret_cast<const double2 *>(Mt), n, batch, sgn,
                                                        sum, partial, status, stack, kel_stack_entries(n), p.kc,
                                                        slots, slot_flags, ctr);
    return static_cast<int>(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Allocation-free variant: the depth-first stack lives in a fixed array in
// device memory that belongs to the library (no caller workspace).
// ---------------------------------------------------------------------------

constexpr int kKelNoAllocMaxN = 14;
constexpr int kKelNoAllocBlocks = 50;
constexpr int kKelNoAllocWarps = kKelNoAllocBlocks * kKelWarps;
constexpr size_t kKelNoAllocStack = kel_stack_entries(kKelNoAllocMaxN);
static_assert(kKelNoAllocWarps == 600 && kKelNoAllocStack == 2716, "600 warp slots of an order-14 stack");

// 600 warps x 2716 complex entries x 16 B = 26.1 MB per device.
static __device__ __align__(256) double2 g_kel_noalloc_stack[kKelNoAllocWarps * kKelNoAllocStack];

}  // namespace apm

#include <mutex>

namespace {
std::mutex g_noalloc_mu;
constexpr int kNoAllocMaxDevices = 64;
void *g_noalloc_addr[kNoAllocMaxDevices] = {};
}  // namespace

extern "C" apm_status_t apm_keldysh_sum_noalloc(const double *Mt, int n, int64_t batch, int flags,
                                                double *sum, double *partial, uint32_t *status,
                                                apm_stream_t stream) {
    using namespace apm;
    if (n < 1 || n > kKelNoAllocMaxN) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0 || (flags & ~APM_KELDYSH_SIGNED)) return APM_ERR_ARG;
    auto bad_ptr = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) != 0; };
    if (batch > 0 && (!Mt || !sum || bad_ptr(Mt) || bad_ptr(sum))) return APM_ERR_ARG;
    if ((partial && bad_ptr(partial)) || (status && bad_ptr(status))) return APM_ERR_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return APM_ERR_CUDA;
    const size_t smem = kKelWarps * sizeof(KelWarpSmem);
    void *scratch = nullptr;
    {
        // first call on this device, even with batch 0: resolve the device
        // address of the array (a host-side name of a __device__ array is not a
        // device address; the lookup also loads the module, and with it the
        // array, if lazy loading has not done so yet) and allow the kernel its
        // shared memory
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *q = nullptr;
            if (cudaGetSymbolAddress(&q, g_kel_noalloc_stack) != cudaSuccess || !q) return APM_ERR_CUDA;
            if (cudaFuncSetAttribute(keldysh_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem)) != cudaSuccess)
                return APM_ERR_CUDA;
            g_noalloc_addr[dev] = q;
        }
        scratch = g_noalloc_addr[dev];
    }
    if (batch == 0) return APM_OK;
    const int64_t need = (batch + kKelWarps - 1) / kKelWarps;
    const int grid = static_cast<int>(need < kKelNoAllocBlocks ? need : kKelNoAllocBlocks);
    keldysh_kernel<<<grid, kKelWarps * 32, smem, reinterpret_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const double2 *>(Mt), n, batch, (flags & APM_KELDYSH_SIGNED) ? 1 : 0, sum,
        partial, status, static_cast<double2 *>(scratch), kel_stack_entries(n), 0, nullptr, nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? APM_OK : APM_ERR_CUDA;
}
