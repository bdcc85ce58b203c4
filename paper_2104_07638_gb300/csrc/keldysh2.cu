// Two-spin Keldysh sum: sum over the 2^n Keldysh assignments alpha, shared by
// both spins, of det(M_up,alpha) det(M_dn,alpha) (complex128).
//
// Paper: Section V.D (the sum over Keldysh assignments of a determinant is the
// sum of the XOR minors of the 2n x 2n block matrix, by the binary tree of
// Section III.D, with the lower orders as side products) applied to the two
// determinants per configuration of Eq. CTINT (one per spin): the tree is
// walked once for both matrices, a node carrying one Schur complement per spin
// and the product of both spins' pivots along its path; the per-depth sums are
// the same sums for the first d vertices.
//
// Mapping as in keldysh.cu, with two matrices per node: one warp per matrix
// pair; the upper vertices depth first (both spins' path matrices on a per-warp
// stack in caller scratch), the last 6 vertices breadth first in shared memory
// (the lanes cover the entries of both spins at once), and the last three
// vertices of every 6 x 6 node pair in closed form: lane (a0, a1) forms, per
// spin, the two 3 x 3 XOR minors with a2 = 0, 1 and adds their products. The
// running sums stay in lane registers and are reduced once per matrix.
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

constexpr int kK2Tail = 6;
constexpr int kK2Warps = 12;  // 17 KB of shared memory per warp, 168 registers per thread: 12 warps fill an SM
// Tail nodes are stored as in keldysh.cu, without the off-diagonal entries of
// the 2 x 2 blocks (never read by an XOR minor): row r of a node of size m
// holds its m - 1 columns q != r ^ 1 in order. Per spin: bufE holds the root
// (132) and level 1 (224), bufO levels 0 (180) and 2 (240).
constexpr int kK2BufE = 224, kK2BufO = 240;
constexpr int kK2Fac = 48;  // row factors per spin: 8 children x 6 rows at level 2; 30 for a depth-first step
constexpr int kK2MaxN = 16;

struct alignas(16) K2WarpSmem {
    double2 bufE[2][kK2BufE];  // [spin]
    double2 bufO[2][kK2BufO];
    double2 fac[2][kK2Fac];
    double2 inv[2][8];
    double2 ndet[2][8];  // node products (both spins, signed) of the current and the next level
    double2 part[kK2MaxN + 1];
    double2 pdet[kK2MaxN + 1];
};

// per-warp stack entries (double2) for order n, both spins: depths 1..D-1, D = n - 6
__host__ __device__ constexpr size_t k2_stack_entries(int n) {
    const int D = n > kK2Tail ? n - kK2Tail : 0;
    size_t t = 0;
    for (int d = 1; d < D; ++d) t += static_cast<size_t>(2 * (n - d)) * (2 * (n - d));
    return 2 * t;
}

struct K2Acc {
    double2 v[kK2Tail];  // r = n - depth: r = 0 the full sum, r >= 1 the tail's lower orders
};

// One breadth-first level J of a tail over S vertices, both spins: the 2^J node
// pairs of size m = 2(S-J) in cur give 2^(J+1) children of size m-2 in nxt
// (compact layout: the pivot (alpha, alpha) is compact column 0 of row alpha,
// entry (r+2, alpha) column alpha of row r+2, entry (alpha, q+2) column q+1 of
// row alpha, entry (r+2, q+2) the child's compact column of (r, q) plus 2).
template <int S, int J>
__device__ __forceinline__ void k2_tail_level(const double2 *cur0, const double2 *cur1, double2 *nxt0,
                                              double2 *nxt1, bool want_part, bool sgn, K2WarpSmem &w, int lane,
                                              int &bad, K2Acc &acc) {
    constexpr int m = 2 * (S - J), m2 = m - 2, rl = m - 1, rl2 = m2 - 1, mm = m * rl, mm2 = m2 * rl2;
    constexpr int nchild = 2 << J;
    static_assert(2 * nchild <= 32, "a lane per child and spin");
    if (lane < 2 * nchild) {  // lanes [0, nchild) spin up, [nchild, 2 nchild) spin down
        const int sp = lane >= nchild ? 1 : 0, c = lane - sp * nchild, alpha = c & 1;
        w.inv[sp][c] = crcp((sp ? cur1 : cur0)[(c >> 1) * mm + alpha * rl], bad);
    }
    if (lane < nchild) {
        const int alpha = lane & 1;
        const double2 p0 = cur0[(lane >> 1) * mm + alpha * rl];
        const double2 p1 = cur1[(lane >> 1) * mm + alpha * rl];
        const double2 nd = cneg_if(cmul(cmul(w.ndet[J & 1][lane >> 1], p0), p1), sgn && alpha);
        w.ndet[(J + 1) & 1][lane] = nd;
        if (want_part) acc.v[S - 1 - J] = cadd(acc.v[S - 1 - J], nd);
    }
    __syncwarp();
    for (int idx = lane; idx < 2 * nchild * m2; idx += 32) {
        const int sp = idx / (nchild * m2), i = idx - sp * nchild * m2;
        const int c = i / m2, r = i - c * m2, alpha = c & 1;
        const double2 *P = (sp ? cur1 : cur0) + (c >> 1) * mm;
        w.fac[sp][i] = cmul(P[(r + 2) * rl + alpha], w.inv[sp][c]);
    }
    __syncwarp();
    for (int e = lane; e < 2 * nchild * mm2; e += 32) {
        const int sp = e / (nchild * mm2), i = e - sp * nchild * mm2;
        const int c = i / mm2, rem = i - c * mm2, r = rem / rl2, cc = rem - r * rl2, alpha = c & 1;
        const int q = cc + (cc >= (r ^ 1));
        const double2 *P = (sp ? cur1 : cur0) + (c >> 1) * mm;
        (sp ? nxt1 : nxt0)[i] = cfms(w.fac[sp][c * m2 + r], P[alpha * rl + q + 1], P[(r + 2) * rl + cc + 2]);
    }
    __syncwarp();
}

// Per spin, for lane (a0, a1) of a 6 x 6 node (compact rows of 5): the leading
// entry A, the leading 2 x 2 cofactor C2 and the two 3 x 3 XOR minors (a2 = 0,
// 1), by expansion along the last row. Entry (i, j) of another block than i's
// is at compact column j - (j > i), the diagonal entry (i, i) at i & ~1.
struct K2Minors {
    double2 A, C2, d0, d1;
};
__device__ __forceinline__ K2Minors k2_minors3(const double2 *M, int a0, int a1) {
    const int r0 = a0, r1 = 2 + a1;
    K2Minors o;
    o.A = M[r0 * 5];
    const double2 B = M[r0 * 5 + r1 - 1], Dv = M[r1 * 5 + r0], E = M[r1 * 5 + 2];
    o.C2 = cfms(B, Dv, cmul(o.A, E));
#pragma unroll
    for (int a2 = 0; a2 < 2; ++a2) {
        const int r2 = 4 + a2;
        const double2 C = M[r0 * 5 + r2 - 1], F = M[r1 * 5 + r2 - 1];
        const double2 G = M[r2 * 5 + r0], H = M[r2 * 5 + r1], Iv = M[r2 * 5 + 4];
        const double2 u = cfms(C, E, cmul(B, F));
        const double2 v = cfms(C, Dv, cmul(o.A, F));
        const double2 det = cfma(Iv, o.C2, cfms(H, v, cmul(G, u)));
        if (a2 == 0) o.d0 = det;
        else o.d1 = det;
    }
    return o;
}

// Closed form for the last three vertices of NODES node pairs (6 x 6 each): the
// products of the two spins' minors, summed over a2, four lanes per node.
template <int NODES>
__device__ __forceinline__ void k2_closed3(const double2 *cur0, const double2 *cur1, const double2 *nd,
                                           bool want_part, bool sgn, int lane, K2Acc &acc) {
    for (int idx = lane; idx < 4 * NODES; idx += 32) {
        const int k = idx >> 2, a0 = idx & 1, a1 = (idx >> 1) & 1;
        const K2Minors u = k2_minors3(cur0 + k * 30, a0, a1);
        const K2Minors d = k2_minors3(cur1 + k * 30, a0, a1);
        const double2 t0 = cmul(u.d0, d.d0), t1 = cmul(u.d1, d.d1);
        const double2 tot = sgn ? csub(t0, t1) : cadd(t0, t1);
        const double2 dk = cneg_if(nd[k], sgn && (a0 ^ a1));
        acc.v[0] = cfma(dk, tot, acc.v[0]);
        if (want_part) {
            acc.v[1] = cfma(dk, cmul(u.C2, d.C2), acc.v[1]);
            if (a1 == 0) acc.v[2] = cfma(dk, cmul(u.A, d.A), acc.v[2]);
        }
    }
}

// Orders 1 and 2 (one node pair, the whole matrices; compact rows of 3 and 1).
__device__ __forceinline__ void k2_closed2(const double2 *M0, const double2 *M1, double2 det0, bool want_part,
                                           bool sgn, int lane, K2Acc &acc) {
    if (lane < 4) {
        const int a0 = lane & 1, a1 = lane >> 1;
        double2 d[2], A[2];
#pragma unroll
        for (int sp = 0; sp < 2; ++sp) {
            const double2 *M = sp ? M1 : M0;
            A[sp] = M[a0 * 3];
            d[sp] = cfms(M[a0 * 3 + 1 + a1], M[(2 + a1) * 3 + a0], cmul(A[sp], M[(2 + a1) * 3 + 2]));
        }
        const double2 dk = cneg_if(det0, sgn && (a0 ^ a1));
        acc.v[0] = cfma(dk, cmul(d[0], d[1]), acc.v[0]);
        if (want_part && a1 == 0) acc.v[1] = cfma(dk, cmul(A[0], A[1]), acc.v[1]);
    }
}
__device__ __forceinline__ void k2_closed1(const double2 *M0, const double2 *M1, double2 det0, bool sgn, int lane,
                                           K2Acc &acc) {
    if (lane == 0) {
        const double2 t0 = cmul(M0[0], M1[0]), t1 = cmul(M0[1], M1[1]);
        acc.v[0] = cfma(det0, sgn ? csub(t0, t1) : cadd(t0, t1), acc.v[0]);
    }
}

template <int S, int J>
__device__ __forceinline__ void k2_tail_levels(double2 *c0, double2 *c1, double2 *n0, double2 *n1, double2 det0,
                                               bool want_part, bool sgn, K2WarpSmem &w, int lane, int &bad,
                                               K2Acc &acc) {
    if constexpr (S <= 2) {
        if constexpr (S == 2) k2_closed2(c0, c1, det0, want_part, sgn, lane, acc);
        else k2_closed1(c0, c1, det0, sgn, lane, acc);
    } else if constexpr (J < S - 3) {
        k2_tail_level<S, J>(c0, c1, n0, n1, want_part, sgn, w, lane, bad, acc);
        k2_tail_levels<S, J + 1>(n0, n1, c0, c1, det0, want_part, sgn, w, lane, bad, acc);
    } else {
        k2_closed3<(1 << J)>(c0, c1, w.ndet[J & 1], want_part, sgn, lane, acc);
    }
}

// Breadth-first tail over the last S vertices; the root pair (2S x 2S each) is
// in bufE with product det0; adds into the lane accumulators.
template <int S>
__device__ __forceinline__ void k2_tail(double2 det0, bool want_part, bool sgn, K2WarpSmem &w, int lane, int &bad,
                                        K2Acc &acc) {
    if (lane == 0) w.ndet[0][0] = det0;
    __syncwarp();
    k2_tail_levels<S, 0>(w.bufE[0], w.bufE[1], w.bufO[0], w.bufO[1], det0, want_part, sgn, w, lane, bad, acc);
    __syncwarp();
}

template <int S>
__device__ __forceinline__ void k2_tail_order(int n, bool want_part, bool sgn, K2WarpSmem &w, int lane, int &bad,
                                              K2Acc &acc) {
    if constexpr (S >= 1) {
        if (n == S) k2_tail<S>(make_double2(1.0, 0.0), want_part, sgn, w, lane, bad, acc);
        else k2_tail_order<S - 1>(n, want_part, sgn, w, lane, bad, acc);
    }
}

// One depth-first Schur step for both spins: src (m x m, dense) -> dst ((m-2) x
// (m-2)): the entries a minor can read, dense on the stack (the blocks'
// off-diagonal entries left unwritten) or compact in the tail root.
__device__ __forceinline__ void k2_schur(const double2 *s0, const double2 *s1, int m, int alpha, double2 *d0,
                                         double2 *d1, bool root, K2WarpSmem &w, int lane, double2 &p0,
                                         double2 &p1, int &bad) {
    p0 = s0[alpha * m + alpha];
    p1 = s1[alpha * m + alpha];
    // one reciprocal per lane (even lanes spin up, odd lanes spin down), then
    // exchanged: a warp instruction costs the FP64 pipe the same for 1 or 32 lanes
    const double2 ivl = crcp((lane & 1) ? p1 : p0, bad);
    const double2 ivo = make_double2(__shfl_xor_sync(0xffffffffu, ivl.x, 1), __shfl_xor_sync(0xffffffffu, ivl.y, 1));
    const double2 iv0 = (lane & 1) ? ivo : ivl, iv1 = (lane & 1) ? ivl : ivo;
    const int m2 = m - 2;
    for (int idx = lane; idx < 2 * m2; idx += 32) {
        const int sp = idx >= m2, r = idx - sp * m2;
        w.fac[sp][r] = cmul((sp ? s1 : s0)[(r + 2) * m + alpha], sp ? iv1 : iv0);
    }
    __syncwarp();
    const int rl2 = m2 - 1, mm2 = m2 * rl2;
    for (int e = lane; e < 2 * mm2; e += 32) {
        const int sp = e >= mm2, i = e - sp * mm2, r = i / rl2, c = i - r * rl2, q = c + (c >= (r ^ 1));
        const double2 *P = sp ? s1 : s0;
        (sp ? d1 : d0)[root ? i : r * m2 + q] = cfms(w.fac[sp][r], P[alpha * m + q + 2], P[(r + 2) * m + q + 2]);
    }
    __syncwarp();
}

// One matrix pair of order n (whole warp): writes sum[2], partial[(n+1)*2] (if
// not NULL) and the status word; NaN where a pivot failed or an input is not finite.
__device__ __forceinline__ void k2_matrix(const double2 *Au, const double2 *Ad, int n, bool sgn, double *sum_out,
                                          double *partial_out, uint32_t *status_out, double2 *stack,
                                          K2WarpSmem &w, int lane) {
    const bool want_part = partial_out != nullptr;
    const int s = n < kK2Tail ? n : kK2Tail;
    const int D = n - s;
    const int m0 = 2 * n;
    int bad = 0, nonfin = 0;
    for (int e = lane; e < m0 * m0; e += 32) {
        const double2 u = Au[e], d = Ad[e];
        nonfin |= nonfinite_bits(u.x) | nonfinite_bits(u.y) | nonfinite_bits(d.x) | nonfinite_bits(d.y);
    }
    nonfin = __any_sync(0xffffffffu, nonfin);
    K2Acc acc;
#pragma unroll
    for (int r = 0; r < kK2Tail; ++r) acc.v[r] = make_double2(0.0, 0.0);
    if (lane <= n) w.part[lane] = make_double2(lane == 0 ? 1.0 : 0.0, 0.0);
    if (lane == 0) w.pdet[0] = make_double2(1.0, 0.0);
    __syncwarp();
    if (D == 0) {
        for (int e = lane; e < m0 * (m0 - 1); e += 32) {  // compact tail roots
            const int r = e / (m0 - 1), c = e - r * (m0 - 1), q = c + (c >= (r ^ 1));
            w.bufE[0][e] = Au[r * m0 + q];
            w.bufE[1][e] = Ad[r * m0 + q];
        }
        __syncwarp();
        k2_tail_order<kK2Tail>(n, want_part, sgn, w, lane, bad, acc);
    } else {
        const size_t half = k2_stack_entries(n) / 2;  // the down spin's path matrices follow the up spin's
        for (int64_t t = 0; t < (int64_t(1) << D); ++t) {
            const int d0 = t == 0 ? 0 : D - __ffsll(t);
            size_t off = 0;  // stack offset of depth d0 (depths 1..D-1 are stacked)
            for (int d = 1; d < d0; ++d) off += static_cast<size_t>(2 * (n - d)) * (2 * (n - d));
            for (int d = d0; d < D; ++d) {
                const int alpha = static_cast<int>((t >> (D - 1 - d)) & 1);
                const int m = 2 * (n - d);
                const double2 *s0 = d == 0 ? Au : stack + off;
                const double2 *s1 = d == 0 ? Ad : stack + half + off;
                if (d > 0) off += static_cast<size_t>(m) * m;
                double2 *t0 = (d + 1 == D) ? w.bufE[0] : stack + off;
                double2 *t1 = (d + 1 == D) ? w.bufE[1] : stack + half + off;
                double2 p0, p1;
                k2_schur(s0, s1, m, alpha, t0, t1, d + 1 == D, w, lane, p0, p1, bad);
                if (lane == 0) {
                    const double2 pd = cneg_if(cmul(cmul(w.pdet[d], p0), p1), sgn && alpha);
                    w.pdet[d + 1] = pd;
                    if (want_part) w.part[d + 1] = cadd(w.part[d + 1], pd);
                }
                __syncwarp();
            }
            k2_tail<kK2Tail>(w.pdet[D], want_part, sgn, w, lane, bad, acc);
        }
    }
#pragma unroll
    for (int r = 0; r < kK2Tail; ++r) {
        if (r == 0 || want_part) {
            const double2 v = warp_csum(acc.v[r]);
            if (lane == 0 && n - r >= 1) w.part[n - r] = cadd(w.part[n - r], v);
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    __syncwarp();
    const double nanv = __longlong_as_double(0x7ff8000000000000ll);
    if (lane == 0) {
        const double2 r = (bad || nonfin) ? make_double2(nanv, nanv) : w.part[n];
        sum_out[0] = r.x;
        sum_out[1] = r.y;
        if (status_out) *status_out = (bad ? APM_ST_ZERO_PIVOT : 0u) | (nonfin ? APM_ST_NONFINITE_INPUT : 0u);
    }
    if (want_part && lane <= n) {
        const double2 r = (bad || nonfin) ? make_double2(nanv, nanv) : w.part[lane];
        partial_out[2 * lane] = r.x;
        partial_out[2 * lane + 1] = r.y;
    }
    __syncwarp();
}

__global__ void __launch_bounds__(kK2Warps * 32, 1) keldysh2_kernel(
    const double2 *__restrict__ Mu, const double2 *__restrict__ Md, int n, int64_t batch, int sgn_flag,
    double *sum, double *partial, uint32_t *status, double2 *stack_base, size_t stack_per_warp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    K2WarpSmem &w = reinterpret_cast<K2WarpSmem *>(smem_raw)[wid];
    const int64_t gw = static_cast<int64_t>(blockIdx.x) * kK2Warps + wid;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * kK2Warps;
    double2 *stack = stack_base ? stack_base + gw * stack_per_warp : nullptr;
    const int64_t m0 = 2 * n;
    for (int64_t b = gw; b < batch; b += nw)
        k2_matrix(Mu + b * m0 * m0, Md + b * m0 * m0, n, sgn_flag != 0, sum + 2 * b,
                  partial ? partial + b * (n + 1) * 2 : nullptr, status ? status + b : nullptr, stack, w, lane);
}

int keldysh2_grid(int64_t batch, int *err) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = kK2Warps * sizeof(K2WarpSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(keldysh2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, keldysh2_kernel, kK2Warps * 32, smem);
    if (e != cudaSuccess || per_sm < 1) {
        *err = e != cudaSuccess ? static_cast<int>(e) : static_cast<int>(cudaErrorInvalidConfiguration);
        return 0;
    }
    *err = 0;
    const int64_t need = (batch + kK2Warps - 1) / kK2Warps;
    int64_t g = static_cast<int64_t>(sms) * per_sm;
    if (need < g) g = need;
    return static_cast<int>(g < 1 ? 1 : g);
}

size_t keldysh2_workspace_bytes(int n, int64_t batch, int *err) {
    *err = 0;
    const size_t per = k2_stack_entries(n);
    if (per == 0 || batch == 0) return 0;
    const int grid = keldysh2_grid(batch, err);
    if (*err) return 0;
    return static_cast<size_t>(grid) * kK2Warps * per * sizeof(double2);
}

int launch_keldysh2(const double *Mu, const double *Md, int n, int64_t batch, int sgn, double *sum,
                    double *partial, uint32_t *status, void *workspace, cudaStream_t s) {
    int err = 0;
    const int grid = keldysh2_grid(batch, &err);
    if (err) return err;
    const size_t smem = kK2Warps * sizeof(K2WarpSmem);
    keldysh2_kernel<<<grid, kK2Warps * 32, smem, s>>>(
        reinterpret_cast<const double2 *>(Mu), reinterpret_cast<const double2 *>(Md), n, batch, sgn, sum, partial,
        status, static_cast<double2 *>(workspace), k2_stack_entries(n));
    return static_cast<int>(cudaGetLastError());
}

}  // namespace apm
