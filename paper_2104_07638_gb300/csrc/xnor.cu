// XNOR principal minors of 2n x 2n block matrices, and the Nambu CDet weights.
//
// Paper: Section III.B (XNOR minors: for a matrix of 2 x 2 blocks, the minors of
// the submatrices that keep both rows and columns of a subset of the blocks, by
// a binary tree whose left branch drops a block and whose right branch takes
// the Schur complement with respect to the 2 x 2 pivot block; 2^n minors in
// O(2^n), no pivot correction possible) and Section V.B (the CDet expansion
// around BCS theory needs exactly these minors of the Nambu matrix; the
// recursion that follows is the plain CDet one).
//
// minors[S] = det of the rows and columns 2i, 2i+1 of every vertex i in S;
// minors[0] = 1. The det of a child that keeps vertex v is the parent's det
// times det(P), P the 2 x 2 pivot block of the parent's Schur complement.
//
// Mapping: one warp per matrix. The vertices are eliminated from the last one
// down, so that every node matrix is the leading block of its vertices and
// dropping a vertex is only a smaller view of the same rows (no copy). The
// upper vertices s..n-1 (s = min(n, 8)) are walked depth first (the matrices
// of kept pivots on a per-warp stack in caller scratch, L2-resident); the last
// s vertices are expanded breadth first in shared memory, and the 4 x 4 nodes
// of the last two vertices are finished in closed form, one node per lane,
// each lane writing the four minors of its node as two 16-byte stores (the
// tail vertices are the low mask bits, so the writes of a warp are
// contiguous). An FP64 warp instruction costs the same pipe time whatever the
// number of active lanes, so the tail is sized to share each level's pivot
// inversions among many nodes: 8 vertices (2 to 32 nodes per level, 21 KB of
// shared memory per warp) measured 0.77 TFLOP/s at n = 12 against 0.70 for 7.
#include <cuda_runtime.h>
#include <stdint.h>

#include "apm_internal.cuh"

// x is infinite or NaN: the exponent bits all set, tested on the high word in
// integer arithmetic (no FP64 compare)
__device__ __forceinline__ bool nonfinite_bits(double x) {
    return (static_cast<unsigned>(__double2hiint(x)) & 0x7ff00000u) == 0x7ff00000u;
}
namespace apm {

// vertices expanded breadth first (S) and warps per CTA
#ifndef APM_XN_TAIL
#define APM_XN_TAIL 8
#endif
constexpr int kXnTail = APM_XN_TAIL;
static_assert(kXnTail == 7 || kXnTail == 8, "tail of 7 or 8 vertices");
constexpr int kXnWarps = kXnTail == 7 ? 4 : 2;

// Tail level J (J = 0..S-2) holds 2^J nodes of size 2(S-J); even levels in
// bufE, odd levels in bufO. S = 7: bufE 196, 400, 576; bufO 288, 512, 512.
// S = 8: bufE 256, 576, 1024, 1024; bufO 392, 800, 1152.
__host__ __device__ constexpr int xn_level_entries(int S, int J) {
    return (1 << J) * (2 * (S - J)) * (2 * (S - J));
}
__host__ __device__ constexpr int xn_buf_entries(int S, int parity) {
    int b = 0;
    for (int J = parity; J <= S - 2; J += 2) b = b > xn_level_entries(S, J) ? b : xn_level_entries(S, J);
    return b;
}
// row factors of one level: 2 per row of every kept child (2^J x 2(S-J-1)), or
// of one depth-first step (at most 2 x 30)
__host__ __device__ constexpr int xn_fac_entries(int S) {
    int b = 60;
    for (int J = 0; J <= S - 3; ++J) b = b > (2 << J) * (2 * (S - J - 1)) ? b : (2 << J) * (2 * (S - J - 1));
    return b;
}
constexpr int kXnBufE = xn_buf_entries(kXnTail, 0);
constexpr int kXnBufO = xn_buf_entries(kXnTail, 1);
constexpr int kXnFac = xn_fac_entries(kXnTail);
static_assert(kXnTail != 7 || (kXnBufE == 576 && kXnBufO == 512 && kXnFac == 128), "7-vertex tail");
static_assert(kXnTail != 8 || (kXnBufE == 1024 && kXnBufO == 1152 && kXnFac == 256), "8-vertex tail");
constexpr int kXnMaxN = 16;

struct alignas(16) XnWarpSmem {
    double bufE[kXnBufE];
    double bufO[kXnBufO];
    double F[kXnFac];                  // row factors C P^-1 of one level or depth-first step
    double pinv[1 << (kXnTail - 3)][4];  // inverse pivot block of every node of one level
    double nd[2][1 << (kXnTail - 2)];    // node determinants of the current and the next level
    double pdet[kXnMaxN + 1];
    const double *vp[kXnMaxN + 1];  // depth-first views: first element and row stride
    int vs[kXnMaxN + 1];
};

static_assert(sizeof(XnWarpSmem) % 16 == 0, "per-warp blocks stay 16-byte aligned");

// stack entries (doubles) for order n: the kept-pivot matrices of depths 1..D-1 (D = n - S)
__host__ __device__ constexpr size_t xn_stack_entries(int n) {
    const int D = n > kXnTail ? n - kXnTail : 0;
    size_t t = 0;
    for (int d = 1; d < D; ++d) t += static_cast<size_t>(2 * (n - d)) * (2 * (n - d));
    return t;
}

// determinant of a 2 x 2 pivot block; flags a zero or non-finite value
__device__ __forceinline__ double xn_det2(double a, double b, double c, double d, int &bad) {
    const double det = fma(a, d, -b * c);
    const long long bits = __double_as_longlong(det);
    if ((bits << 1) == 0 || ((bits >> 52) & 0x7ff) == 0x7ff) bad = 1;
    return det;
}

// One breadth-first level J of a tail over S vertices: the 2^J nodes of size
// m = 2(S-J) in cur give 2^(J+1) children of size m-2 in nxt. Child 2k drops the
// node's last vertex (the leading block, copied: no arithmetic); child 2k+1
// keeps it: the Schur complement with respect to the trailing 2 x 2 block P,
// entry (r,q) = node(r,q) - F(r,0) node(m-2,q) - F(r,1) node(m-1,q), F = C P^-1.
template <int S, int J>
__device__ __forceinline__ void xn_tail_level(const double *cur, double *nxt, XnWarpSmem &w, int lane, int &bad) {
    constexpr int m = 2 * (S - J), m2 = m - 2, mm = m * m, mm2 = m2 * m2, nodes = 1 << J;
    const double *ndc = w.nd[J & 1];
    double *ndn = w.nd[(J + 1) & 1];
    if (lane < nodes) {
        const double *P = cur + lane * mm;
        const double a = P[(m - 2) * m + m - 2], b = P[(m - 2) * m + m - 1];
        const double c = P[(m - 1) * m + m - 2], d = P[(m - 1) * m + m - 1];
        const double det = xn_det2(a, b, c, d, bad);
        const double id = rcp_nr(det);
        w.pinv[lane][0] = d * id;
        w.pinv[lane][1] = -b * id;
        w.pinv[lane][2] = -c * id;
        w.pinv[lane][3] = a * id;
        ndn[2 * lane] = ndc[lane];
        ndn[2 * lane + 1] = ndc[lane] * det;
    }
    __syncwarp();
    for (int idx = lane; idx < nodes * m2; idx += 32) {
        const int k = idx / m2, r = idx - k * m2;
        const double *P = cur + k * mm;
        const double c0 = P[r * m + m - 2], c1 = P[r * m + m - 1];
        w.F[2 * idx] = fma(c0, w.pinv[k][0], c1 * w.pinv[k][2]);
        w.F[2 * idx + 1] = fma(c0, w.pinv[k][1], c1 * w.pinv[k][3]);
    }
    __syncwarp();
    for (int e = lane; e < nodes * mm2; e += 32) {
        const int k = e / mm2, rem = e - k * mm2, r = rem / m2, q = rem - r * m2;
        nxt[(2 * k) * mm2 + rem] = cur[k * mm + r * m + q];
    }
    for (int e = lane; e < nodes * mm2; e += 32) {
        const int k = e / mm2, rem = e - k * mm2, r = rem / m2, q = rem - r * m2;
        const double *P = cur + k * mm;
        const int f = 2 * (k * m2 + r);
        nxt[(2 * k + 1) * mm2 + rem] =
            fma(-w.F[f + 1], P[(m - 1) * m + q], fma(-w.F[f], P[(m - 2) * m + q], P[r * m + q]));
    }
    __syncwarp();
}

// The last two vertices (0 and 1) of every 4 x 4 node k, in closed form: the
// minors of {}, {0}, {1}, {0,1} are nd * (1, det B00, det B11, det of the node),
// the 4 x 4 determinant by Laplace expansion along rows 0 and 1 (products of
// complementary 2 x 2 minors). They go to out[4k .. 4k+3].
template <int S>
__device__ __forceinline__ void xn_bottom(const double *cur, const double *nd, double *out, int lane) {
    constexpr int nodes = 1 << (S - 2);
    for (int k = lane; k < nodes; k += 32) {
        const double *M = cur + 16 * k;
        // s_jk: rows 0,1 and columns j,k; c_jk: rows 2,3 and columns j,k
        const double s01 = fma(M[0], M[5], -M[1] * M[4]), s02 = fma(M[0], M[6], -M[2] * M[4]);
        const double s03 = fma(M[0], M[7], -M[3] * M[4]), s12 = fma(M[1], M[6], -M[2] * M[5]);
        const double s13 = fma(M[1], M[7], -M[3] * M[5]), s23 = fma(M[2], M[7], -M[3] * M[6]);
        const double c01 = fma(M[8], M[13], -M[9] * M[12]), c02 = fma(M[8], M[14], -M[10] * M[12]);
        const double c03 = fma(M[8], M[15], -M[11] * M[12]), c12 = fma(M[9], M[14], -M[10] * M[13]);
        const double c13 = fma(M[9], M[15], -M[11] * M[13]), c23 = fma(M[10], M[15], -M[11] * M[14]);
        double det4 = s01 * c23;
        det4 = fma(-s02, c13, det4);
        det4 = fma(s03, c12, det4);
        det4 = fma(s12, c03, det4);
        det4 = fma(-s13, c02, det4);
        det4 = fma(s23, c01, det4);
        const double d = nd[k];
        double2 *o = reinterpret_cast<double2 *>(out + 4 * k);
        o[0] = make_double2(d, d * s01);
        o[1] = make_double2(d * c23, d * det4);
    }
}

template <int S, int J>
__device__ __forceinline__ void xn_tail_levels(double *cur, double *nxt, double *out, XnWarpSmem &w, int lane,
                                               int &bad) {
    if constexpr (J < S - 2) {
        xn_tail_level<S, J>(cur, nxt, w, lane, bad);
        xn_tail_levels<S, J + 1>(nxt, cur, out, w, lane, bad);
    } else {
        xn_bottom<S>(cur, w.nd[J & 1], out, lane);
    }
}

// Breadth-first tail over the last S vertices (0..S-1); the root (2S x 2S,
// dense) is in bufE with determinant det0; writes out[0 .. 2^S).
template <int S>
__device__ __forceinline__ void xn_tail(double det0, double *out, XnWarpSmem &w, int lane, int &bad) {
    if constexpr (S == 1) {
        if (lane == 0) {
            out[0] = det0;
            out[1] = det0 * fma(w.bufE[0], w.bufE[3], -w.bufE[1] * w.bufE[2]);
        }
    } else {
        if (lane == 0) w.nd[0][0] = det0;
        __syncwarp();
        xn_tail_levels<S, 0>(w.bufE, w.bufO, out, w, lane, bad);
    }
    __syncwarp();
}

// Whole matrix of order n <= S as one tail.
template <int S>
__device__ __forceinline__ void xn_tail_order(int n, double *out, XnWarpSmem &w, int lane, int &bad) {
    if constexpr (S >= 1) {
        if (n == S) xn_tail<S>(1.0, out, w, lane, bad);
        else xn_tail_order<S - 1>(n, out, w, lane, bad);
    }
}

// Schur complement of the m x m view P (row stride st) with respect to its
// trailing 2 x 2 block, into dst ((m-2) x (m-2), dense); det = det of the block.
__device__ __forceinline__ void xn_schur(const double *P, int st, int m, double *dst, XnWarpSmem &w, int lane,
                                         int &bad, double &det) {
    const int m2 = m - 2;
    const double a = P[(m - 2) * st + m - 2], b = P[(m - 2) * st + m - 1];
    const double c = P[(m - 1) * st + m - 2], d = P[(m - 1) * st + m - 1];
    det = xn_det2(a, b, c, d, bad);
    const double id = rcp_nr(det);
    const double i00 = d * id, i01 = -b * id, i10 = -c * id, i11 = a * id;
    for (int r = lane; r < m2; r += 32) {
        const double c0 = P[r * st + m - 2], c1 = P[r * st + m - 1];
        w.F[2 * r] = fma(c0, i00, c1 * i10);
        w.F[2 * r + 1] = fma(c0, i01, c1 * i11);
    }
    __syncwarp();
    for (int e = lane; e < m2 * m2; e += 32) {
        const int r = e / m2, q = e - r * m2;
        dst[e] = fma(-w.F[2 * r + 1], P[(m - 1) * st + q], fma(-w.F[2 * r], P[(m - 2) * st + q], P[r * st + q]));
    }
    __syncwarp();
}

// One matrix of order n (whole warp): all 2^n XNOR minors into out, and the
// status word. A zero or non-finite pivot block, or a non-finite input, sets
// the status and makes the whole row NaN.
__device__ __forceinline__ void xn_matrix(const double *A, int n, double *out, uint32_t *status_out,
                                          double *stack, XnWarpSmem &w, int lane) {
    const int s = n < kXnTail ? n : kXnTail;
    const int D = n - s;
    const int m0 = 2 * n;
    int bad = 0, nonfin = 0;
    for (int e = lane; e < m0 * m0; e += 32)
        nonfin |= nonfinite_bits(A[e]);
    nonfin = __any_sync(0xffffffffu, nonfin);
    if (!nonfin) {
        if (D == 0) {
            for (int e = lane; e < m0 * m0; e += 32) w.bufE[e] = A[e];
            __syncwarp();
            xn_tail_order<kXnTail>(n, out, w, lane, bad);
        } else {
            if (lane == 0) {
                w.vp[0] = A;
                w.vs[0] = m0;
                w.pdet[0] = 1.0;
            }
            __syncwarp();
            for (int64_t t = 0; t < (int64_t(1) << D); ++t) {
                // first depth whose decision changed from t-1 to t (vertex n-1 <-> top bit)
                const int d0 = t == 0 ? 0 : D - __ffsll(t);
                for (int d = d0; d < D; ++d) {
                    const int keep = static_cast<int>((t >> (D - 1 - d)) & 1);
                    const double *P = w.vp[d];
                    const int st = w.vs[d], m = 2 * (n - d);
                    if (keep) {
                        double *dst = w.bufE;
                        if (d + 1 < D) {  // stack slot of depth d+1
                            size_t off = 0;
                            for (int k = 1; k <= d; ++k) off += static_cast<size_t>(2 * (n - k)) * (2 * (n - k));
                            dst = stack + off;
                        }
                        double det;
                        xn_schur(P, st, m, dst, w, lane, bad, det);
                        if (lane == 0) {
                            w.vp[d + 1] = dst;
                            w.vs[d + 1] = m - 2;
                            w.pdet[d + 1] = w.pdet[d] * det;
                        }
                    } else {
                        if (d + 1 == D) {  // the tail root must be dense
                            const int m2 = m - 2;
                            for (int e = lane; e < m2 * m2; e += 32) {
                                const int r = e / m2, q = e - r * m2;
                                w.bufE[e] = P[r * st + q];
                            }
                        }
                        if (lane == 0) {
                            w.vp[d + 1] = d + 1 == D ? w.bufE : P;
                            w.vs[d + 1] = d + 1 == D ? m - 2 : st;
                            w.pdet[d + 1] = w.pdet[d];
                        }
                    }
                    __syncwarp();
                }
                xn_tail<kXnTail>(w.pdet[D], out + (t << s), w, lane, bad);
            }
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    if (bad || nonfin) {
        const double nanv = __longlong_as_double(0x7ff8000000000000ll);
        for (int64_t e = lane; e < (int64_t(1) << n); e += 32) out[e] = nanv;
    }
    if (lane == 0 && status_out)
        *status_out = (bad ? APM_ST_ZERO_PIVOT : 0u) | (nonfin ? APM_ST_NONFINITE_INPUT : 0u);
    __syncwarp();
}

// CTAs per SM that the shared memory allows (228 KB per SM, 1 KB reserved per CTA)
constexpr int kXnMinBlocks = static_cast<int>((228 * 1024) / (kXnWarps * sizeof(XnWarpSmem) + 1024));

__global__ void __launch_bounds__(kXnWarps * 32, kXnMinBlocks) xnor_kernel(const double *__restrict__ M, int n, int64_t batch,
                                                             double *minors, uint32_t *status, double *stack_base,
                                                             size_t stack_per_warp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    XnWarpSmem &w = reinterpret_cast<XnWarpSmem *>(smem_raw)[wid];
    const int64_t gw = static_cast<int64_t>(blockIdx.x) * kXnWarps + wid;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * kXnWarps;
    double *stack = stack_base ? stack_base + gw * stack_per_warp : nullptr;
    const int64_t m0 = 2 * n, N = int64_t(1) << n;
    for (int64_t b = gw; b < batch; b += nw)
        xn_matrix(M + b * m0 * m0, n, minors + b * N, status ? status + b : nullptr, stack, w, lane);
}

int xnor_grid(int64_t batch, int *err) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = kXnWarps * sizeof(XnWarpSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(xnor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xnor_kernel, kXnWarps * 32, smem);
    if (e != cudaSuccess || per_sm < 1) {
        *err = e != cudaSuccess ? static_cast<int>(e) : static_cast<int>(cudaErrorInvalidConfiguration);
        return 0;
    }
    *err = 0;
    const int64_t need = (batch + kXnWarps - 1) / kXnWarps;
    int64_t g = static_cast<int64_t>(sms) * per_sm;
    if (need < g) g = need;
    return static_cast<int>(g < 1 ? 1 : g);
}

size_t xnor_workspace_bytes(int n, int64_t batch, int *err) {
    *err = 0;
    const size_t per = xn_stack_entries(n);
    if (per == 0 || batch == 0) return 0;
    const int grid = xnor_grid(batch, err);
    if (*err) return 0;
    return static_cast<size_t>(grid) * kXnWarps * per * sizeof(double);
}

int launch_xnor(const double *M, int n, int64_t batch, double *minors, uint32_t *status, void *workspace,
                cudaStream_t s) {
    int err = 0;
    const int grid = xnor_grid(batch, &err);
    if (err) return err;
    const size_t smem = kXnWarps * sizeof(XnWarpSmem);
    xnor_kernel<<<grid, kXnWarps * 32, smem, s>>>(M, n, batch, minors, status, static_cast<double *>(workspace),
                                                 xn_stack_entries(n));
    return static_cast<int>(cudaGetLastError());
}

}  // namespace apm
