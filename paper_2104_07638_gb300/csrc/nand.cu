// NAND principal minors of 2n x 2n block matrices, and the weights of the CDet
// summed over two vertex types.
//
// Paper: Section III.C (NAND minors: for a matrix of 2 x 2 blocks, the minors of
// the submatrices that keep at most one row and column of each block, 3^n of
// them; a ternary tree whose left branch drops a block and whose two right
// branches take the Schur complement with respect to the block's first or
// second diagonal entry, dropping the other; O(3^n)) and Section V.C (summing
// the CDet over the two types of every vertex needs, for each vertex subset S,
// the sum over the 2^|S| type assignments of these minors; the recursion that
// follows is the plain CDet one).
//
// Indexing: a ternary assignment sigma (vertex i <-> base-3 digit i: 0 drops
// the block, 1 keeps row/column 2i, 2 keeps row/column 2i+1) has index
// sum_i sigma_i 3^i; minors3[0] = 1. The type sums: abar[S] = sum over sigma
// with {i : sigma_i != 0} = S, abar[0] = 1.
//
// Mapping: one warp per matrix, as for the XNOR minors: vertices eliminated
// from the last one down (a dropped vertex is a smaller view of the same
// rows), the upper vertices s..n-1 (s = min(n, 6)) depth first in base 3 (the
// matrices of kept pivots on a per-warp stack in caller scratch), the last s
// vertices breadth first in shared memory, and the 4 x 4 nodes of the last two
// vertices in closed form (9 minors per node). For the type sums the closed
// form gives the 4 sums over the types of those two vertices, and the other
// tail vertices are reduced in shared memory vertex by vertex (the two kept
// types of one vertex added, in a fixed order) to 2^s sums, which the warp
// adds into the matrix's row.
//
// Pivot correction (Section III.C: as in the FPM tree, with the corrections
// back-propagated at the end). Two launches: the first runs the tree without
// shifts and only flags the matrices that meet a pivot below the threshold;
// the second redoes the flagged ones (usually none) with the corrections, so
// that the common path keeps the plain tree's code. A pivot p with
// |p| <= thr ||A||max is replaced
// by p + C, C = sign(p) shift ||A||max, and the minors of the kept child's
// subtree are those of the shifted matrix; det(A[S]) = det(A~[S]) - C
// det(A[S \ {row}]) turns them back, the minors of the dropped sibling's
// subtree supplying det(A[S \ {row}]), deepest vertex first. In the ternary
// index that is out[b + t 3^v + L] -= C out[b + L] over the 3^v lower indices
// L of the node (b the node's base, t the corrected type of vertex v). Tail
// corrections are applied per tail (to its 3^s minors, or to its partial type
// sums just before vertex v is reduced); depth-first corrections are logged
// and applied to the whole row at the end (all-minor mode), or, for the type
// sums, the dropped branch of a corrected node adds its leaves' sums a second
// time, times -(C_1 + C_2), into the sets that keep the node's vertex (a list
// of target masks and weights per depth).
#include <cuda_runtime.h>
#include <stdint.h>

#include "apm_internal.cuh"

namespace apm {

constexpr int kNdTail = 6;   // vertices expanded breadth first
constexpr int kNdWarps = 2;  // warps per CTA
constexpr int kNdMaxN = 16;
// per-warp correction records in caller scratch, after the depth-first stack:
// every pivot of a tail (2 (1 + 3 + 9 + 27) for 6 vertices), depth-first
// pivots of the all-minor mode, and per depth the type-sum target lists
constexpr int kNdTlogCap = 80;
constexpr int kNdDlogCap = 256;
constexpr int kNdFanCap = 16;
constexpr int kNdCorrDoubles = 2 * kNdTlogCap + 2 * kNdDlogCap + 2 * (kNdMaxN + 1) * kNdFanCap;

__host__ __device__ constexpr int nd_pow3(int k) {
    int r = 1;
    for (int i = 0; i < k; ++i) r *= 3;
    return r;
}
// Tail nodes are stored without the two off-diagonal entries of each 2 x 2
// diagonal block: a minor keeps at most one row and column of a block, and a
// Schur update of entry (r, q) reads only (r, q), (r, p), (p, q) and (p, p)
// with the pivot p in another block, so entries (2i, 2i+1) and (2i+1, 2i) are
// never read. Row r of a node of size m holds its m - 1 columns q != r ^ 1 in
// order (compact column c <-> q = c + (c >= (r ^ 1))); a column of another
// block has the same compact index in a node and in its children.
// Tail level J (J = 0..S-2) holds 3^J nodes of size m = 2(S-J), m(m-1) entries
// each; even levels in bufE, odd in bufO. S = 6: bufE 132, 504, 972; bufO 270, 810.
__host__ __device__ constexpr int nd_level_entries(int S, int J) {
    return nd_pow3(J) * (2 * (S - J)) * (2 * (S - J) - 1);
}
__host__ __device__ constexpr int nd_buf_entries(int S, int parity) {
    int b = 0;
    for (int J = parity; J <= S - 2; J += 2) b = b > nd_level_entries(S, J) ? b : nd_level_entries(S, J);
    return b;
}
constexpr int kNdBufE = nd_buf_entries(kNdTail, 0);
constexpr int kNdBufO = nd_buf_entries(kNdTail, 1);
static_assert(kNdBufE == 972 && kNdBufO == 810, "6-vertex tail");
static_assert(kNdBufO >= 729 && kNdBufE >= 729, "the 3^6 tail minors fit in either buffer");
// row factors of one level: 2 kept children per node, m-2 rows each (27 x 2 x 4)
constexpr int kNdFac = 216;

// 16-byte aligned, and a multiple of 16 bytes, so that every warp's buffers
// take 16-byte (double2) stores
struct alignas(16) NdWarpSmem {
    double bufE[kNdBufE];
    double bufO[kNdBufO];
    double f[kNdFac];                          // row factors of one level or depth-first step
    double inv[2 * nd_pow3(kNdTail - 3)];       // reciprocal pivots of one level (2 per node)
    double nd[2][nd_pow3(kNdTail - 2)];         // node determinants, current and next level
    double pdet[kNdMaxN + 1];
    const double *vp[kNdMaxN + 1];  // depth-first views: first element and row stride
    int vs[kNdMaxN + 1];
    int tcnt;                // correction records of the current tail
    int dcnt;                // depth-first correction records of the matrix (all-minor mode)
    int smask[kNdMaxN + 1];  // kept upper vertices (bit v) along the depth-first path
    int fcnt[kNdMaxN + 1];   // type-sum targets per depth: 1 = the path's own set (smask) alone,
                             // more = the list in the correction records
};

static_assert(sizeof(NdWarpSmem) % 16 == 0, "per-warp blocks stay 16-byte aligned");

// stack entries (doubles) for order n: the kept-pivot matrices of depths 1..D-1 (D = n - S)
__host__ __device__ constexpr size_t nd_stack_entries(int n) {
    const int D = n > kNdTail ? n - kNdTail : 0;
    size_t t = 0;
    for (int d = 1; d < D; ++d) t += static_cast<size_t>(2 * (n - d)) * (2 * (n - d));
    return t;
}
// per-warp scratch (doubles): the stack, then the correction records
__host__ __device__ constexpr size_t nd_warp_doubles(int n) { return nd_stack_entries(n) + kNdCorrDoubles; }

// Pivot-correction state of one matrix: the scaled threshold and shift, the
// warp's record areas, and per-lane flags (OR-reduced at the end).
struct NdCorr {
    double thrA, Cm;
    double *tlog;  // [kNdTlogCap][2]: code, C
    double *dlog;  // [kNdDlogCap][2]: code, C
    double *fan;   // [kNdMaxN + 1][kNdFanCap][2]: target mask, weight
    int corr, ovf;
};

// record code: vertex v, type t (1, 2), node index k (the digits of the vertices above v)
__device__ __forceinline__ double nd_code(int v, int t, int k) {
    return __longlong_as_double(static_cast<long long>(v) | (static_cast<long long>(t) << 5) |
                                (static_cast<long long>(k) << 8));
}
__device__ __forceinline__ void nd_decode(double c, int &v, int &t, int &k) {
    const long long x = __double_as_longlong(c);
    v = static_cast<int>(x & 31);
    t = static_cast<int>((x >> 5) & 7);
    k = static_cast<int>(x >> 8);
}

// |p| <= thrA (false for NaN)
__device__ __forceinline__ bool nd_small(double p, const NdCorr &cc) { return fabs(p) <= cc.thrA; }
// shift for pivot p: C = sign(p) Cm where |p| <= thrA (sign(0) = +1), else 0
__device__ __forceinline__ double nd_shift(double p, const NdCorr &cc) {
    return nd_small(p, cc) ? (p >= 0.0 ? cc.Cm : -cc.Cm) : 0.0;
}

// 1/p for a pivot; flags a zero or non-finite value
__device__ __forceinline__ double nd_inv(double p, int &bad) {
    const long long bits = __double_as_longlong(p);
    if ((bits << 1) == 0 || ((bits >> 52) & 0x7ff) == 0x7ff) bad = 1;
    return rcp_nr(p);
}

// The pivot phase of one tail level (nodes of size m, mm entries each, tail
// vertex v) when some pivot is below the threshold: rare, so out of line. Every
// pivot is taken again, the small ones shifted, and the shifted ones recorded.
// Returns the level's zero-pivot flag in bit 0 and the records' overflow in bit 1.
__device__ __noinline__ int nd_shift_level(const double *cur, const double *ndc, double *ndn, double *inv, int m,
                                           int mm, int nodes, int v, double thrA, double Cm, double *log, int *cnt,
                                           int lane) {
    int bad = 0, ovf = 0;
    for (int i0 = 0; i0 < 2 * nodes; i0 += 32) {
        const int i = i0 + lane;
        double C = 0.0;
        if (i < 2 * nodes) {
            const int k = i >> 1, t = i & 1;
            const double p = cur[k * mm + (m - 2 + t) * (m - 1) + (m - 2)];
            C = fabs(p) <= thrA ? (p >= 0.0 ? Cm : -Cm) : 0.0;
            const double pp = p + C;
            inv[i] = nd_inv(pp, bad);
            ndn[3 * k + 1 + t] = ndc[k] * pp;
        }
        const bool has = C != 0.0;
        const unsigned msk = __ballot_sync(0xffffffffu, has);
        const int base = *cnt;
        __syncwarp();
        if (has) {
            const int pos = base + __popc(msk & ((1u << lane) - 1u));
            if (pos < kNdTlogCap) {
                log[2 * pos] = nd_code(v, (i & 1) + 1, i >> 1);
                log[2 * pos + 1] = C;
            } else {
                ovf = 1;
            }
        }
        if (lane == 0) *cnt = base + __popc(msk);
        __syncwarp();
    }
    return bad | (ovf << 1);
}

// One breadth-first level J of a tail over S vertices: the 3^J nodes of size
// m = 2(S-J) in cur give 3^(J+1) children of size m-2 in nxt. Child 3k drops the
// node's last vertex (the leading block, copied); child 3k+1+t keeps its row
// and column p = m-2+t (t = 0, 1) and drops the other: the rank-1 Schur update
// (r,q) -= f(r) node(p, q), f(r) = node(r, p) / node(p, p). In the compact
// layout node(p, p) is at column m-2 of row p, node(r, p) at column p-1 of row
// r, and node(p, q), q < m-2, at column q of row p. A pivot below the threshold
// is flagged (kCorr = false), or shifted and recorded (tail vertex S-1-J, type
// t+1, node k).
template <int S, int J, bool kCorr>
__device__ __forceinline__ void nd_tail_level(const double *cur, double *nxt, NdWarpSmem &w, int lane, int &bad,
                                              NdCorr &cc) {
    constexpr int m = 2 * (S - J), m2 = m - 2, rl = m - 1, rl2 = m2 - 1;
    constexpr int mm = m * rl, mm2 = m2 * rl2, nodes = nd_pow3(J);
    const double *ndc = w.nd[J & 1];
    double *ndn = w.nd[(J + 1) & 1];
    int has = 0, badl = 0;
    for (int i = lane; i < 2 * nodes; i += 32) {
        const int k = i >> 1, t = i & 1, pi = m - 2 + t;
        const double p = cur[k * mm + pi * rl + (m - 2)];
        if constexpr (kCorr) {
            has |= nd_small(p, cc);
        } else {
            // the first pass on the high words in integer arithmetic: also true
            // up to 2^-20 above thrA, which only sends the matrix to the second
            // pass, whose test is exact
            has |= (static_cast<unsigned>(__double2hiint(p)) & 0x7fffffffu) <=
                   static_cast<unsigned>(__double2hiint(cc.thrA));
        }
        w.inv[i] = nd_inv(p, badl);
        ndn[3 * k + 1 + t] = ndc[k] * p;
        if (t == 0) ndn[3 * k] = ndc[k];
    }
    if constexpr (kCorr) {
        if (__any_sync(0xffffffffu, has)) {  // some pivot is shifted: the level's pivots again
            __syncwarp();
            cc.corr = 1;
            const int r = nd_shift_level(cur, ndc, ndn, w.inv, m, mm, nodes, S - 1 - J, cc.thrA, cc.Cm, cc.tlog,
                                         &w.tcnt, lane);
            badl = r & 1;
            cc.ovf |= r >> 1;
        }
    } else {
        cc.corr |= has;  // the matrix is redone with corrections
    }
    bad |= badl;
    __syncwarp();
    for (int idx = lane; idx < 2 * nodes * m2; idx += 32) {
        const int kt = idx / m2, r = idx - kt * m2;
        w.f[idx] = cur[(kt >> 1) * mm + r * rl + (m - 3 + (kt & 1))] * w.inv[kt];
    }
    __syncwarp();
    for (int e = lane; e < nodes * mm2; e += 32) {
        const int k = e / mm2, rem = e - k * mm2, r = rem / rl2, c = rem - r * rl2;
        nxt[(3 * k) * mm2 + rem] = cur[k * mm + r * rl + c];
    }
    for (int e = lane; e < 2 * nodes * mm2; e += 32) {
        const int kt = e / mm2, rem = e - kt * mm2, r = rem / rl2, c = rem - r * rl2;
        const int q = c + (c >= (r ^ 1));
        const int k = kt >> 1, t = kt & 1;
        const double *P = cur + k * mm;
        nxt[(3 * k + 1 + t) * mm2 + rem] = fma(-w.f[kt * m2 + r], P[(m - 2 + t) * rl + q], P[r * rl + c]);
    }
    __syncwarp();
}

// The last two vertices (0: rows 0,1; 1: rows 2,3) of every 4 x 4 node k in
// closed form: the 9 minors nd * (1, M00, M11, M22, det{0,2}, det{1,2}, M33,
// det{0,3}, det{1,3}) at out[9k + sigma_0 + 3 sigma_1]. A compact 4 x 4 node
// holds (M00 M02 M03 | M11 M12 M13 | M20 M21 M22 | M30 M31 M33).
template <int S>
__device__ __forceinline__ void nd_bottom(const double *cur, const double *nd, double *out, int lane) {
    constexpr int nodes = nd_pow3(S - 2);
    for (int k = lane; k < nodes; k += 32) {
        const double *M = cur + 12 * k;
        const double d = nd[k];
        double *o = out + 9 * k;
        o[0] = d;
        o[1] = d * M[0];
        o[2] = d * M[3];
        o[3] = d * M[8];
        o[4] = d * fma(M[0], M[8], -M[1] * M[6]);
        o[5] = d * fma(M[3], M[8], -M[4] * M[7]);
        o[6] = d * M[11];
        o[7] = d * fma(M[0], M[11], -M[2] * M[9]);
        o[8] = d * fma(M[3], M[11], -M[5] * M[10]);
    }
}

// The type sums of the last two vertices of every 4 x 4 node k: out[4k + b],
// bit 0 of b <-> vertex 0 kept, bit 1 <-> vertex 1 kept: nd * (1, M00 + M11,
// M22 + M33, the four minors of one row/column of each). The sum of the four
// 2 x 2 minors is (M00 + M11)(M22 + M33) minus the four off-block products.
template <int S>
__device__ __forceinline__ void nd_bottom_sum(const double *cur, const double *nd, double *out, int lane) {
    constexpr int nodes = nd_pow3(S - 2);
    for (int k = lane; k < nodes; k += 32) {
        const double *M = cur + 12 * k;
        const double d = nd[k];
        const double a = M[0] + M[3], b = M[8] + M[11];
        const double x = fma(M[1], M[6], fma(M[4], M[7], fma(M[2], M[9], M[5] * M[10])));
        double2 *o = reinterpret_cast<double2 *>(out + 4 * k);
        o[0] = make_double2(d, d * a);
        o[1] = make_double2(d * b, d * fma(a, b, -x));
    }
}

// Applies the records of vertex v in log[0 .. cnt) to an array whose index is
// L + (sigma_v + 3 k) * span, L < span, k the node index: entry (t, k, L) -=
// C * entry (0, k, L). Records of one vertex write disjoint entries and read
// only sigma_v = 0 ones.
__device__ __noinline__ void nd_apply(double *a, int v, int64_t span, const double *log, int cnt, int lane) {
    for (int j = 0; j < cnt; ++j) {
        int rv, t, k;
        nd_decode(log[2 * j], rv, t, k);
        if (rv != v) continue;
        const double C = log[2 * j + 1];
        double *b = a + static_cast<int64_t>(3 * k) * span;
        for (int64_t L = lane; L < span; L += 32) b[t * span + L] = fma(-C, b[L], b[t * span + L]);
    }
    __syncwarp();
}

// Type sums over the remaining tail vertices 2..s-1: a holds, for each node,
// the 4 sums of the last two vertices (index low + 4 * (ternary digits of
// vertices 2..s-1)); vertex by vertex, the tail's corrections of that vertex
// are applied and the entries of its two kept types are added (type 1 + type
// 2, a fixed order). Returns the buffer holding the 2^s sums (bit v <-> vertex
// v kept).
template <bool kCorr>
__device__ __forceinline__ const double *nd_type_sum(int s, double *a, double *b, const NdCorr &cc, int tcnt,
                                                     int lane) {
    int rest = nd_pow3(s - 3);
    for (int v = 2; v < s; ++v, rest /= 3) {
        const int lowsz = 1 << v;
        if constexpr (kCorr)
            if (tcnt) nd_apply(a, v, lowsz, cc.tlog, tcnt, lane);
        for (int j = lane; j < lowsz * rest; j += 32) {
            const int low = j & (lowsz - 1), r = j >> v;
            const int base = low + lowsz * 3 * r, i0 = low + lowsz * 2 * r;
            b[i0] = a[base];
            b[i0 + lowsz] = a[base + lowsz] + a[base + 2 * lowsz];
        }
        __syncwarp();
        double *t = a;
        a = b;
        b = t;
    }
    return a;
}

// Tail over the last S vertices; the root (2S x 2S, compact) is in bufE with
// determinant det0. kSum = false: the 3^S minors go to gout[0 .. 3^S), then
// the tail's corrections are applied to them; kSum = true: their type sums,
// corrected, are added to gout[mask0 + (0 .. 2^S)] (fcnt = 1), or to
// gout[mask + (0 .. 2^S)] times weight for every (mask, weight) of the target
// list fan[0 .. fcnt).
template <int S, int J, bool kSum, bool kCorr>
__device__ __forceinline__ void nd_tail_levels(double *cur, double *nxt, double *gout, int mask0, const double *fan,
                                               int fcnt, NdWarpSmem &w, int lane, int &bad, NdCorr &cc) {
    if constexpr (J < S - 2) {
        nd_tail_level<S, J, kCorr>(cur, nxt, w, lane, bad, cc);
        nd_tail_levels<S, J + 1, kSum, kCorr>(nxt, cur, gout, mask0, fan, fcnt, w, lane, bad, cc);
    } else if constexpr (!kSum) {
        nd_bottom<S>(cur, w.nd[J & 1], gout, lane);
        if constexpr (kCorr) {
            const int tcnt = w.tcnt < kNdTlogCap ? w.tcnt : kNdTlogCap;
            if (tcnt) {
                __syncwarp();
                for (int v = 2; v < S; ++v) nd_apply(gout, v, nd_pow3(v), cc.tlog, tcnt, lane);
            }
        }
    } else {
        nd_bottom_sum<S>(cur, w.nd[J & 1], nxt, lane);
        __syncwarp();
        const int tcnt = kCorr ? (w.tcnt < kNdTlogCap ? w.tcnt : kNdTlogCap) : 0;
        const double *T = nd_type_sum<kCorr>(S, nxt, cur, cc, tcnt, lane);
        if constexpr (!kCorr) {
            // atomic additions performed in L2 (no FP64 instruction, no load
            // latency on the SM); one warp owns the row and adds its leaves in
            // order, so the sums are the same on every run
            for (int i = lane; i < (1 << S); i += 32) atomicAdd(gout + mask0 + i, T[i]);
        } else if (fcnt <= 1) {
            for (int i = lane; i < (1 << S); i += 32) gout[mask0 + i] += T[i];
        } else {
            for (int j = 0; j < fcnt; ++j) {
                const int mk = static_cast<int>(fan[2 * j]);
                const double wt = fan[2 * j + 1];
                for (int i = lane; i < (1 << S); i += 32) gout[mk + i] = fma(wt, T[i], gout[mk + i]);
            }
        }
    }
}

template <int S, bool kSum, bool kCorr>
__device__ __forceinline__ void nd_tail(double det0, double *gout, int mask0, const double *fan, int fcnt,
                                        NdWarpSmem &w, int lane, int &bad, NdCorr &cc) {
    if constexpr (S == 1) {  // order 1: the whole matrix, no depth-first part (mask0 = 0, fcnt = 1)
        if (lane == 0) {
            if constexpr (kSum) {
                gout[0] += det0;
                gout[1] += det0 * (w.bufE[0] + w.bufE[1]);
            } else {
                gout[0] = det0;
                gout[1] = det0 * w.bufE[0];
                gout[2] = det0 * w.bufE[1];
            }
        }
    } else {
        if (lane == 0) {
            w.nd[0][0] = det0;
            w.tcnt = 0;
        }
        __syncwarp();
        nd_tail_levels<S, 0, kSum, kCorr>(w.bufE, w.bufO, gout, mask0, fan, fcnt, w, lane, bad, cc);
    }
    __syncwarp();
}

// Whole matrix of order n <= S as one tail.
template <int S, bool kSum, bool kCorr>
__device__ __forceinline__ void nd_tail_order(int n, double *gout, NdWarpSmem &w, int lane, int &bad, NdCorr &cc) {
    if constexpr (S >= 1) {
        if (n == S) nd_tail<S, kSum, kCorr>(1.0, gout, 0, nullptr, 1, w, lane, bad, cc);
        else nd_tail_order<S - 1, kSum, kCorr>(n, gout, w, lane, bad, cc);
    }
}

// Depth-first bookkeeping of the corrections (one lane, out of line).
// A record of a shifted depth-first pivot (all-minor mode); returns 1 on overflow.
__device__ __noinline__ int nd_dlog(double *dlog, int *dcnt, double code, double C) {
    const int j = *dcnt;
    *dcnt = j + 1;
    if (j >= kNdDlogCap) return 1;
    dlog[2 * j] = code;
    dlog[2 * j + 1] = C;
    return 0;
}
// Kept vertex v: the targets of depth d+1 are those of depth d with bit v set.
__device__ __noinline__ void nd_fan_keep(const double *fd, double *fn, int fc, int v) {
    for (int j = 0; j < fc; ++j) {
        fn[2 * j] = static_cast<double>(static_cast<int>(fd[2 * j]) | (1 << v));
        fn[2 * j + 1] = fd[2 * j + 1];
    }
}
// Dropped vertex v: the targets of depth d, and with Cs = C_1 + C_2 != 0 each
// once more with bit v set and weight -w Cs. Returns the new count, or -1 on
// overflow (the list is then cut at kNdFanCap).
__device__ __noinline__ int nd_fan_drop(const double *fd, double *fn, int fc, int v, double Cs) {
    int nc = fc, ovf = 0;
    for (int j = 0; j < fc; ++j) {
        fn[2 * j] = fd[2 * j];
        fn[2 * j + 1] = fd[2 * j + 1];
    }
    if (Cs != 0.0) {
        for (int j = 0; j < fc; ++j) {
            if (nc < kNdFanCap) {
                fn[2 * nc] = static_cast<double>(static_cast<int>(fd[2 * j]) | (1 << v));
                fn[2 * nc + 1] = -fd[2 * j + 1] * Cs;
                ++nc;
            } else {
                ovf = 1;
            }
        }
    }
    return ovf ? -1 : nc;
}

// One matrix of order n (whole warp). kSum = false: all 3^n minors into out;
// kSum = true: the 2^n type sums. kCorr = false (first pass): returns 1, and
// writes neither status nor NaN, when a pivot is below thr ||A||max, the row
// then being redone by the second pass; kCorr = true: such pivots are shifted
// and corrected as described at the top. A zero or non-finite pivot, a
// non-finite input or more corrections than the records hold set the status
// and make the whole row NaN.
template <bool kSum, bool kCorr>
__device__ __forceinline__ int nd_matrix(const double *A, int n, double *out, uint32_t *status_out, double thr,
                                         double shf, double *scratch, NdWarpSmem &w, int lane) {
    const int s = n < kNdTail ? n : kNdTail;
    const int D = n - s;
    const int m0 = 2 * n;
    const int64_t row = kSum ? (int64_t(1) << n) : static_cast<int64_t>(nd_pow3(n));
    double *stack = scratch;
    NdCorr cc;
    cc.tlog = scratch + nd_stack_entries(n);
    cc.dlog = cc.tlog + 2 * kNdTlogCap;
    cc.fan = cc.dlog + 2 * kNdDlogCap;
    cc.corr = 0;
    cc.ovf = 0;
    int bad = 0, nonfin = 0;
    // ||A||max and the finiteness test on the bit patterns of |x|, off the FP64 pipe
    unsigned long long am = 0;
    for (int e = lane; e < m0 * m0; e += 32) {
        const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(A[e])) & 0x7fffffffffffffffull;
        nonfin |= u >= 0x7ff0000000000000ull;
        am = u > am ? u : am;
    }
    nonfin = __any_sync(0xffffffffu, nonfin);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, am, o);
        am = y > am ? y : am;
    }
    const double amax = __longlong_as_double(static_cast<long long>(am));
    const double sc = amax > 0.0 ? amax : 1.0;
    cc.thrA = thr * sc;
    cc.Cm = shf * sc;
    if (kSum)
        for (int64_t e = lane; e < row; e += 32) out[e] = 0.0;
    if (lane == 0) {
        w.smask[0] = 0;  // depth 0: the row itself, weight 1
        w.fcnt[0] = 1;
        w.dcnt = 0;
    }
    __syncwarp();
    if (!nonfin) {
        if (D == 0) {
            for (int e = lane; e < m0 * (m0 - 1); e += 32) {  // compact tail root
                const int r = e / (m0 - 1), c = e - r * (m0 - 1);
                w.bufE[e] = A[r * m0 + c + (c >= (r ^ 1))];
            }
            __syncwarp();
            nd_tail_order<kNdTail, kSum, kCorr>(n, out, w, lane, bad, cc);
        } else {
            if (lane == 0) {
                w.vp[0] = A;
                w.vs[0] = m0;
                w.pdet[0] = 1.0;
            }
            __syncwarp();
            const int64_t T3 = nd_pow3(D), tail3 = nd_pow3(s);
            for (int64_t t = 0; t < T3; ++t) {
                // first depth whose digit changed from t-1 to t (vertex n-1 <-> top digit)
                int d0 = 0;
                if (t) {
                    int p = 0;
                    for (int64_t u = t; u % 3 == 0; u /= 3) ++p;
                    d0 = D - 1 - p;
                }
                for (int d = d0; d < D; ++d) {
                    const int digit = static_cast<int>((t / nd_pow3(D - 1 - d)) % 3);
                    const double *P = w.vp[d];
                    const int st = w.vs[d], m = 2 * (n - d), m2 = m - 2, v = n - 1 - d;
                    const double *fd = cc.fan + 2 * kNdFanCap * d;
                    double *fn = cc.fan + 2 * kNdFanCap * (d + 1);
                    const int fc = w.fcnt[d];
                    if (digit) {
                        const int pi = m - 2 + (digit - 1);
                        double *dst = w.bufE;
                        if (d + 1 < D) {  // stack slot of depth d+1
                            size_t off = 0;
                            for (int k = 1; k <= d; ++k) off += static_cast<size_t>(2 * (n - k)) * (2 * (n - k));
                            dst = stack + off;
                        }
                        const double piv = P[pi * st + pi];
                        double pp = piv;
                        if constexpr (kCorr) {
                            const double C = nd_shift(piv, cc);
                            pp = piv + C;
                            if (C != 0.0) {
                                cc.corr = 1;
                                if (lane == 0 && !kSum)  // logged for the row's final pass
                                    cc.ovf |= nd_dlog(cc.dlog, &w.dcnt,
                                                      nd_code(v, digit, static_cast<int>(t / nd_pow3(D - d))), C);
                            }
                        } else {
                            cc.corr |= nd_small(piv, cc);
                        }
                        const double iv = nd_inv(pp, bad);
                        for (int r = lane; r < m2; r += 32) w.f[r] = P[r * st + pi] * iv;
                        if (lane == 0) {
                            if (kSum) {  // the targets keep vertex v
                                w.smask[d + 1] = w.smask[d] | (1 << v);
                                if (kCorr && fc > 1) nd_fan_keep(fd, fn, fc, v);
                                w.fcnt[d + 1] = fc;
                            }
                        }
                        __syncwarp();
                        // the entries a minor can read (no within-block off-diagonals): dense on
                        // the stack, compact in the tail root
                        const bool root = d + 1 == D;
                        for (int e = lane; e < m2 * (m2 - 1); e += 32) {
                            const int r = e / (m2 - 1), c = e - r * (m2 - 1), q = c + (c >= (r ^ 1));
                            dst[root ? e : r * m2 + q] = fma(-w.f[r], P[pi * st + q], P[r * st + q]);
                        }
                        __syncwarp();
                        if (lane == 0) {
                            w.vp[d + 1] = dst;
                            w.vs[d + 1] = m2;
                            w.pdet[d + 1] = w.pdet[d] * pp;
                        }
                    } else {
                        double Cs = 0.0;
                        if (kSum && kCorr) {  // shifts of the node's two kept children, one pivot per lane
                            const double pv = lane < 2 ? P[(m - 2 + lane) * st + (m - 2 + lane)] : 0.0;
                            const double cl = lane < 2 ? nd_shift(pv, cc) : 0.0;
                            Cs = __shfl_sync(0xffffffffu, cl, 0) + __shfl_sync(0xffffffffu, cl, 1);
                        }
                        if (d + 1 == D) {  // the tail root is a compact copy
                            for (int e = lane; e < m2 * (m2 - 1); e += 32) {
                                const int r = e / (m2 - 1), c = e - r * (m2 - 1);
                                w.bufE[e] = P[r * st + c + (c >= (r ^ 1))];
                            }
                        }
                        if (lane == 0) {
                            w.vp[d + 1] = d + 1 == D ? w.bufE : P;
                            w.vs[d + 1] = d + 1 == D ? m2 : st;
                            w.pdet[d + 1] = w.pdet[d];
                            if (kSum) {
                                // the sets that keep v get this branch's sums again, times
                                // -(C_1 + C_2) of the node's kept children
                                w.smask[d + 1] = w.smask[d];
                                if (!kCorr || (Cs == 0.0 && fc == 1)) {
                                    w.fcnt[d + 1] = 1;
                                } else if (fc == 1) {  // the implicit list becomes two entries
                                    fn[0] = static_cast<double>(w.smask[d]);
                                    fn[1] = 1.0;
                                    fn[2] = static_cast<double>(w.smask[d] | (1 << v));
                                    fn[3] = -Cs;
                                    w.fcnt[d + 1] = 2;
                                } else {
                                    const int nc = nd_fan_drop(fd, fn, fc, v, Cs);
                                    if (nc < 0) cc.ovf = 1;
                                    w.fcnt[d + 1] = nc < 0 ? kNdFanCap : nc;
                                }
                            }
                        }
                    }
                    __syncwarp();
                }
                double *gout = kSum ? out : out + t * tail3;
                nd_tail<kNdTail, kSum, kCorr>(w.pdet[D], gout, kSum ? w.smask[D] : 0, cc.fan + 2 * kNdFanCap * D,
                                              kSum ? w.fcnt[D] : 1, w, lane, bad, cc);
            }
            if (kCorr && !kSum) {  // depth-first corrections over the whole row, deepest vertex first
                __syncwarp();
                const int dcnt = w.dcnt < kNdDlogCap ? w.dcnt : kNdDlogCap;
                if (dcnt)
                    for (int v = s; v < n; ++v) nd_apply(out, v, nd_pow3(v), cc.dlog, dcnt, lane);
            }
        }
    }
    bad = __any_sync(0xffffffffu, bad);
    const int ovf = __any_sync(0xffffffffu, cc.ovf);
    const int corr = __any_sync(0xffffffffu, cc.corr);
    if (!kCorr && corr && !nonfin) return 1;  // redone by the second pass
    if (bad || nonfin || ovf) {
        const double nanv = __longlong_as_double(0x7ff8000000000000ll);
        for (int64_t e = lane; e < row; e += 32) out[e] = nanv;
    }
    if (lane == 0 && status_out)
        *status_out = (bad ? APM_ST_ZERO_PIVOT : 0u) | (nonfin ? APM_ST_NONFINITE_INPUT : 0u) |
                      (kCorr && corr ? APM_ST_PIVOT_CORRECTED : 0u) | (ovf ? APM_ST_CORRECTION_OVERFLOW : 0u);
    __syncwarp();
    return 0;
}

// CTAs per SM that the shared memory allows (228 KB per SM, 1 KB reserved per CTA)
constexpr int kNdMinBlocks = static_cast<int>((228 * 1024) / (kNdWarps * sizeof(NdWarpSmem) + 1024));

// kCorr = false: every matrix, flag[b] = 1 where the second pass must redo it;
// kCorr = true: only the flagged matrices, with the corrections.
template <bool kSum, bool kCorr>
__global__ void __launch_bounds__(kNdWarps * 32, kNdMinBlocks) nand_kernel(const double *__restrict__ M, int n,
                                                                         int64_t batch, double *out,
                                                                         uint32_t *status, uint32_t *flag,
                                                                         double thr, double shf, double *scratch_base,
                                                                         size_t scratch_per_warp) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    NdWarpSmem &w = reinterpret_cast<NdWarpSmem *>(smem_raw)[wid];
    const int64_t gw = static_cast<int64_t>(blockIdx.x) * kNdWarps + wid;
    const int64_t nw = static_cast<int64_t>(gridDim.x) * kNdWarps;
    double *scratch = scratch_base + gw * scratch_per_warp;
    const int64_t m0 = 2 * n;
    const int64_t row = kSum ? (int64_t(1) << n) : static_cast<int64_t>(nd_pow3(n));
    for (int64_t b = gw; b < batch; b += nw) {
        if (kCorr && flag[b] == 0u) continue;
        const int redo = nd_matrix<kSum, kCorr>(M + b * m0 * m0, n, out + b * row, status ? status + b : nullptr,
                                                thr, shf, scratch, w, lane);
        if (!kCorr && lane == 0) flag[b] = static_cast<uint32_t>(redo);
    }
}

int nand_grid(int64_t batch, int *err) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = kNdWarps * sizeof(NdWarpSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(nand_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(nand_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(nand_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(nand_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
    int per_sm2 = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nand_kernel<true, false>, kNdWarps * 32, smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, nand_kernel<true, true>, kNdWarps * 32, smem);
    if (per_sm2 < per_sm) per_sm = per_sm2;
    if (e != cudaSuccess || per_sm < 1) {
        *err = e != cudaSuccess ? static_cast<int>(e) : static_cast<int>(cudaErrorInvalidConfiguration);
        return 0;
    }
    *err = 0;
    const int64_t need = (batch + kNdWarps - 1) / kNdWarps;
    int64_t g = static_cast<int64_t>(sms) * per_sm;
    if (need < g) g = need;
    return static_cast<int>(g < 1 ? 1 : g);
}

// per resident warp the stack and correction records, then one flag per matrix
size_t nand_workspace_bytes(int n, int64_t batch, int *err) {
    *err = 0;
    if (batch == 0) return 0;
    const int grid = nand_grid(batch, err);
    if (*err) return 0;
    return static_cast<size_t>(grid) * kNdWarps * nd_warp_doubles(n) * sizeof(double) +
           ((static_cast<size_t>(batch) * sizeof(uint32_t) + 15) & ~static_cast<size_t>(15));
}

int launch_nand(const double *M, int n, int64_t batch, double *out, bool type_sums, double thr, double shf,
                uint32_t *status, void *workspace, cudaStream_t s) {
    int err = 0;
    const int grid = nand_grid(batch, &err);
    if (err) return err;
    const size_t smem = kNdWarps * sizeof(NdWarpSmem);
    double *scratch = static_cast<double *>(workspace);
    const size_t per = nd_warp_doubles(n);
    uint32_t *flag = reinterpret_cast<uint32_t *>(scratch + static_cast<size_t>(grid) * kNdWarps * per);
    if (type_sums) {
        nand_kernel<true, false><<<grid, kNdWarps * 32, smem, s>>>(M, n, batch, out, status, flag, thr, shf,
                                                                   scratch, per);
        nand_kernel<true, true><<<grid, kNdWarps * 32, smem, s>>>(M, n, batch, out, status, flag, thr, shf,
                                                                  scratch, per);
    } else {
        nand_kernel<false, false><<<grid, kNdWarps * 32, smem, s>>>(M, n, batch, out, status, flag, thr, shf,
                                                                    scratch, per);
        nand_kernel<false, true><<<grid, kNdWarps * 32, smem, s>>>(M, n, batch, out, status, flag, thr, shf,
                                                                   scratch, per);
    }
    return static_cast<int>(cudaGetLastError());
}

}  // namespace apm
