// Fused all-principal-minors (Schur-complement tree with pivot correction) and
// CDet connected-sum recursion, FP64, one CTA per matrix, persistent over the
// batch.
//
// Paper: Section II (Eq. dets_schur, lemma1, lemma2, Eq. minor, Alg. 1, the
// pivot-correction paragraph and the depth-first remark), Section V.A
// (a[S] = det M_up[S] det M_dn[S], Eq. recursion).
//
// Layout on chip (doubles, for n <= 12 in shared memory, else in per-CTA global
// scratch):  MA[2^n]  minors, then a[]      MC[max(2^n,16)]  tree scratch, then c[]
//            MU[2^n]  (only with a separate A_dn) minors of A_dn
//
// Minors (per matrix):
//   The tree node of mask m over the elements < l holds the Schur complement of
//   A with respect to A[m], restricted to the elements l..n-1 (size (n-l)^2).
//   Its (1,1) entry p gives det A[m | {l}] = det A[m] * p (Eq. minor). The left
//   child (element l excluded) is the same matrix without its first row and
//   column; the right child (l included) is its Schur complement with respect
//   to p. Levels 0..L-1 (L = n-4) are expanded breadth first across the CTA
//   (per level: one thread per node for its minor and pivot reciprocal, then
//   the pivot rows scaled and the child entries formed, one entry per thread
//   step); the 2^L nodes of level L (4x4 each) are finished by one thread each:
//   one more Schur step on the node's first element (a pivot like the others,
//   corrected when tiny) and the 8 minors of each 3x3 child in closed form (56
//   FP64 operations per node against 73 for a 4x4 closed form). Level buffers
//   alternate between MC and the not yet written upper part of MA, so the tree
//   needs no memory beyond MA and MC.
//   Pivot correction: a pivot with |p| <= thr is shifted by C; the node's minor
//   is stored with p + C and the right subtree is built from the shifted
//   matrix. The shift equals adding C to A_ll for every mask of that subtree, so
//   by linearity in row l the exact minors follow from
//       det[m] = det~[m] - C det[m \ {l}]
//   for every mask of its right subtree below the node, applied deepest level
//   first (a shallower correction must see deeper ones already removed). The
//   node's own minor is written as det[m \ {l}] p with the logged unshifted
//   pivot: the subtraction would leave it with an error of eps C |det[m \ {l}]|,
//   large next to the minor itself when p is tiny.
//
// Connected sums: popcount layers k = 2..n in order (every proper subset of a
// k-set lies in an earlier layer). For S with lowest element j and
// S' = S \ {j}, c[S] = a[S] - sum_{U proper subset of S'} c[{j} u U] a[S' \ U].
// A group of g lanes (g = 2^r chosen per layer by a cost model) shares one S:
// lane t fixes the lowest r elements of S' to the bits of t and walks the
// submasks of the rest; the group sum is reduced with warp shuffles.
#include <cuda_runtime.h>
#include <stdint.h>

#include "apm_internal.cuh"

namespace apm {

constexpr int kBlkB = 10;  // low elements per block of the blocked recursion (orders above 12)

__device__ uint16_t g_popmasks[1 << 16];  // masks < 2^16 ordered by (popcount, value)
__device__ int g_popoff[18];              // first index of each popcount class
__constant__ int c_binom[17][17];

struct __align__(16) CdetSmemHdr {
    double log_p[kCorrCap];  // the unshifted pivot (C = sign(p) shift)
    int log_x[kCorrCap];
    int log_l[kCorrCap];
    double red[kCdetThreads / 32];
    unsigned long long red_u[kCdetThreads / 32];
    int ncorr;
    int flags;
    double anorm;
};

// doubles of global scratch per CTA slot: MA, MC, MU
__host__ __device__ inline size_t slot_doubles(int n) {
    const size_t N = size_t(1) << n;
    return 2 * N + (N > 16 ? N : 16);
}

struct CdetKernelParams {
    CdetArgs a;
    unsigned long long gsel;    // 3 bits per popcount layer k: log2 of the lane-group size
    unsigned long long gsel_b;  // the same for blocks of kBlkB elements (orders above 12)
};

struct VarlenParams {
    CdetArgs a;                    // batch, mode, flags, base pointers, gscratch
    const int64_t *a_off;          // element offset of each input matrix
    const int *n_arr;              // order of each matrix
    const int64_t *c_off;          // element offset of each output row (2^n entries)
    const int *order;              // processing order (longest first)
    unsigned *ctr;                 // work counter, zeroed by varlen_order_kernel
    int smem_max_n;
    int n_max;
    unsigned long long gsel[17];   // lane-group table per order
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bulk (TMA engine) copy of `bytes` from shared to global memory; issued by one
// thread after a CTA barrier that ordered the shared-memory writes.
__device__ __forceinline__ void bulk_store(double *gdst, const double *ssrc, uint32_t bytes) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                 "r"(smem_u32(ssrc)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read() {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------

// max |A_ij| and finiteness of one n x n matrix, on integer bit patterns (the
// magnitude order of finite doubles is the order of their bits without sign).
// over (if not NULL): the scale to use instead of the matrix's own max (a leaf
// of a larger matrix takes that matrix's ||A||max).
__device__ __forceinline__ void matrix_norm(const double *__restrict__ Ag, int n, CdetSmemHdr &h,
                                            const double *over) {
    const int tid = threadIdx.x;
    unsigned long long mx = 0ull;
    int bad = 0;
    for (int i = tid; i < n * n; i += blockDim.x) {
        unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(__ldg(Ag + i)));
        u &= 0x7fffffffffffffffull;
        if (u >= 0x7ff0000000000000ull) bad = 1;
        else if (u > mx) mx = u;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long v = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = v > mx ? v : mx;
    }
    bad = __any_sync(0xffffffffu, bad);
    if ((tid & 31) == 0) {
        h.red_u[tid >> 5] = mx;
        if (bad) atomicOr(&h.flags, APM_ST_NONFINITE_INPUT);
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long m = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = h.red_u[w] > m ? h.red_u[w] : m;
        double an = over ? *over : __longlong_as_double(static_cast<long long>(m));
        h.anorm = an > 0.0 ? an : 1.0;
    }
    __syncthreads();
}

// Node bookkeeping when a BFS-level matrix's (1,1) entry v is final: store the
// node's minor det[x | {lev}] = det[x] * p (Eq. minor), correct p if it is
// tiny, and replace v by 1/p for the Schur step of the next level.
__device__ __forceinline__ void node_pivot(int x, int lev, double &v, double *MA, double thr,
                                           double shift, CdetSmemHdr &h) {
    double piv = v;
    if (fabs(piv) <= thr) {
        const int slot = atomicAdd(&h.ncorr, 1);
        if (slot < kCorrCap) {
            h.log_x[slot] = x;
            h.log_l[slot] = lev;
            h.log_p[slot] = piv;
        }
        piv += piv >= 0.0 ? shift : -shift;
    }
    MA[x | (1 << lev)] = MA[x] * piv;
    v = 1.0 / piv;
}

// All 15 principal minors of a 4x4 matrix w (row-major) times `pre`, written to
// MA[m | X << L] for X = 1 .. 2^s - 1 (s = min(n,4)); closed-form cofactor and
// Laplace expansions, no division.
__device__ __forceinline__ void bottom4(const double *__restrict__ w, double pre, double *MA, int m,
                                        int L, int s) {
    const double a = w[0], b = w[1], c = w[2], d = w[3];
    const double e = w[4], f = w[5], g = w[6], hh = w[7];
    const double i = w[8], j = w[9], k = w[10], l = w[11];
    const double mm = w[12], nn = w[13], o = w[14], p = w[15];
    // 2x2 principal
    const double d01 = fma(a, f, -b * e);
    const double d02 = fma(a, k, -c * i);
    const double d03 = fma(a, p, -d * mm);
    const double d12 = fma(f, k, -g * j);
    const double d13 = fma(f, p, -hh * nn);
    const double d23 = fma(k, p, -l * o);
    // off-principal 2x2 minors used by the 3x3 and 4x4 expansions
    const double ek_gi = fma(e, k, -g * i);
    const double ej_fi = fma(e, j, -f * i);
    const double ep_hm = fma(e, p, -hh * mm);
    const double en_fm = fma(e, nn, -f * mm);
    const double ip_lm = fma(i, p, -l * mm);
    const double io_km = fma(i, o, -k * mm);
    const double jp_ln = fma(j, p, -l * nn);
    const double jo_kn = fma(j, o, -k * nn);
    // 3x3 principal (cofactor expansion along the first row of each subset)
    const double d012 = fma(a, d12, fma(-b, ek_gi, c * ej_fi));
    const double d013 = fma(a, d13, fma(-b, ep_hm, d * en_fm));
    const double d023 = fma(a, d23, fma(-c, ip_lm, d * io_km));
    const double d123 = fma(f, d23, fma(-g, jp_ln, hh * jo_kn));
    // 4x4 by Laplace expansion along rows 0,1
    const double s02 = fma(a, g, -c * e);
    const double s03 = fma(a, hh, -d * e);
    const double s12 = fma(b, g, -c * f);
    const double s13 = fma(b, hh, -d * f);
    const double s23 = fma(c, hh, -d * g);
    const double c01 = fma(i, nn, -j * mm);
    double d0123 = d01 * d23;
    d0123 = fma(-s02, jp_ln, d0123);
    d0123 = fma(s03, jo_kn, d0123);
    d0123 = fma(s12, ip_lm, d0123);
    d0123 = fma(-s13, io_km, d0123);
    d0123 = fma(s23, c01, d0123);
    MA[m | (1 << L)] = pre * a;
    if (s < 2) return;
    MA[m | (2 << L)] = pre * f;
    MA[m | (3 << L)] = pre * d01;
    if (s < 3) return;
    MA[m | (4 << L)] = pre * k;
    MA[m | (5 << L)] = pre * d02;
    MA[m | (6 << L)] = pre * d12;
    MA[m | (7 << L)] = pre * d012;
    if (s < 4) return;
    MA[m | (8 << L)] = pre * p;
    MA[m | (9 << L)] = pre * d03;
    MA[m | (10 << L)] = pre * d13;
    MA[m | (11 << L)] = pre * d013;
    MA[m | (12 << L)] = pre * d23;
    MA[m | (13 << L)] = pre * d023;
    MA[m | (14 << L)] = pre * d123;
    MA[m | (15 << L)] = pre * d0123;
}

// The 7 principal minors other than the empty one of a 3 x 3 node C (row-major
// stride 4 from c) with node minor d, written to MA[base | X << sh] for
// X = 1..7: row 0 scaled by d first, the 2 x 2 minors directly, the whole by
// expansion along row 0 (no division).
__device__ __forceinline__ void cf3_store(const double *c, int st, double d, double *MA, int base, int sh) {
    const double c00 = c[0], c01 = c[1], c02 = c[2];
    const double c10 = c[st], c11 = c[st + 1], c12 = c[st + 2];
    const double c20 = c[2 * st], c21 = c[2 * st + 1], c22 = c[2 * st + 2];
    const double a0 = d * c00, a1 = d * c01, a2 = d * c02;
    const double m12 = fma(c11, c22, -c12 * c21);
    const double m02 = fma(c10, c22, -c12 * c20);
    const double m01 = fma(c10, c21, -c11 * c20);
    MA[base | (1 << sh)] = a0;
    MA[base | (2 << sh)] = d * c11;
    MA[base | (3 << sh)] = fma(a0, c11, -a1 * c10);
    MA[base | (4 << sh)] = d * c22;
    MA[base | (5 << sh)] = fma(a0, c22, -a2 * c20);
    MA[base | (6 << sh)] = d * m12;
    MA[base | (7 << sh)] = fma(a0, m12, fma(-a1, m02, a2 * m01));
}

// The 15 principal minors of a 4x4 node w (elements L..L+3, node minor MA[m])
// by one Schur step on its first element, a pivot of the tree, and the closed
// forms of the two 3x3 children. A tiny pivot p is shifted by C as on the
// other levels, but its correction is finished here: the node's right subtree
// is the 7 minors of its kept child, all in this thread, and this is the
// deepest level with pivots, so det[m] = det~[m] - C det[m without element L]
// is applied at once (before the logged corrections of the shallower levels),
// and the node's own minor is written with the unshifted pivot. No log entry.
__device__ __forceinline__ void bottom43(const double *__restrict__ w, double *MA, int m, int L, double thr,
                                         double shift, CdetSmemHdr &h) {
    const double p = w[0], d = MA[m];
    const bool corr = fabs(p) <= thr;
    const double C = corr ? (p >= 0.0 ? shift : -shift) : 0.0;
    const double piv = p + C;
    const double v = 1.0 / piv;
    const int mk = m | (1 << L);
    MA[mk] = d * p;
    const double g1 = w[4] * v, g2 = w[8] * v, g3 = w[12] * v;
    double S[9];
    S[0] = fma(-g1, w[1], w[5]);
    S[1] = fma(-g1, w[2], w[6]);
    S[2] = fma(-g1, w[3], w[7]);
    S[3] = fma(-g2, w[1], w[9]);
    S[4] = fma(-g2, w[2], w[10]);
    S[5] = fma(-g2, w[3], w[11]);
    S[6] = fma(-g3, w[1], w[13]);
    S[7] = fma(-g3, w[2], w[14]);
    S[8] = fma(-g3, w[3], w[15]);
    cf3_store(w + 5, 4, d, MA, m, L + 1);      // element L dropped
    cf3_store(S, 3, d * piv, MA, mk, L + 1);   // element L kept (shifted minor when corrected)
    if (corr) {
#pragma unroll
        for (int X = 1; X < 8; ++X) MA[mk | (X << (L + 1))] = fma(-C, MA[m | (X << (L + 1))], MA[mk | (X << (L + 1))]);
        atomicOr(&h.flags, APM_ST_PIVOT_CORRECTED);
    }
}

// All principal minors of the n x n matrix Ag, times root (the minor of the
// empty set), into MA[0 .. 2^n), MC as scratch.
__device__ __forceinline__ void fpm_tree(const double *__restrict__ Ag, int n, double *MA, double *MC, double thr,
                         double shift, CdetSmemHdr &h, double root = 1.0) {
    const int tid = threadIdx.x, T = blockDim.x;
    const int L = n > 4 ? n - 4 : 0;
    double *const bufA = MA + (1 << L);
    // level-l buffer: MC when L-l is even, else the upper part of MA
#define APM_BUF(lv) ((((L) - (lv)) & 1) ? bufA : MC)
    double *W0 = APM_BUF(0);
    if (n >= 4) {
        for (int t = tid; t < n * n; t += T) W0[t] = __ldg(Ag + t);
    } else {
        for (int t = tid; t < 16; t += T) {
            const int r = t >> 2, q = t & 3;
            W0[t] = (r < n && q < n) ? __ldg(Ag + r * n + q) : (r == q ? 1.0 : 0.0);
        }
    }
    if (tid == 0) MA[0] = root;
    __syncthreads();
    for (int l = 0; l < L; ++l) {
        const int s = n - l, s1 = s - 1, ss = s * s, ss1 = s1 * s1, P = 1 << l;
        double *Wl = APM_BUF(l);
        double *Wn = APM_BUF(l + 1);
        // one thread per node: the node's minor and pivot (the division runs
        // with a lane per node, not one lane of a warp busy with Schur entries),
        // then its pivot row scaled by 1/p; row 0 is not part of the left child,
        // so it can be scaled in place (Wl[0] keeps 1/p)
        for (int m = tid; m < P; m += T) {
            double *Wm = Wl + m * ss;
            double v = Wm[0];
            node_pivot(m, l, v, MA, thr, shift, h);
            Wm[0] = v;
        }
        __syncthreads();
        // the pivot rows scaled by 1/p, one entry per thread step
        for (int e = tid; e < P * s1; e += T) {
            const int m = e / s1, q = e - m * s1 + 1;
            Wl[m * ss + q] *= Wl[m * ss];
        }
        __syncthreads();
        const int E = 2 * P * ss1;
        for (int e = tid; e < E; e += T) {
            const int x = e / ss1;
            const int rem = e - x * ss1;
            const int p = rem / s1;
            const int q = rem - p * s1;
            const double *Wp = Wl + (x & (P - 1)) * ss;
            double v = Wp[(p + 1) * s + q + 1];
            if (x >> l)  // right child: Schur complement w.r.t. the pivot
                v = fma(-Wp[(p + 1) * s], Wp[q + 1], v);
            Wn[x * ss1 + rem] = v;
        }
        __syncthreads();
    }
    const double *WL = APM_BUF(L);
#undef APM_BUF
    if (n >= 4) {
        for (int m = tid; m < (1 << L); m += T) bottom43(WL + m * 16, MA, m, L, thr, shift, h);
    } else {
        const int s = n;
        for (int m = tid; m < (1 << L); m += T) bottom4(WL + m * 16, MA[m], MA, m, L, s);
    }
    __syncthreads();
    // back-propagation of pivot corrections, deepest level first (the log is in
    // non-decreasing level order: each level's pivots are logged in its own
    // pivot phase, after a barrier that ends the previous level)
    const int nc = h.ncorr;
    if (nc > kCorrCap) {
        for (int t = tid; t < (1 << n); t += T) MA[t] = __longlong_as_double(0x7ff8000000000000ll);
        if (tid == 0) h.flags |= APM_ST_CORRECTION_OVERFLOW;
        __syncthreads();
        return;
    }
    for (int ci = nc - 1; ci >= 0; --ci) {
        const int x = h.log_x[ci], lv = h.log_l[ci];
        const double pv = h.log_p[ci];
        const double cs = pv >= 0.0 ? shift : -shift;
        const int cnt = 1 << (n - lv - 1);
        for (int t = tid; t < cnt; t += T) {
            const int src = x | (t << (lv + 1));
            const int tgt = src | (1 << lv);
            MA[tgt] = t == 0 ? MA[src] * pv : fma(-cs, MA[src], MA[tgt]);
        }
        __syncthreads();
    }
    if (nc > 0 && tid == 0) h.flags |= APM_ST_PIVOT_CORRECTED;
}

// Connected sums c[S] = init[S] - sum_{U proper subset of S'} c[{j} u U] a[S' \ U]
// (init = a for the plain recursion) for all masks of n elements.
__device__ __forceinline__ void cdet_layers(const double *init, const double *a, double *c, int n,
                                            unsigned long long gsel) {
    const int tid = threadIdx.x, T = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    for (int t = tid; t < (1 << n); t += T) c[t] = 0.0;
    __syncthreads();
    for (int x = tid; x < n; x += T) c[1 << x] = init[1 << x];
    __syncthreads();
    for (int k = 2; k <= n; ++k) {
        const int cnt = c_binom[n][k];
        const uint16_t *masks = g_popmasks + g_popoff[k];
        const int r = static_cast<int>((gsel >> (3 * k)) & 7ull);
        const int spw = 32 >> r;  // sets per warp step
        const int gl = lane & ((1 << r) - 1);
        for (int base = warp * spw; base < cnt; base += nw * spw) {
            const int G = base + (lane >> r);
            const bool act = G < cnt;
            const int S = masks[act ? G : cnt - 1];
            const int j = S & (-S);
            const int Sp = S ^ j;
            int UL = 0, low = 0, tmp = Sp;
            for (int i = 0; i < r; ++i) {
                const int bt = tmp & (-tmp);
                tmp ^= bt;
                low |= bt;
                if ((gl >> i) & 1) UL |= bt;
            }
            const int H = Sp ^ low;
            // c[S] itself (U = Sp) is still 0 here (c[] of this layer is zeroed
            // before the layer), so the term U = Sp adds exactly 0 and needs no test
            double acc = 0.0;
            int UH = H;
            while (true) {
                const int U = UL | UH;
                acc = fma(c[j | U], a[Sp ^ U], acc);
                if (UH == 0) break;
                UH = (UH - 1) & H;
            }
            for (int o = (1 << r) >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (act && gl == 0) c[S] = init[S] - acc;
        }
        __syncthreads();
    }
}

// acc[S] += sum over all U subset of S' of cb[{j} u U] ab[S' \ U] for every
// nonempty mask S of b elements (j = lowest element of S, S' = S \ {j}): the
// contribution of one off-diagonal block pair of the blocked recursion. All
// masks are independent; lane groups as in cdet_layers.
__device__ __forceinline__ void block_conv(const double *cb, const double *ab, double *acc, int b,
                                           unsigned long long gsel) {
    const int tid = threadIdx.x, T = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = T >> 5;
    for (int k = 1; k <= b; ++k) {
        const int cnt = c_binom[b][k];
        const uint16_t *masks = g_popmasks + g_popoff[k];
        const int r = static_cast<int>((gsel >> (3 * k)) & 7ull);
        const int spw = 32 >> r;
        const int gl = lane & ((1 << r) - 1);
        for (int base = warp * spw; base < cnt; base += nw * spw) {
            const int G = base + (lane >> r);
            const bool act = G < cnt;
            const int S = masks[act ? G : cnt - 1];
            const int j = S & (-S);
            const int Sp = S ^ j;
            int UL = 0, low = 0, tmp = Sp;
            for (int i = 0; i < r; ++i) {
                const int bt = tmp & (-tmp);
                tmp ^= bt;
                low |= bt;
                if ((gl >> i) & 1) UL |= bt;
            }
            const int H = Sp ^ low;
            double sum = 0.0;
            int UH = H;
            while (true) {
                const int U = UL | UH;
                sum = fma(cb[j | U], ab[Sp ^ U], sum);
                if (UH == 0) break;
                UH = (UH - 1) & H;
            }
            for (int o = (1 << r) >> 1; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (act && gl == 0) acc[S] += sum;
        }
    }
}

// Connected sums for n > kBlkB, blocked over the lowest kBlkB elements:
// S = S_H u S_L. For each S_H (increasing), every proper T_H of S_H contributes
// the block convolution of c[T_H u .] with a[(S_H \ T_H) u .] (with j in the
// low part, T_L = S_L allowed), the S_L = {} entry only when the lowest element
// of S_H lies in T_H; then the diagonal block solves its own recursion with
// init a[S_H u S_L] - acc[S_L] and the pure-low block a[0 u .]. a (global) and
// c (global output row) are read block-wise into shared memory (blk: 6 x 2^kBlkB)
// by asynchronous 16-byte copies (both rows and every block are 16-byte aligned).
__device__ void cdet_blocked(const double *a, double *c, int n, double *blk, unsigned long long gsel_b) {
    const int tid = threadIdx.x, T = blockDim.x;
    const int b = kBlkB, NB = 1 << kBlkB, h = n - b;
    double *cb = blk, *ab = blk + NB, *acc = blk + 2 * NB, *cs = blk + 3 * NB, *as = blk + 4 * NB,
           *a0 = blk + 5 * NB;
    for (int t = tid; t < NB / 2; t += T) cp_async16(a0 + 2 * t, a + 2 * t);
    for (int SH = 0; SH < (1 << h); ++SH) {
        const double *aS = a + (static_cast<size_t>(SH) << b);
        for (int t = tid; t < NB / 2; t += T) cp_async16(as + 2 * t, aS + 2 * t);
        for (int t = tid; t < NB; t += T) acc[t] = 0.0;
        const int jH = SH & (-SH);
        cp_async_wait_all();
        __syncthreads();
        if (SH) {
            for (int TH = (SH - 1) & SH;; TH = (TH - 1) & SH) {
                const double *cT = c + (static_cast<size_t>(TH) << b), *aR = a + (static_cast<size_t>(SH ^ TH) << b);
                for (int t = tid; t < NB / 2; t += T) {
                    cp_async16(cb + 2 * t, cT + 2 * t);
                    cp_async16(ab + 2 * t, aR + 2 * t);
                }
                cp_async_wait_all();
                __syncthreads();
                block_conv(cb, ab, acc, b, gsel_b);
                if (tid == 0 && (TH & jH)) acc[0] = fma(cb[0], ab[0], acc[0]);
                __syncthreads();
                if (TH == 0) break;
            }
        }
        for (int t = tid; t < NB; t += T) as[t] -= acc[t];
        __syncthreads();
        cdet_layers(as, a0, cs, b, gsel_b);
        for (int t = tid; t < NB; t += T)
            c[(static_cast<size_t>(SH) << b) + t] = (t == 0) ? (SH ? as[0] : 0.0) : cs[t];
        __syncthreads();
    }
}

// One matrix: minors (and optionally the connected sums) into the output rows.
// MA/MC/MU are on chip (in_smem) or in the CTA's global scratch slot. given:
// the warp-per-matrix minors kernel has already left this matrix's minors in
// mo (in co when mo is NULL) and its status; only the weights and the
// connected sums remain.
__device__ __forceinline__ void cdet_item(const CdetArgs &p, int n, const double *Au, const double *Ad,
                                          const double *ain, double *mo, double *co, uint32_t *st,
                                          double *MA, double *MC, double *MU, bool in_smem,
                                          unsigned long long gsel, unsigned long long gsel_b, double *blk,
                                          CdetSmemHdr &h, const double *anorm_over, double root,
                                          bool given = false) {
    const int tid = threadIdx.x;
    const int N = 1 << n;
    if (tid == 0) bulk_wait_read();  // the previous item's bulk stores have read their source
    if (tid == 0) {
        h.ncorr = 0;
        h.flags = 0;
    }
    __syncthreads();
    if (p.mode == kModeWeights) {
        for (int t = tid; t < N; t += blockDim.x) MA[t] = __ldg(ain + t);
        __syncthreads();
    } else if (given) {
        // the weights from the given minors (one matrix: det^2, or det)
        const double *src = mo ? mo : co;
        for (int t = tid; t < N; t += blockDim.x) {
            const double m = src[t];
            MA[t] = p.single_det ? m : m * m;
        }
        __syncthreads();
    } else {
        if (p.two_mats) {
            matrix_norm(Ad, n, h, anorm_over);
            fpm_tree(Ad, n, MA, MC, p.piv_thr * h.anorm, p.piv_shift * h.anorm, h);
            for (int t = tid; t < N; t += blockDim.x) MU[t] = MA[t];
            if (tid == 0) h.ncorr = 0;
            __syncthreads();
        }
        matrix_norm(Au, n, h, anorm_over);
        fpm_tree(Au, n, MA, MC, p.piv_thr * h.anorm, p.piv_shift * h.anorm, h, root);
        if (mo) {
            if (in_smem) {
                if (tid == 0) {
                    bulk_store(mo, MA, N * 8u);
                    if (p.two_mats) bulk_store(mo + N, MU, N * 8u);
                    bulk_wait_read();
                }
            } else {
                for (int t = tid; t < N; t += blockDim.x) {
                    mo[t] = MA[t];
                    if (p.two_mats) mo[N + t] = MU[t];
                }
            }
        }
        if (tid == 0 && st) *st = static_cast<uint32_t>(h.flags);
        __syncthreads();
        if (p.mode == kModeMinors) return;
        if (!p.single_det) {
            if (p.two_mats)
                for (int t = tid; t < N; t += blockDim.x) MA[t] *= MU[t];
            else
                for (int t = tid; t < N; t += blockDim.x) MA[t] *= MA[t];
        }
        __syncthreads();
    }
    if (in_smem) {
        cdet_layers(MA, MA, MC, n, gsel);
        if (tid == 0) bulk_store(co, MC, N * 8u);
    } else if (p.fsc_from_n && n >= p.fsc_from_n) {
        // the weights go to the output row; the fast subset convolution that
        // follows in its own launch turns them into the connected sums in place
        for (int t = tid; t < N; t += blockDim.x) co[t] = MA[t];
    } else {
        cdet_blocked(MA, co, n, blk, gsel_b);
    }
    // the next item's first barrier orders these reads before any overwrite
}

template <bool kSmemArrays>
__global__ void __launch_bounds__(kCdetThreads, 3) fpm_cdet_kernel(const CdetKernelParams P) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    CdetSmemHdr &h = *reinterpret_cast<CdetSmemHdr *>(smem_raw);
    const CdetArgs &p = P.a;
    const int n = p.n;
    const int N = 1 << n;
    const int NC = N > 16 ? N : 16;
    double *const sbase = reinterpret_cast<double *>(smem_raw + ((sizeof(CdetSmemHdr) + 127) & ~size_t(127)));
    double *base;
    if (kSmemArrays)
        base = sbase;
    else
        base = p.gscratch + static_cast<size_t>(blockIdx.x) * slot_doubles(n);
    double *MA = base;
    double *MC = base + N;
    double *MU = MC + NC;
    const int64_t mat = static_cast<int64_t>(n) * n;
    auto item = [&](int64_t b) {
        cdet_item(p, n, p.A_up ? p.A_up + b * mat : nullptr, p.A_dn ? p.A_dn + b * mat : nullptr,
                  p.a_in ? p.a_in + b * N : nullptr,
                  p.minors_out ? p.minors_out + b * (p.two_mats ? 2 * N : N) : nullptr,
                  p.c_out ? p.c_out + b * N : nullptr, p.status ? p.status + b : nullptr, MA, MC, MU,
                  kSmemArrays, P.gsel, P.gsel_b, sbase, h, p.anorm_in ? p.anorm_in + (b >> p.anorm_shift) : nullptr,
                  p.pre ? p.pre[b] : 1.0, p.wflag && n >= p.warp_from_n && !p.wflag[b]);
    };
    if (p.redo_list) {
        // only the matrices the warp-per-matrix minors kernel flagged (usually none)
        const int64_t cnt = *p.redo_count < p.batch ? static_cast<int64_t>(*p.redo_count) : p.batch;
        for (int64_t i = blockIdx.x; i < cnt; i += gridDim.x) item(p.redo_list[i]);
    } else {
        for (int64_t b = blockIdx.x; b < p.batch; b += gridDim.x) item(b);
    }
    if (threadIdx.x == 0) bulk_wait_all();
}

// Uneven batch: items taken longest-first from `order` through a global
// counter; arrays on chip for n <= smem_max_n, else in the CTA's scratch slot.
__global__ void __launch_bounds__(kCdetThreads, 3) fpm_cdet_varlen_kernel(const VarlenParams V) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    CdetSmemHdr &h = *reinterpret_cast<CdetSmemHdr *>(smem_raw);
    __shared__ unsigned long long gsel_s[17];
    __shared__ int item_s;
    const CdetArgs &p = V.a;
    if (threadIdx.x < 17) gsel_s[threadIdx.x] = V.gsel[threadIdx.x];
    double *const sbase = reinterpret_cast<double *>(smem_raw + ((sizeof(CdetSmemHdr) + 127) & ~size_t(127)));
    double *const gbase = p.gscratch ? p.gscratch + static_cast<size_t>(blockIdx.x) * slot_doubles(V.n_max) : nullptr;
    while (true) {
        __syncthreads();  // gsel_s ready; item_s free for reuse
        if (threadIdx.x == 0) item_s = static_cast<int>(atomicAdd(V.ctr, 1u));
        __syncthreads();
        const int item = item_s;
        if (item >= p.batch) break;
        const int b = V.order[item];
        const int n = V.n_arr[b];
        if (n < 1 || n > V.n_max) {
            if (threadIdx.x == 0 && p.status) p.status[b] = APM_ST_BAD_ORDER;
            continue;
        }
        const int N = 1 << n;
        const int NC = N > 16 ? N : 16;
        const bool in_smem = n <= V.smem_max_n;
        double *MA = in_smem ? sbase : gbase;
        double *MC = MA + N;
        double *MU = MC + NC;
        const int64_t ao = V.a_off[b], co = V.c_off[b];
        cdet_item(p, n, p.A_up ? p.A_up + ao : nullptr, p.A_dn ? p.A_dn + ao : nullptr,
                  p.a_in ? p.a_in + co : nullptr,
                  p.minors_out ? p.minors_out + (p.two_mats ? 2 * co : co) : nullptr,
                  p.c_out ? p.c_out + co : nullptr, p.status ? p.status + b : nullptr, MA, MC, MU, in_smem,
                  gsel_s[n], gsel_s[kBlkB], sbase, h, nullptr, 1.0,
                  p.wflag && p.warp_from_n && n >= p.warp_from_n && !p.wflag[b]);
    }
    if (threadIdx.x == 0) bulk_wait_all();
}

// Longest-first order of an uneven batch: counting sort by decreasing order n
// (one CTA), and reset of the work counter of the consumer kernel; per order m
// the first index and the count of its items (ctr[2 + 2m], ctr[3 + 2m]).
__global__ void __launch_bounds__(1024) varlen_order_kernel(const int *__restrict__ n_arr, int64_t batch,
                                                            int n_max, int *order, unsigned *ctr, int fsc_from_n) {
    __shared__ int hist[18];
    __shared__ int start[18];
    if (threadIdx.x < 18) hist[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t b = threadIdx.x; b < batch; b += blockDim.x) {
        int n = n_arr[b];
        n = (n < 1 || n > n_max) ? 0 : n;  // invalid orders go last (bucket 0)
        atomicAdd(&hist[n], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int pos = 0;
        for (int n = 17; n >= 0; --n) {
            start[n] = pos;
            pos += hist[n];
        }
        ctr[0] = 0u;
        // items of the orders that take the fast subset convolution: the first
        // ones of the longest-first order
        int nf = 0;
        for (int n = fsc_from_n; n <= 16; ++n) nf += hist[n];
        ctr[1] = static_cast<unsigned>(nf);
        for (int n = 0; n <= 16; ++n) {
            ctr[2 + 2 * n] = static_cast<unsigned>(start[n]);
            ctr[3 + 2 * n] = static_cast<unsigned>(hist[n]);
        }
    }
    __syncthreads();
    for (int64_t b = threadIdx.x; b < batch; b += blockDim.x) {
        int n = n_arr[b];
        n = (n < 1 || n > n_max) ? 0 : n;
        const int slot = atomicAdd(&start[n], 1);
        order[slot] = static_cast<int>(b);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static inline size_t hdr_bytes() { return (sizeof(CdetSmemHdr) + 127) & ~size_t(127); }

size_t cdet_slot_doubles(int n) { return slot_doubles(n); }

size_t cdet_smem_bytes(int n, bool two_mats, bool smem_arrays) {
    if (!smem_arrays) return hdr_bytes() + 6 * sizeof(double) * (size_t(1) << kBlkB);
    const size_t N = size_t(1) << n;
    return hdr_bytes() + 8 * ((two_mats ? 2 : 1) * N + (N > 16 ? N : 16));
}

int cdet_smem_max_n(bool two_mats) {
    (void)two_mats;
    return 12;  // above: a[] and c[] in global memory, recursion blocked through shared memory
}

void cdet_group_table(int n, int threads, uint8_t *gsel) {
    // Per popcount layer k: choose the group size g = 2^r lanes per set that
    // minimises the FP64 warp-instructions of the layer,
    //   ceil(C(n,k) g / 32) * (2^{k-1-r} + r + 1),
    // breaking near-ties (within 3%) toward larger groups, whose lanes read
    // neighbouring subsets (fewer shared-memory bank conflicts).
    (void)threads;
    for (int k = 0; k <= 16; ++k) gsel[k] = 0;
    double binom[17][17] = {};
    for (int a = 0; a <= 16; ++a) {
        binom[a][0] = 1;
        for (int b = 1; b <= a; ++b) binom[a][b] = binom[a - 1][b - 1] + (b <= a - 1 ? binom[a - 1][b] : 0);
    }
    for (int k = 2; k <= n; ++k) {
        const double cnt = binom[n][k];
        double best = 1e300;
        int rb = 0;
        double cost[6];
        const int rmax = (k - 1) < 5 ? (k - 1) : 5;
        for (int r = 0; r <= rmax; ++r) {
            const double tasks = ceil(cnt * double(1 << r) / 32.0);
            cost[r] = tasks * (double(1 << (k - 1 - r)) + r + 1);
            if (cost[r] < best) { best = cost[r]; rb = r; }
        }
        for (int r = rmax; r > rb; --r)
            if (cost[r] <= best * 1.03) { rb = r; break; }
        gsel[k] = static_cast<uint8_t>(rb);
    }
}

// Lane-group tables installed by apm_cdet_tune_set (0 = use the cost model).
static unsigned long long g_tuned[17] = {};
// Knobs installed by apm_tune_options_set: the order from which the connected
// sums take the fast subset convolution, and the persistent CTAs per SM of the
// uneven batch (0: as many as fit).
static int g_fsc_from_n = kFscFromN;
static int g_varlen_ctas = 0;

int cdet_fsc_from_n() { return g_fsc_from_n; }
int cdet_varlen_ctas_per_sm() { return g_varlen_ctas; }
void cdet_tune_options_set(int fsc_from_n, int cdet_ctas_per_sm) {
    g_fsc_from_n = fsc_from_n;
    g_varlen_ctas = cdet_ctas_per_sm;
}

unsigned long long cdet_gsel_packed(int n) {
    if (n >= 0 && n <= 16 && g_tuned[n]) return g_tuned[n];
    uint8_t gsel[17];
    cdet_group_table(n, kCdetThreads, gsel);
    unsigned long long packed = 0ull;
    for (int k = 0; k <= 16; ++k) packed |= static_cast<unsigned long long>(gsel[k] & 7) << (3 * k);
    return packed;
}

void cdet_tune_set(const unsigned long long *table) {
    for (int n = 0; n <= 16; ++n) g_tuned[n] = table ? table[n] : 0ull;
}

int cdet_grid(int n, int64_t batch, bool two_mats, bool smem_arrays, int *err) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = cdet_smem_bytes(n, two_mats, smem_arrays);
    if (e == cudaSuccess) {
        if (smem_arrays) {
            e = cudaFuncSetAttribute(fpm_cdet_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem));
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fpm_cdet_kernel<true>,
                                                                  kCdetThreads, smem);
        } else {
            e = cudaFuncSetAttribute(fpm_cdet_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(smem));
            if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fpm_cdet_kernel<false>,
                                                                  kCdetThreads, smem);
        }
    }
    if (e != cudaSuccess || per_sm < 1) {
        if (err) *err = e != cudaSuccess ? static_cast<int>(e) : static_cast<int>(cudaErrorInvalidConfiguration);
        return 0;
    }
    if (err) *err = 0;
    int64_t g = static_cast<int64_t>(sms) * per_sm;
    if (batch < g) g = batch;
    return static_cast<int>(g < 1 ? 1 : g);
}

int ensure_tables() {
    static int done_mask = 0;  // bit per device id < 32
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 32 && (done_mask >> dev) & 1) return 0;
    static uint16_t masks[1 << 16];
    int off[18];
    int pos = 0;
    for (int k = 0; k <= 16; ++k) {
        off[k] = pos;
        for (int S = 0; S < (1 << 16); ++S)
            if (__builtin_popcount(static_cast<unsigned>(S)) == k) masks[pos++] = static_cast<uint16_t>(S);
    }
    off[17] = pos;
    int binom[17][17] = {};
    for (int a = 0; a <= 16; ++a) {
        binom[a][0] = 1;
        for (int b = 1; b <= a; ++b) binom[a][b] = binom[a - 1][b - 1] + (b <= a - 1 ? binom[a - 1][b] : 0);
    }
    e = cudaMemcpyToSymbol(g_popmasks, masks, sizeof(masks));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_popoff, off, sizeof(off));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_binom, binom, sizeof(binom));
    if (e != cudaSuccess) return e;
    if (dev < 32) done_mask |= 1 << dev;
    return 0;
}

int launch_fpm_cdet(const CdetArgs &a, cudaStream_t s) {
    int err = ensure_tables();
    if (err) return err;
    CdetKernelParams P;
    P.a = a;
    P.gsel = cdet_gsel_packed(a.n);
    P.gsel_b = cdet_gsel_packed(kBlkB);
    const bool smem_arrays = a.n <= cdet_smem_max_n(a.two_mats != 0);
    const int grid = cdet_grid(a.n, a.batch, a.two_mats != 0, smem_arrays, &err);
    if (err) return err;
    const size_t smem = cdet_smem_bytes(a.n, a.two_mats != 0, smem_arrays);
    const bool fsc = a.mode == kModeCdet && a.n >= g_fsc_from_n;
    P.a.fsc_from_n = fsc ? g_fsc_from_n : 0;
    if (a.wflag && a.warp_from_n && a.n >= a.warp_from_n) {
        // the minors first, one warp per matrix (its stack in the slots' region,
        // which the fused kernel takes over after it)
        err = launch_fpm_warp_route(a.A_up, a.n, a.batch, a.minors_out ? a.minors_out : a.c_out, a.piv_thr,
                                    a.wflag, a.status, a.gscratch, nullptr, nullptr, nullptr, nullptr, nullptr, s);
        if (err) return err;
    }
    if (smem_arrays)
        fpm_cdet_kernel<true><<<grid, kCdetThreads, smem, s>>>(P);
    else
        fpm_cdet_kernel<false><<<grid, kCdetThreads, smem, s>>>(P);
    err = static_cast<int>(cudaGetLastError());
    if (err || !fsc) return err;
    // the workspace holds the fused kernel's slots, then the ranked arrays
    return launch_fsc(a.c_out, a.n, a.batch, a.c_out, a.gscratch, s);
}

// ---------------------------------------------------------------------------
// uneven batches
// ---------------------------------------------------------------------------

constexpr int kVarlenSmemMaxN = 12;

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

int cdet_varlen_grid(bool two_mats, int *err) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = cdet_smem_bytes(kVarlenSmemMaxN, two_mats, true);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fpm_cdet_varlen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(smem));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fpm_cdet_varlen_kernel, kCdetThreads, smem);
    if (e != cudaSuccess || per_sm < 1) {
        *err = e != cudaSuccess ? static_cast<int>(e) : static_cast<int>(cudaErrorInvalidConfiguration);
        return 0;
    }
    *err = 0;
    if (g_varlen_ctas > 0 && g_varlen_ctas < per_sm) per_sm = g_varlen_ctas;
    return sms * per_sm;
}

// Orders from which the connected-sum paths of one matrix per item take their
// minors from the warp-per-matrix kernel (0: never).
static int warp_route_from(int n_max, bool two_mats) {
    return !two_mats && n_max >= kWarpRouteFromN ? kWarpRouteFromN : 0;
}

// Workspace of an uneven batch: [counter 256 B][order: batch int32]
// [flags of the warp-kernel minors: batch bytes, with orders >= 13 of one
// matrix per item][per-CTA slots; the same region holds the warp kernel's
// stacks before and the ranked arrays after the persistent kernel]
size_t cdet_varlen_workspace(int n_max, int64_t batch, bool two_mats, int *err) {
    size_t bytes = 256 + align256(static_cast<size_t>(batch) * sizeof(int));
    if (n_max > kVarlenSmemMaxN) {
        const int grid = cdet_varlen_grid(two_mats, err);
        if (*err) return 0;
        size_t slots = static_cast<size_t>(grid) * slot_doubles(n_max) * sizeof(double);
        if (n_max >= g_fsc_from_n) {  // the same region then holds the ranked arrays
            const size_t f = fsc_workspace_bytes(n_max, batch, err);
            if (*err) return 0;
            if (f > slots) slots = f;
        }
        if (warp_route_from(n_max, two_mats)) {
            const size_t st = fpm_warp_route_stack_bytes(n_max, batch, err);
            if (*err) return 0;
            if (st > slots) slots = st;
            bytes += align256(static_cast<size_t>(batch));
        }
        bytes += slots;
    } else {
        *err = 0;
    }
    return bytes;
}

int launch_order(const int *n_arr, int64_t batch, int n_max, int *order, unsigned *ctr, cudaStream_t s,
                 int fsc_from_n) {
    varlen_order_kernel<<<1, 1024, 0, s>>>(n_arr, batch, n_max, order, ctr, fsc_from_n);
    return static_cast<int>(cudaGetLastError());
}

int launch_cdet_varlen(const CdetArgs &a, const int64_t *a_off, const int *n_arr, const int64_t *c_off,
                       int n_max, void *workspace, cudaStream_t s) {
    int err = ensure_tables();
    if (err) return err;
    const bool two = a.two_mats != 0;
    const int grid = cdet_varlen_grid(two, &err);
    if (err) return err;
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    unsigned *ctr = reinterpret_cast<unsigned *>(ws);
    int *order = reinterpret_cast<int *>(ws + 256);
    size_t off = 256 + align256(static_cast<size_t>(a.batch) * sizeof(int));
    const int wfrom = n_max > kVarlenSmemMaxN && a.mode == kModeCdet ? warp_route_from(n_max, two) : 0;
    uint8_t *wflag = wfrom ? ws + off : nullptr;
    if (wfrom) off += align256(static_cast<size_t>(a.batch));
    double *slots = reinterpret_cast<double *>(ws + off);
    const int fsc_from = g_fsc_from_n;
    err = launch_order(n_arr, a.batch, n_max, order, ctr, s, fsc_from);
    if (err) return err;
    // the minors of the items of orders >= wfrom, one launch per order from its
    // first index and count in the sorted list, one warp per matrix
    for (int m = n_max; wfrom && m >= wfrom && !err; --m)
        err = launch_fpm_warp_route(a.A_up, m, a.batch, a.minors_out ? a.minors_out : a.c_out, a.piv_thr, wflag,
                                    a.status, slots, order, a_off, c_off, ctr + 2 + 2 * m, ctr + 3 + 2 * m, s);
    if (err) return err;
    VarlenParams V;
    V.a = a;
    V.a.wflag = wflag;
    V.a.warp_from_n = wfrom;
    V.a.gscratch = n_max > kVarlenSmemMaxN ? slots : nullptr;
    V.a_off = a_off;
    V.n_arr = n_arr;
    V.c_off = c_off;
    V.order = order;
    V.ctr = ctr;
    V.smem_max_n = kVarlenSmemMaxN;
    V.n_max = n_max;
    for (int n = 0; n <= 16; ++n) V.gsel[n] = cdet_gsel_packed(n);
    const bool fsc = a.mode == kModeCdet && n_max >= fsc_from;
    V.a.fsc_from_n = fsc ? fsc_from : 0;
    const int64_t g = a.batch < grid ? a.batch : grid;
    fpm_cdet_varlen_kernel<<<static_cast<int>(g), kCdetThreads, cdet_smem_bytes(kVarlenSmemMaxN, two, true), s>>>(V);
    err = static_cast<int>(cudaGetLastError());
    if (err || !fsc) return err;
    // the items of the orders >= fsc_from (the longest-first prefix), one launch
    // per order from its first index and count as the order kernel left them,
    // in place on their output rows
    for (int m = n_max; m >= fsc_from && !err; --m)
        err = launch_fsc_items(a.c_out, c_off, order, ctr + 2 + 2 * m, ctr + 3 + 2 * m, a.batch, m, slots, s);
    return err;
}

}  // namespace apm
