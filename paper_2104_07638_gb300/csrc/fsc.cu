// Connected sums by the fast subset convolution, O(n^2 2^n) (FP64).
//
// Paper: Section V.A notes that the CDet recursion (Eq. recursion) is a subset
// convolution and can also be evaluated in O(n^2 2^n) with the fast subset
// convolution of Bjorklund, Husfeldt, Kaski and Koivisto. With a[{}] = 1 the
// recursion states a[S] = sum over the set partitions of S of the products of
// c over the blocks, i.e. a = exp(c) in the ring of set functions under subset
// convolution. The ranked zeta transform
//     Z_k(X) = sum_{S subset of X, |S| = k} a[S]          (Z_0 = 1)
// turns subset convolution into products of polynomials in one variable t per
// mask X (exact on the coefficient of t^|S| after the Mobius transform), so
//     L(X; t) = log Z(X; t)   (power series to degree n),
//     c[S] = sum_{X subset of S} (-1)^{|S \ X|} L_{|S|}(X).
// The logarithm comes from k Z_k = sum_{j=1..k} j L_j Z_{k-j}: with M_k = k L_k,
//     M_k = k Z_k - sum_{m=1..k-1} Z_m M_{k-m}.
//
// One CTA (256 threads) per matrix, persistent over the batch; the ranked
// arrays R[k][X] (k = 1..n) are transformed in tiles of 512 masks in shared
// memory. n <= 9 is one tile (init, zeta, logarithm, Mobius, read-out, all in
// shared memory). Above, the low 9 elements are handled inside a tile and the
// high h = n - 9 across tiles, through the CTA's slot of the workspace:
//   pass A  per high pattern X_H: rank init and zeta over the low elements,
//           only for the ranks |X_H| .. |X_H| + 9 (no other rank can be
//           nonzero after a zeta over 9 elements); the other ranks are zero;
//   pass B  per group of 512 / 2^h low patterns (all high patterns): zeta over
//           the high elements, the logarithm of every mask, Mobius over the
//           high elements;
//   pass C  per X_H: Mobius over the low elements for the ranks |X_H| ..
//           |X_H| + 9 (the only ones read out) and c[X] = L_{|X|}(X).
// Butterflies run two elements at a time (a quad of entries per thread step,
// the additions of the two single steps in their order), the last element of
// an odd count alone; a warp skips a step when all its pairs are known no-ops
// (zero sources in a zeta, targets that are never read out in a Mobius); the
// pairs or quads are visited in popcount order of their other elements (of
// the tile bits in passes A and C, of the high part in pass B), so that the
// no-ops fall into whole warps: 39 % of the transforms' pair visits are
// skipped at n = 16 (28 % in mask order). The butterfly loops are kept rolled,
// which keeps the kernel within the registers of three CTAs per SM. The
// transforms act on M_k = k L_k (linear), and the read-out divides by |S|.
// The input row and the ranked arrays come into the tile by asynchronous
// copies (cp.async, 16 bytes where the layout allows), all of a thread's
// copies of a staging step in flight at once. The logarithm keeps Z and M of
// one mask in registers and skips the terms Z_m = 0 (m > |X|) when every lane of the warp
// has |X| <= 9: in pass B the masks of a tile are visited in order of
// popcount (|X| = popcount of the tile index + that of the group), so that
// the warps are mostly uniform in |X|.
#include <cuda_runtime.h>
#include <stdint.h>

#include "apm_internal.cuh"

namespace apm {

constexpr int kFscThreads = 256;
constexpr int kFscTileBits = 9;
constexpr int kFscTile = 1 << kFscTileBits;
constexpr int kFscMaxN = 16;

// C(m, k) for m <= 9
__device__ __forceinline__ int binom_small(int m, int k) {
    if (k < 0 || k > m) return 0;
    int r = 1;
    for (int i = 1; i <= k; ++i) r = r * (m - k + i) / i;
    return r;
}

// zeta (sum over subsets) or Mobius (its inverse) over all 2^bits tile masks
// (the low elements) of the rank rows 0..nr-1 of T (rows kFscTile apart). Row r
// holds the rank whose low part has c = c0 + r elements (zeta: the nonzero
// inputs; Mobius: the masks read out). With a full tile (bits = 9, every warp
// busy for nr rounds) a warp skips a step when every lane's pair is known to
// be a no-op: zeta, the source still sums over no mask with c elements (after
// the elements below d, it sums over the masks between its part above d and
// itself); Mobius, no mask with c elements is reached from the target by
// adding elements above d (its value is never read out). With a full tile the
// pairs of a step are visited in popcount order of their other 8 elements
// (ord8), which puts the no-ops of both kinds mostly into whole warps.
__device__ __forceinline__ void fsc_butterfly_low(double *T, int bits, int nr, int c0, bool mobius,
                                                  const uint8_t *ord8, int d0 = 0) {
    const int half = 1 << (bits - 1);
    const bool prune = bits == kFscTileBits;
#pragma unroll 1
    for (int d = d0; d < bits; ++d) {
#pragma unroll 1
        for (int q = threadIdx.x; q < half * nr; q += kFscThreads) {
            const int r = q >> (bits - 1), p = prune ? ord8[q & (half - 1)] : q & (half - 1);
            const int lo = ((p >> d) << (d + 1)) | (p & ((1 << d) - 1)), hi = lo | (1 << d);
            if (prune) {
                const int c = c0 + r;
                bool skip;
                if (!mobius) {
                    skip = __popc(lo) < c || __popc(lo >> d) > c;
                } else {
                    const int ph = __popc(hi), free_above = (bits - 1 - d) - __popc(lo >> (d + 1));
                    skip = ph > c || ph + free_above < c;
                }
                if (__all_sync(0xffffffffu, skip)) continue;
            }
            double *row = T + r * kFscTile;
            const double v = row[lo];
            row[hi] = mobius ? row[hi] - v : row[hi] + v;
        }
        __syncthreads();
    }
}

// Two steps at once of a full-tile transform over the low elements (tile bits
// d and d + 1): one quad (x, x + 2^d, x + 2^(d+1), x + 2^d + 2^(d+1)) per
// thread step, the quads visited in popcount order of their other 7 bits
// (ord7); a warp skips a quad step when each of its four pairs is a no-op by
// the rules of fsc_butterfly_low. The additions are those of the two single
// steps, in the same order.
__device__ __forceinline__ bool fsc_low_noop(int lo, int d, int c, bool mobius) {
    if (!mobius) return __popc(lo) < c || __popc(lo >> d) > c;
    const int ph = __popc(lo) + 1, free_above = (kFscTileBits - 1 - d) - __popc(lo >> (d + 1));
    return ph > c || ph + free_above < c;
}
__device__ __forceinline__ void fsc_butterfly_low4(double *T, int nr, int c0, int d, bool mobius,
                                                   const uint8_t *ord7) {
#pragma unroll 1
    for (int q = threadIdx.x; q < (kFscTile / 4) * nr; q += kFscThreads) {
        const int r = q >> (kFscTileBits - 2), p = ord7[q & (kFscTile / 4 - 1)];
        const int a = ((p >> d) << (d + 2)) | (p & ((1 << d) - 1));  // bits d, d+1 clear
        const int b = a | (1 << d), cq = a | (1 << (d + 1)), e = b | cq, c = c0 + r;
        const bool skip = fsc_low_noop(a, d, c, mobius) && fsc_low_noop(cq, d, c, mobius) &&
                          fsc_low_noop(a, d + 1, c, mobius) && fsc_low_noop(b, d + 1, c, mobius);
        if (__all_sync(0xffffffffu, skip)) continue;
        double *row = T + r * kFscTile;
        const double va = row[a], vb = row[b], vc = row[cq], ve = row[e];
        if (!mobius) {
            row[b] = vb + va;
            row[cq] = vc + va;
            row[e] = (ve + vc) + (vb + va);
        } else {
            row[b] = vb - va;
            row[cq] = vc - va;
            row[e] = (ve - vc) - (vb - va);
        }
    }
    __syncthreads();
}

// A full-tile transform over the 9 low elements: four double steps, then the
// last element alone.
__device__ __forceinline__ void fsc_transform_low(double *T, int nr, int c0, bool mobius, const uint8_t *ord8,
                                                  const uint8_t *ord7) {
    for (int d = 0; d + 1 < kFscTileBits; d += 2) fsc_butterfly_low4(T, nr, c0, d, mobius, ord7);
    fsc_butterfly_low(T, kFscTileBits, nr, c0, mobius, ord8, kFscTileBits - 1);
}

// pass B: zeta or Mobius over the high tile bits [lg, 9) (the h = 9 - lg high
// elements) of the rank rows 0..n-1 (rank k = row + 1), the pairs of a step
// visited in popcount order of their high part (ordh: the masks of h - 1 bits
// by popcount) so that warps skip together: zeta, the source holds zeros (after
// pass A only high parts with k - 9 .. k elements are nonzero, and after the
// high elements below d the source sums over the high parts between its part
// above d and itself); Mobius, no high part with k - 9 .. k elements (the only
// ones pass C reads at rank k) is reached from the target by adding elements
// above d.
__device__ __forceinline__ void fsc_butterfly_high(double *T, int lg, int n, bool mobius, const uint8_t *ordh,
                                                   int dh0 = 0) {
    const int h = kFscTileBits - lg;
#pragma unroll 1
    for (int dh = dh0; dh < h; ++dh) {
        const int d = lg + dh;
#pragma unroll 1
        for (int q = threadIdx.x; q < (kFscTile / 2) * n; q += kFscThreads) {
            const int r = q >> (kFscTileBits - 1), pq = q & (kFscTile / 2 - 1);
            const int xr = ordh[pq >> lg];                                             // h - 1 bits
            const int xlo = ((xr >> dh) << (dh + 1)) | (xr & ((1 << dh) - 1));         // bit dh clear
            const int lo = (xlo << lg) | (pq & ((1 << lg) - 1)), hi = lo | (1 << d);
            const int k = r + 1, pl = __popc(xlo);
            bool skip;
            if (!mobius) {
                skip = pl < k - kFscTileBits || __popc(xlo >> dh) > k;
            } else {
                const int free_above = (h - 1 - dh) - __popc(xlo >> (dh + 1));
                skip = pl + 1 > k || pl + 1 + free_above < k - kFscTileBits;
            }
            if (__all_sync(0xffffffffu, skip)) continue;
            double *row = T + r * kFscTile;
            const double v = row[lo];
            row[hi] = mobius ? row[hi] - v : row[hi] + v;
        }
        __syncthreads();
    }
}

// Two steps at once of the pass-B transform: the high elements dh and dh+1
// (tile bits d = lg + dh and d + 1), one quad (x, x + 2^d, x + 2^(d+1),
// x + 2^d + 2^(d+1)) per thread step, the quads visited in popcount order of
// their other h - 2 high bits (ordh2). A warp skips a quad step when each of
// its four pairs (two per element) is a no-op by the rules of
// fsc_butterfly_high.
__device__ __forceinline__ bool fsc_pair_noop(int xlo, int dh, int h, int k, bool mobius) {
    if (!mobius) return __popc(xlo) < k - kFscTileBits || __popc(xlo >> dh) > k;
    const int free_above = (h - 1 - dh) - __popc(xlo >> (dh + 1));
    const int pl = __popc(xlo);
    return pl + 1 > k || pl + 1 + free_above < k - kFscTileBits;
}
__device__ __forceinline__ void fsc_butterfly_high4(double *T, int lg, int n, int dh, bool mobius,
                                                    const uint8_t *ordh2) {
    const int h = kFscTileBits - lg, d = lg + dh;
#pragma unroll 1
    for (int q = threadIdx.x; q < (kFscTile / 4) * n; q += kFscThreads) {
        const int r = q >> (kFscTileBits - 2), pq = q & (kFscTile / 4 - 1);
        const int xr = ordh2[pq >> lg];                                              // h - 2 bits
        const int xlo = ((xr >> dh) << (dh + 2)) | (xr & ((1 << dh) - 1));          // bits dh, dh+1 clear
        const int k = r + 1;
        const int bd = 1 << dh, bd1 = 1 << (dh + 1);
        // the pairs of element dh (sources x and x + 2^(dh+1)) and of element dh+1
        // (sources x and x + 2^dh, the latter already summed over element dh)
        const bool skip = fsc_pair_noop(xlo, dh, h, k, mobius) && fsc_pair_noop(xlo | bd1, dh, h, k, mobius) &&
                          fsc_pair_noop(xlo, dh + 1, h, k, mobius) && fsc_pair_noop(xlo | bd, dh + 1, h, k, mobius);
        if (__all_sync(0xffffffffu, skip)) continue;
        double *row = T + r * kFscTile;
        const int a = (xlo << lg) | (pq & ((1 << lg) - 1)), b = a | (1 << d), c = a | (1 << (d + 1)), e = b | c;
        const double va = row[a], vb = row[b], vc = row[c], ve = row[e];
        if (!mobius) {
            row[b] = vb + va;
            row[c] = vc + va;
            row[e] = (ve + vc) + (vb + va);
        } else {
            row[b] = vb - va;
            row[c] = vc - va;
            row[e] = (ve - vc) - (vb - va);
        }
    }
    __syncthreads();
}

// The pass-B transform over the h high elements: two elements at a time, and
// the last one alone when h is odd.
__device__ __forceinline__ void fsc_transform_high(double *T, int lg, int n, bool mobius, const uint8_t *ordh,
                                                   const uint8_t *ordh2) {
    const int h = kFscTileBits - lg;
    int dh = 0;
    for (; dh + 1 < h; dh += 2) fsc_butterfly_high4(T, lg, n, dh, mobius, ordh2);
    if (dh < h) fsc_butterfly_high(T, lg, n, mobius, ordh, dh);
}

// M_1..M_n (M_k = k L_k, L = log Z) of tile entry t in place of Z_1..Z_n,
// for a mask with at most X elements (Z_m = 0 for m > X; X <= n). The Z_m
// are read from the tile as they are needed and the M_k kept in registers,
// then stored together, which keeps the kernel within the registers of three
// CTAs per SM without a spill.
template <int X>
__device__ __forceinline__ void fsc_log_entry(double *T, int t, int n) {
    double M[kFscMaxN + 1];
#pragma unroll
    for (int k = 1; k <= kFscMaxN; ++k) {
        if (k <= n) {
            double s = 0.0;
            if (k <= X) s = static_cast<double>(k) * T[(k - 1) * kFscTile + t];
#pragma unroll
            for (int m = 1; m < kFscMaxN; ++m)
                if (m < k && m <= X) s = fma(-T[(m - 1) * kFscTile + t], M[k - m], s);
            M[k] = s;
        }
    }
#pragma unroll
    for (int k = 1; k <= kFscMaxN; ++k)
        if (k <= n) T[(k - 1) * kFscTile + t] = M[k];
}

// the logarithm for the tile entries order[i] (i < nx; identity when order is
// NULL), whose masks have popcount(entry) + xoff elements
__device__ __forceinline__ void fsc_log(double *T, int nx, int n, const uint16_t *order, int xoff) {
    for (int base = 0; base < nx; base += kFscThreads) {
        const int i = base + threadIdx.x;
        const bool act = i < nx;
        const int t = act ? (order ? order[i] : i) : 0;
        const int x = act ? __popc(t) + xoff : 0;
        const int xm = __reduce_max_sync(0xffffffffu, static_cast<unsigned>(x));
        if (!act) continue;
        // two specialisations: more would not fit the registers of three CTAs per SM
        if (xm <= 9)
            fsc_log_entry<9>(T, t, n);
        else
            fsc_log_entry<kFscMaxN>(T, t, n);
    }
}

// Rows: a + b 2^n -> c + b 2^n for b < batch, or, with `order`, in place on the
// rows c + c_off[order[*first + i]] for i < *count (a may equal c: every row is
// read in pass A before pass C writes it).
__global__ void __launch_bounds__(kFscThreads, 3) fsc_kernel(const double *a, int n, int64_t batch, double *c,
                                                              double *ws, const int *order, const int64_t *c_off,
                                                              const unsigned *first, const unsigned *count) {
    extern __shared__ __align__(16) double T[];
    __shared__ uint16_t s_order[kFscTile];  // tile entries by (popcount, value)
    __shared__ double s_inv[kFscMaxN + 1];  // 1/k
    __shared__ uint8_t s_ordh[1 << (kFscMaxN - kFscTileBits - 1)];  // masks of h - 1 bits by popcount
    __shared__ uint8_t s_ordh2[1 << (kFscMaxN - kFscTileBits - 2)];  // masks of h - 2 bits by popcount
    __shared__ uint8_t s_ord8[kFscTile / 2];                        // masks of 8 bits by popcount
    __shared__ uint8_t s_ord7[kFscTile / 4];                        // masks of 7 bits by popcount
    const int tid = threadIdx.x;
    const int N = 1 << n;
    if (tid <= kFscMaxN) s_inv[tid] = tid ? 1.0 / tid : 0.0;
    for (int t = tid; t < kFscTile; t += kFscThreads) {
        // position of t: the classes of fewer elements first, then the rank of t
        // among the masks of its popcount (combinatorial number system)
        const int p = __popc(t);
        int pos = 0;
        for (int c = 0; c < p; ++c) pos += binom_small(kFscTileBits, c);
        int i = 0;
        for (int r = t; r; r &= r - 1) pos += binom_small(__ffs(r) - 1, ++i);
        s_order[pos] = static_cast<uint16_t>(t);
    }
    for (int t = tid; t < kFscTile / 2; t += kFscThreads) {
        const int p = __popc(t);
        int pos = 0;
        for (int c = 0; c < p; ++c) pos += binom_small(kFscTileBits - 1, c);
        int i = 0;
        for (int r = t; r; r &= r - 1) pos += binom_small(__ffs(r) - 1, ++i);
        s_ord8[pos] = static_cast<uint8_t>(t);
    }
    for (int t = tid; t < kFscTile / 4; t += kFscThreads) {
        const int p = __popc(t);
        int pos = 0;
        for (int c = 0; c < p; ++c) pos += binom_small(kFscTileBits - 2, c);
        int i = 0;
        for (int r = t; r; r &= r - 1) pos += binom_small(__ffs(r) - 1, ++i);
        s_ord7[pos] = static_cast<uint8_t>(t);
    }
    const int hb = n > kFscTileBits ? n - kFscTileBits - 1 : 0;  // bits of the high part minus one
    for (int t = tid; t < (1 << hb); t += kFscThreads) {
        const int p = __popc(t);
        int pos = 0;
        for (int c = 0; c < p; ++c) pos += binom_small(hb, c);
        int i = 0;
        for (int r = t; r; r &= r - 1) pos += binom_small(__ffs(r) - 1, ++i);
        s_ordh[pos] = static_cast<uint8_t>(t);
    }
    const int hb2 = n > kFscTileBits + 1 ? n - kFscTileBits - 2 : 0;  // bits of the high part minus two
    for (int t = tid; t < (1 << hb2); t += kFscThreads) {
        const int p = __popc(t);
        int pos = 0;
        for (int c = 0; c < p; ++c) pos += binom_small(hb2, c);
        int i = 0;
        for (int r = t; r; r &= r - 1) pos += binom_small(__ffs(r) - 1, ++i);
        s_ordh2[pos] = static_cast<uint8_t>(t);
    }
    __syncthreads();
    const int64_t items = order ? static_cast<int64_t>(*count) : batch;
    const int64_t i0 = order ? static_cast<int64_t>(*first) : 0;
    auto row_in = [&](int64_t i) { return order ? c + c_off[order[i0 + i]] : a + i * N; };
    auto row_out = [&](int64_t i) { return order ? c + c_off[order[i0 + i]] : c + i * N; };
    if (n <= kFscTileBits) {
        for (int64_t b = blockIdx.x; b < items; b += gridDim.x) {
            const double *ab = row_in(b);
            for (int q = tid; q < n * N; q += kFscThreads) {
                const int r = q >> n, x = q & (N - 1);
                T[r * kFscTile + x] = __popc(x) == r + 1 ? ab[x] : 0.0;
            }
            __syncthreads();
            fsc_butterfly_low(T, n, n, 1, false, s_ord8);
            fsc_log(T, N, n, nullptr, 0);
            __syncthreads();
            fsc_butterfly_low(T, n, n, 1, true, s_ord8);
            double *cb = row_out(b);
            for (int x = tid; x < N; x += kFscThreads)
                cb[x] = x ? T[(__popc(x) - 1) * kFscTile + x] * s_inv[__popc(x)] : 0.0;
            __syncthreads();
        }
        return;
    }
    const int h = n - kFscTileBits, NH = 1 << h, lg = kFscTileBits - h;  // G = 2^lg low patterns per group
    double *R = ws + static_cast<size_t>(blockIdx.x) * n * N;           // [n][N]
    for (int64_t b = blockIdx.x; b < items; b += gridDim.x) {
        const double *ab = row_in(b);
        // pass A: partial zeta over the low elements
        for (int XH = 0; XH < NH; ++XH) {
            const int p = __popc(XH), k0 = p > 1 ? p : 1, k1 = p + kFscTileBits < n ? p + kFscTileBits : n;
            const int nr = k1 - k0 + 1;
            const size_t base = static_cast<size_t>(XH) << kFscTileBits;
            for (int q = tid; q < nr * kFscTile; q += kFscThreads) {
                const int r = q >> kFscTileBits, x = q & (kFscTile - 1);
                if (__popc(x) + p == k0 + r)
                    cp_async8(T + q, ab + base + x);
                else
                    T[q] = 0.0;
            }
            cp_async_wait_all();
            __syncthreads();
            fsc_transform_low(T, nr, k0 - p, false, s_ord8, s_ord7);
            for (int q = tid; q < n * kFscTile; q += kFscThreads) {
                const int k = (q >> kFscTileBits) + 1, x = q & (kFscTile - 1);
                R[static_cast<size_t>(k - 1) * N + base + x] =
                    k >= k0 && k <= k1 ? T[(k - k0) * kFscTile + x] : 0.0;
            }
            __syncthreads();
        }
        // pass B: zeta over the high elements, logarithm, Mobius over the high elements
        for (int g = 0; g < NH; ++g) {
            // pairs of entries (lg >= 1: j and j + 1 are adjacent in R as in T)
            for (int q2 = tid; q2 < n * kFscTile / 2; q2 += kFscThreads) {
                const int q = 2 * q2, r = q >> kFscTileBits, t = q & (kFscTile - 1);
                const int XH = t >> lg, j = t & ((1 << lg) - 1);
                cp_async16(T + q, R + static_cast<size_t>(r) * N + (static_cast<size_t>(XH) << kFscTileBits) +
                                      (g << lg) + j);
            }
            cp_async_wait_all();
            __syncthreads();
            fsc_transform_high(T, lg, n, false, s_ordh, s_ordh2);
            fsc_log(T, kFscTile, n, s_order, __popc(g));
            __syncthreads();
            fsc_transform_high(T, lg, n, true, s_ordh, s_ordh2);
            for (int q = tid; q < n * kFscTile; q += kFscThreads) {
                const int r = q >> kFscTileBits, t = q & (kFscTile - 1);
                const int XH = t >> lg, j = t & ((1 << lg) - 1);
                R[static_cast<size_t>(r) * N + (static_cast<size_t>(XH) << kFscTileBits) + (g << lg) + j] = T[q];
            }
            __syncthreads();
        }
        // pass C: Mobius over the low elements and the read-out c[X] = L_|X|(X)
        double *cb = row_out(b);
        for (int XH = 0; XH < NH; ++XH) {
            const int p = __popc(XH), k0 = p > 1 ? p : 1, k1 = p + kFscTileBits < n ? p + kFscTileBits : n;
            const int nr = k1 - k0 + 1;
            const size_t base = static_cast<size_t>(XH) << kFscTileBits;
            for (int q2 = tid; q2 < nr * kFscTile / 2; q2 += kFscThreads) {
                const int q = 2 * q2, r = q >> kFscTileBits, x = q & (kFscTile - 1);
                cp_async16(T + q, R + static_cast<size_t>(k0 + r - 1) * N + base + x);
            }
            cp_async_wait_all();
            __syncthreads();
            fsc_transform_low(T, nr, k0 - p, true, s_ord8, s_ord7);
            for (int x = tid; x < kFscTile; x += kFscThreads)
                cb[base + x] = (XH | x) ? T[(__popc(x) + p - k0) * kFscTile + x] * s_inv[__popc(x) + p] : 0.0;
            __syncthreads();
        }
    }
}

static size_t fsc_smem(int n) { return static_cast<size_t>(n) * kFscTile * sizeof(double); }

int fsc_grid(int n, int64_t batch, int *err) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = fsc_smem(n);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fsc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(fsc_smem(kFscMaxN)));
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fsc_kernel, kFscThreads, smem);
    if (e != cudaSuccess || per_sm < 1) {
        *err = e != cudaSuccess ? static_cast<int>(e) : static_cast<int>(cudaErrorInvalidConfiguration);
        return 0;
    }
    *err = 0;
    int64_t g = static_cast<int64_t>(sms) * per_sm;
    if (batch < g) g = batch;
    return static_cast<int>(g < 1 ? 1 : g);
}

size_t fsc_workspace_bytes(int n, int64_t batch, int *err) {
    *err = 0;
    if (n <= kFscTileBits || batch == 0) return 0;
    const int grid = fsc_grid(n, batch, err);
    if (*err) return 0;
    return static_cast<size_t>(grid) * n * (static_cast<size_t>(1) << n) * sizeof(double);
}

int launch_fsc(const double *a, int n, int64_t batch, double *c, void *workspace, cudaStream_t s) {
    int err = 0;
    const int grid = fsc_grid(n, batch, &err);
    if (err) return err;
    fsc_kernel<<<grid, kFscThreads, fsc_smem(n), s>>>(a, n, batch, c, static_cast<double *>(workspace), nullptr,
                                                      nullptr, nullptr, nullptr);
    return static_cast<int>(cudaGetLastError());
}

int launch_fsc_items(double *c, const int64_t *c_off, const int *order, const unsigned *first,
                     const unsigned *count, int64_t max_items, int n, void *workspace, cudaStream_t s) {
    int err = 0;
    const int grid = fsc_grid(n, max_items, &err);
    if (err) return err;
    fsc_kernel<<<grid, kFscThreads, fsc_smem(n), s>>>(c, n, max_items, c, static_cast<double *>(workspace), order,
                                                      c_off, first, count);
    return static_cast<int>(cudaGetLastError());
}

}  // namespace apm
