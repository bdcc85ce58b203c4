// All principal minors of matrices of order 17..24.
//
// Paper: Section II (Eq. minor, Alg. 1): the minor of a kept set is the minor
// of the set without its last decided element times the pivot of the Schur
// complement reached on the tree path; the pivot correction (the paragraph
// after Eq. minor) shifts a small pivot and back-propagates the shift.
//
// The tree is cut in two. Its upper H = n - 12 levels decide the elements n-1
// down to 12 (the upper set T, bit i of T <-> element 12 + i) and run breadth
// first over the whole batch, one warp per node and one launch per level: a
// node of level l holds the Schur complement, on the elements 0 .. n-1-l, of
// the upper elements kept on its path, and its two children drop or keep its
// last element (the leading block, or the leading block less the rank-1 term
// of the last row and column over the pivot). Its index is the path read as a
// binary number, first decision most significant, so that the 2^H leaves come
// out in the order of T. Every leaf is a 12 x 12 matrix M_T with the minor
// det(A[T]), and det(A[T u U]) = det(A[T]) det(M_T[U]) for U within 0..11: the
// warp-per-matrix minors kernel, with det(A[T]) as its root minor, writes the
// 2^12 minors of M_T already scaled straight into the output row at T * 4096;
// the leaves that meet a small pivot are redone by the fused kernel with its
// own pivot correction, from the same root minor.
//
// A pivot of the upper levels with |p| <= thr ||A||max is shifted by
// C = sign(p) shift ||A||max and recorded with its unshifted value; once the
// rows are complete, deepest level first, det[m] -= C det[m without the
// element] over the kept child's subtree (all T in its range, all U), the
// dropped sibling's rows supplying the second minor, except for the node's own
// minor (the first T of the range, U empty), which is written as the sibling's
// minor times the unshifted pivot. The leaves take the threshold and the shift
// relative to ||A||max of their matrix, not to their own largest entry: a leaf
// is a Schur complement whose entries a small upper pivot can inflate, and its
// pivots are pivots of the same tree as the upper ones. The status word of a
// matrix collects its leaves' bits; an error bit makes the whole row NaN.
#include <cuda_runtime.h>
#include <stdint.h>

#include "apm_internal.cuh"

namespace apm {

constexpr int kBigLeafN = 12;
constexpr int kBigCorrCap = 256;  // upper-level corrections recorded per matrix
constexpr int kBigThreads = 256;

// Workspace parts (bytes, each a multiple of 256).
struct BigPlan {
    int H;
    size_t thr, cm, an, flags, ccount, clog, det, nodeE, nodeO, lstat, leafws, total;
};

static size_t big_align(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

static int big_plan(int n, int64_t batch, BigPlan *p) {
    const size_t b = static_cast<size_t>(batch);
    p->H = n - kBigLeafN;
    size_t e = 0, o = 0;
    for (int l = 1; l <= p->H; ++l) {
        const size_t k = static_cast<size_t>(n - l);
        const size_t sz = b * (static_cast<size_t>(1) << l) * k * k * sizeof(double);
        if (l & 1) o = o > sz ? o : sz;
        else e = e > sz ? e : sz;
    }
    p->thr = big_align(b * sizeof(double));
    p->cm = p->thr;
    p->an = p->thr;
    p->flags = big_align(b * sizeof(uint32_t));
    p->ccount = big_align(b * sizeof(int));
    p->clog = big_align(b * kBigCorrCap * 2 * sizeof(double));
    p->det = big_align(b * (static_cast<size_t>(1) << p->H) * sizeof(double));
    p->nodeE = big_align(e);
    p->nodeO = big_align(o);
    p->lstat = big_align(b * (static_cast<size_t>(1) << p->H) * sizeof(uint32_t));
    int err = 0;
    p->leafws = big_align(fpm_warp_workspace_bytes(kBigLeafN, batch << p->H, &err));
    p->total = p->thr + p->cm + p->an + p->flags + p->ccount + p->clog + 2 * p->det + p->nodeE + p->nodeO + p->lstat +
               p->leafws;
    return err;
}

size_t fpm_big_workspace_bytes(int n, int64_t batch, int *err) {
    *err = 0;
    if (batch == 0) return 0;
    BigPlan p;
    *err = big_plan(n, batch, &p);
    return *err ? 0 : p.total;
}

// One warp per matrix: ||A||max and finiteness; the scaled threshold and
// shift, the norm itself (for the leaves), the root's minor 1, a cleared
// record count.
__global__ void big_prep_kernel(const double *__restrict__ A, int n, int64_t batch, double thr, double shf,
                                double *thrA, double *Cm, double *an, uint32_t *flags, int *ccount, double *det0) {
    const int lane = threadIdx.x & 31;
    const int64_t b = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (b >= batch) return;
    const double *M = A + b * n * n;
    double amax = 0.0;
    int nonfin = 0;
    for (int e = lane; e < n * n; e += 32) {
        const double x = M[e];
        if (!isfinite(x)) nonfin = 1;
        amax = fmax(amax, fabs(x));
    }
    nonfin = __any_sync(0xffffffffu, nonfin);
    for (int o = 16; o > 0; o >>= 1) amax = fmax(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if (lane == 0) {
        const double sc = amax > 0.0 ? amax : 1.0;
        thrA[b] = thr * sc;
        Cm[b] = shf * sc;
        an[b] = sc;
        flags[b] = nonfin ? APM_ST_NONFINITE_INPUT : 0u;
        ccount[b] = 0;
        det0[b] = 1.0;
    }
}

// Level l: one warp per node (matrix b, index i), node = src + (b 2^l + i) k^2,
// k = n - l; children 2i (drop the last element) and 2i+1 (keep it).
__global__ void big_level_kernel(const double *__restrict__ src, double *__restrict__ dst,
                                 const double *__restrict__ dsrc, double *__restrict__ ddst, int n, int l,
                                 int64_t batch, const double *__restrict__ thrA, const double *__restrict__ Cm,
                                 int *ccount, double *clog, uint32_t *flags) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    if (w >= (batch << l)) return;  // whole warps only: blockDim is a multiple of 32
    const int64_t b = w >> l;
    const int k = n - l, k1 = k - 1;
    const double *M = src + w * k * k;
    double *D0 = dst + 2 * w * k1 * k1;
    double *D1 = D0 + static_cast<int64_t>(k1) * k1;
    const double p = M[k1 * k + k1];
    const double C = fabs(p) <= thrA[b] ? (p >= 0.0 ? Cm[b] : -Cm[b]) : 0.0;
    const double pp = p + C;
    const double ip = 1.0 / pp;
    for (int e = lane; e < k1 * k1; e += 32) {
        const int r = e / k1, q = e - r * k1;
        const double v = M[r * k + q];
        D0[e] = v;
        D1[e] = fma(-M[r * k + k1] * ip, M[k1 * k + q], v);
    }
    if (lane == 0) {
        const double d = dsrc[w];
        ddst[2 * w] = d;
        ddst[2 * w + 1] = d * pp;
        const long long bits = __double_as_longlong(pp);
        if ((bits << 1) == 0 || ((bits >> 52) & 0x7ff) == 0x7ff) atomicOr(&flags[b], APM_ST_ZERO_PIVOT);
        if (C != 0.0) {
            const int pos = atomicAdd(&ccount[b], 1);
            if (pos < kBigCorrCap) {
                const int64_t i = w - (b << l);
                clog[(b * kBigCorrCap + pos) * 2] = static_cast<double>(l) + 32.0 * static_cast<double>(i);
                clog[(b * kBigCorrCap + pos) * 2 + 1] = p;
            } else {
                atomicOr(&flags[b], APM_ST_CORRECTION_OVERFLOW);
            }
            atomicOr(&flags[b], APM_ST_PIVOT_CORRECTED);
        }
    }
}

// One CTA per matrix: the upper-level corrections, deepest level first:
// for the kept child of node (l, i), every T in its range and every U,
// out[T, U] -= C out[T - span, U], span = 2^(H-1-l), C = sign(p) Cm; the
// node's own minor (e = 0) is out[T - span, 0] p with the unshifted pivot p.
__global__ void big_backprop_kernel(double *out, int n, int H, const int *ccount, const double *clog,
                                    const double *Cm, const uint32_t *flags) {
    const int64_t b = blockIdx.x;
    const int cnt = ccount[b] < kBigCorrCap ? ccount[b] : kBigCorrCap;
    if (cnt == 0 || (flags[b] & APM_ST_ERROR_MASK)) return;
    double *row = out + (b << n);
    for (int l = H - 1; l >= 0; --l) {
        for (int j = 0; j < cnt; ++j) {
            const double code = clog[(b * kBigCorrCap + j) * 2];
            const int64_t ci = static_cast<int64_t>(code);
            if (static_cast<int>(ci % 32) != l) continue;
            const int64_t i = ci / 32;
            const double pv = clog[(b * kBigCorrCap + j) * 2 + 1];
            const double C = pv >= 0.0 ? Cm[b] : -Cm[b];
            const int64_t span = int64_t(1) << (H - 1 - l);
            const int64_t t0 = (2 * i + 1) * span;
            const int64_t cnt_e = span << kBigLeafN;
            double *kept = row + (t0 << kBigLeafN);
            const double *drop = row + ((t0 - span) << kBigLeafN);
            for (int64_t e = threadIdx.x; e < cnt_e; e += blockDim.x)
                kept[e] = e == 0 ? drop[0] * pv : fma(-C, drop[e], kept[e]);
        }
        __syncthreads();
    }
}

// One CTA per matrix: the status word (the matrix's flags and its leaves'
// bits); an error bit makes the whole row NaN.
__global__ void big_status_kernel(double *out, int n, int H, const uint32_t *flags, const uint32_t *lstat,
                                  uint32_t *status) {
    __shared__ uint32_t s_or;
    const int64_t b = blockIdx.x;
    if (threadIdx.x == 0) s_or = 0u;
    __syncthreads();
    uint32_t acc = 0u;
    for (int64_t t = threadIdx.x; t < (int64_t(1) << H); t += blockDim.x) acc |= lstat[(b << H) + t];
    atomicOr(&s_or, acc);
    __syncthreads();
    const uint32_t st = s_or | flags[b];
    if (threadIdx.x == 0 && status) status[b] = st;
    if (st & APM_ST_ERROR_MASK) {
        const double nanv = __longlong_as_double(0x7ff8000000000000ll);
        double *row = out + (b << n);
        for (int64_t e = threadIdx.x; e < (int64_t(1) << n); e += blockDim.x) row[e] = nanv;
    }
}

int launch_fpm_big(const double *A, int n, int64_t batch, double *minors, double thr, double shf,
                   uint32_t *status, void *workspace, cudaStream_t s) {
    BigPlan p;
    int err = big_plan(n, batch, &p);
    if (err) return err;
    const int H = p.H;
    char *w = static_cast<char *>(workspace);
    double *thrA = reinterpret_cast<double *>(w);
    w += p.thr;
    double *Cm = reinterpret_cast<double *>(w);
    w += p.cm;
    double *an = reinterpret_cast<double *>(w);
    w += p.an;
    uint32_t *flags = reinterpret_cast<uint32_t *>(w);
    w += p.flags;
    int *ccount = reinterpret_cast<int *>(w);
    w += p.ccount;
    double *clog = reinterpret_cast<double *>(w);
    w += p.clog;
    double *det[2] = {reinterpret_cast<double *>(w), reinterpret_cast<double *>(w + p.det)};
    w += 2 * p.det;
    double *node[2] = {reinterpret_cast<double *>(w), reinterpret_cast<double *>(w + p.nodeE)};
    w += p.nodeE + p.nodeO;
    uint32_t *lstat = reinterpret_cast<uint32_t *>(w);
    w += p.lstat;
    void *leafws = w;

    const int64_t warps0 = batch;
    big_prep_kernel<<<static_cast<unsigned>((warps0 * 32 + kBigThreads - 1) / kBigThreads), kBigThreads, 0, s>>>(
        A, n, batch, thr, shf, thrA, Cm, an, flags, ccount, det[0]);
    const double *src = A;
    for (int l = 0; l < H; ++l) {
        const int64_t nodes = batch << l;
        double *dst = node[(l + 1) & 1];
        big_level_kernel<<<static_cast<unsigned>((nodes * 32 + kBigThreads - 1) / kBigThreads), kBigThreads, 0,
                           s>>>(src, dst, det[l & 1], det[(l + 1) & 1], n, l, batch, thrA, Cm, ccount, clog,
                                flags);
        src = dst;
    }
    err = static_cast<int>(cudaGetLastError());
    if (err) return err;
    // the leaves: 12 x 12 matrices in the order of T, their minors into the rows
    err = launch_fpm_warp(src, kBigLeafN, batch << H, minors, thr, shf, lstat, leafws, s, det[H & 1], an, H);
    if (err) return err;
    big_backprop_kernel<<<static_cast<unsigned>(batch), 512, 0, s>>>(minors, n, H, ccount, clog, Cm, flags);
    big_status_kernel<<<static_cast<unsigned>(batch), 512, 0, s>>>(minors, n, H, flags, lstat, status);
    return static_cast<int>(cudaGetLastError());
}

}  // namespace apm
