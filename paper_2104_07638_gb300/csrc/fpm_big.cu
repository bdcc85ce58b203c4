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
constexpr int kBigSubThreads = 512;

// Workspace parts (bytes, each a multiple of 256). The upper levels run in two
// launches: levels 0 .. s1-1 (s1 = H/2) for each matrix, then levels
// s1 .. H-1 for each node of level s1; nodeM holds the nodes of level s1 and
// nodeL the leaves (level H).
struct BigPlan {
    int H, s1;
    size_t thr, cm, an, flags, ccount, clog, det, nodeM, nodeL, lstat, leafws, total;
};

static size_t big_align(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

static int big_plan(int n, int64_t batch, BigPlan *p) {
    const size_t b = static_cast<size_t>(batch);
    p->H = n - kBigLeafN;
    p->s1 = p->H / 2;
    const size_t km = static_cast<size_t>(n - p->s1);
    p->thr = big_align(b * sizeof(double));
    p->cm = p->thr;
    p->an = p->thr;
    p->flags = big_align(b * sizeof(uint32_t));
    p->ccount = big_align(b * sizeof(int));
    p->clog = big_align(b * kBigCorrCap * 2 * sizeof(double));
    p->det = big_align(b * (static_cast<size_t>(1) << p->H) * sizeof(double));
    p->nodeM = big_align(b * (static_cast<size_t>(1) << p->s1) * km * km * sizeof(double));
    p->nodeL = big_align(b * (static_cast<size_t>(1) << p->H) * kBigLeafN * kBigLeafN * sizeof(double));
    p->lstat = big_align(b * (static_cast<size_t>(1) << p->H) * sizeof(uint32_t));
    int err = 0;
    p->leafws = big_align(fpm_warp_workspace_bytes(kBigLeafN, batch << p->H, &err));
    p->total = p->thr + p->cm + p->an + p->flags + p->ccount + p->clog + 2 * p->det + p->nodeM + p->nodeL + p->lstat +
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

// Shared-memory layout of a subtree launch over levels ls .. ls+nl-1 (k0 =
// n - ls): the even and odd relative levels alternate between two buffers
// (level j holds 2^j nodes of k0 - j squared entries), then the reciprocal
// pivots of one level and the node minors of the current and the next level.
struct BigSubLayout {
    size_t odd, ip, nd, bytes;
};
static BigSubLayout big_sub_layout(int n, int ls, int nl) {
    const int k0 = n - ls;
    size_t e = 0, o = 0;
    for (int j = 0; j < nl; ++j) {
        const size_t sz = (static_cast<size_t>(1) << j) * (k0 - j) * (k0 - j);
        if (j & 1) o = o > sz ? o : sz;
        else e = e > sz ? e : sz;
    }
    BigSubLayout L;
    L.odd = e;
    L.ip = e + o;
    L.nd = L.ip + (static_cast<size_t>(1) << (nl - 1));
    L.bytes = (L.nd + 2 * (static_cast<size_t>(1) << nl)) * sizeof(double);
    return L;
}

// One CTA per node of level ls (global index w0 = b 2^ls + i0; for ls = 0 the
// matrix itself): its subtree's levels ls .. ls+nl-1 breadth first in shared
// memory, and the nodes of level ls+nl with their minors written out. Node
// (l, i) of matrix b has global index b 2^l + i and children 2i (drop the
// node's last element: its leading block) and 2i+1 (keep it: the leading
// block less the rank-1 term of the last row and column over the pivot, the
// pivot shifted by C = sign(p) Cm where |p| <= thrA and recorded with its
// unshifted value).
__global__ void __launch_bounds__(kBigSubThreads) big_subtree_kernel(
    const double *__restrict__ src, const double *__restrict__ dsrc, double *__restrict__ dst,
    double *__restrict__ ddst, int n, int ls, int nl, size_t off_odd, size_t off_ip, size_t off_nd,
    const double *__restrict__ thrA, const double *__restrict__ Cm, int *ccount, double *clog, uint32_t *flags) {
    extern __shared__ __align__(16) double sm[];
    const int tid = threadIdx.x, T = blockDim.x;
    const int64_t w0 = blockIdx.x;
    const int64_t b = w0 >> ls;
    const int k0 = n - ls;
    double *const IP = sm + off_ip;
    double *const ND = sm + off_nd;
    const double *R = src + w0 * k0 * k0;
    for (int e = tid; e < k0 * k0; e += T) sm[e] = R[e];
    if (tid == 0) ND[0] = dsrc[w0];
    __syncthreads();
    const double thr = thrA[b], cm = Cm[b];
    for (int j = 0; j < nl; ++j) {
        const int k = k0 - j, k1 = k - 1, kk = k * k, kk1 = k1 * k1, P = 1 << j, l = ls + j;
        const bool last = j == nl - 1;
        const double *cur = sm + ((j & 1) ? off_odd : 0);
        double *nxt = sm + ((j & 1) ? 0 : off_odd);
        const double *ndc = ND + ((j & 1) << nl);
        double *ndn = ND + (((j + 1) & 1) << nl);
        for (int t = tid; t < P; t += T) {
            const int64_t wp = (w0 << j) + t;  // global index at level l
            const double p = cur[t * kk + k1 * k + k1];
            const double C = fabs(p) <= thr ? (p >= 0.0 ? cm : -cm) : 0.0;
            const double pp = p + C;
            IP[t] = 1.0 / pp;
            const double d = ndc[t];
            if (last) {
                ddst[2 * wp] = d;
                ddst[2 * wp + 1] = d * pp;
            } else {
                ndn[2 * t] = d;
                ndn[2 * t + 1] = d * pp;
            }
            const long long bits = __double_as_longlong(pp);
            if ((bits << 1) == 0 || ((bits >> 52) & 0x7ff) == 0x7ff) atomicOr(&flags[b], APM_ST_ZERO_PIVOT);
            if (C != 0.0) {
                const int pos = atomicAdd(&ccount[b], 1);
                if (pos < kBigCorrCap) {
                    const int64_t i = wp - (b << l);
                    clog[(b * kBigCorrCap + pos) * 2] = static_cast<double>(l) + 32.0 * static_cast<double>(i);
                    clog[(b * kBigCorrCap + pos) * 2 + 1] = p;
                } else {
                    atomicOr(&flags[b], APM_ST_CORRECTION_OVERFLOW);
                }
                atomicOr(&flags[b], APM_ST_PIVOT_CORRECTED);
            }
        }
        __syncthreads();
        for (int e = tid; e < P * kk1; e += T) {
            const int t = e / kk1, rem = e - t * kk1, r = rem / k1, q = rem - r * k1;
            const double *M = cur + t * kk;
            const double v = M[r * k + q];
            const double v1 = fma(-M[r * k + k1] * IP[t], M[k1 * k + q], v);
            if (last) {
                double *D0 = dst + 2 * ((w0 << j) + t) * kk1;
                D0[rem] = v;
                D0[kk1 + rem] = v1;
            } else {
                nxt[(2 * t) * kk1 + rem] = v;
                nxt[(2 * t + 1) * kk1 + rem] = v1;
            }
        }
        __syncthreads();
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
    double *nodeM = reinterpret_cast<double *>(w);
    double *leaves = reinterpret_cast<double *>(w + p.nodeM);
    w += p.nodeM + p.nodeL;
    uint32_t *lstat = reinterpret_cast<uint32_t *>(w);
    w += p.lstat;
    void *leafws = w;

    const int64_t warps0 = batch;
    big_prep_kernel<<<static_cast<unsigned>((warps0 * 32 + kBigThreads - 1) / kBigThreads), kBigThreads, 0, s>>>(
        A, n, batch, thr, shf, thrA, Cm, an, flags, ccount, det[0]);
    // levels 0 .. s1-1 for each matrix (det[0]: the roots' minors, 1), then
    // levels s1 .. H-1 for each node of level s1; the leaves' minors in det[0]
    const int s1 = p.s1, s2 = H - s1;
    const BigSubLayout L1 = big_sub_layout(n, 0, s1), L2 = big_sub_layout(n, s1, s2);
    err = static_cast<int>(cudaFuncSetAttribute(big_subtree_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                static_cast<int>(L1.bytes > L2.bytes ? L1.bytes : L2.bytes)));
    if (err) return err;
    big_subtree_kernel<<<static_cast<unsigned>(batch), kBigSubThreads, L1.bytes, s>>>(
        A, det[0], nodeM, det[1], n, 0, s1, L1.odd, L1.ip, L1.nd, thrA, Cm, ccount, clog, flags);
    big_subtree_kernel<<<static_cast<unsigned>(batch << s1), kBigSubThreads, L2.bytes, s>>>(
        nodeM, det[1], leaves, det[0], n, s1, s2, L2.odd, L2.ip, L2.nd, thrA, Cm, ccount, clog, flags);
    const double *src = leaves;
    err = static_cast<int>(cudaGetLastError());
    if (err) return err;
    // the leaves: 12 x 12 matrices in the order of T, their minors into the rows
    err = launch_fpm_warp(src, kBigLeafN, batch << H, minors, thr, shf, lstat, leafws, s, det[0], an, H);
    if (err) return err;
    big_backprop_kernel<<<static_cast<unsigned>(batch), 512, 0, s>>>(minors, n, H, ccount, clog, Cm, flags);
    big_status_kernel<<<static_cast<unsigned>(batch), 512, 0, s>>>(minors, n, H, flags, lstat, status);
    return static_cast<int>(cudaGetLastError());
}

}  // namespace apm
