/*
 * The paper's own algorithm on the host, as the benchmark's second CPU
 * baseline (not the oracle, which evaluates every minor by its own
 * elimination; the tests check this code against the oracle):
 *   - all 2^n principal minors by the depth-first tree of Section II (Alg. 1):
 *     the node of level l holds the Schur complement, on the elements l..n-1,
 *     of the elements kept so far; its pivot p (the leading entry) gives the
 *     minor of the kept set with l added, the left child drops element l (a
 *     view of the same rows) and the right child is the Schur complement with
 *     respect to p;
 *   - the pivot correction of Section II: a pivot with |p| <= thr * ||A||max
 *     becomes p + C, C = sign(p) * shift * ||A||max, the node and its right
 *     subtree are minors of the shifted matrix, and afterwards, deepest level
 *     first, det[m] -= C det[m without l] over the node and its right subtree;
 *   - the connected sums by the CDet recursion (Section V.A, Eq. recursion)
 *     on a[S] = det(A[S])^2, j = the lowest element of S.
 * One matrix per OpenMP thread; plain C, built with -O3 (no target-specific
 * flags) so that it builds and runs the same on x86 and Arm hosts.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int level;
    int mask;  /* the kept elements, level included */
    double C;
} fs_corr;

typedef struct {
    int n;
    double thr, shift;
    double *minors;
    double *buf;      /* right-child matrices, one (n-l-1)^2 block per level */
    size_t *off;      /* offset of level l's block in buf */
    fs_corr *corr;
    int ncorr, capcorr, overflow;
} fs_state;

/* Node of level l: M (k x k, row stride ld, k = n - l) is the Schur complement
 * on elements l..n-1; det is the minor of the kept set `mask` (bits < l). */
static void fs_node(fs_state *st, int l, int mask, double det, const double *M, int ld) {
    const int n = st->n, k = n - l;
    if (k == 0) return;
    /* left: drop element l, the trailing block of the same rows */
    fs_node(st, l + 1, mask, det, M + ld + 1, ld);
    /* right: keep element l */
    double p = M[0];
    if (fabs(p) <= st->thr) {
        const double C = p >= 0.0 ? st->shift : -st->shift;
        p += C;
        if (st->ncorr < st->capcorr) {
            st->corr[st->ncorr].level = l;
            st->corr[st->ncorr].mask = mask | (1 << l);
            st->corr[st->ncorr].C = C;
            st->ncorr++;
        } else {
            st->overflow = 1;
        }
    }
    const double dk = det * p;
    st->minors[mask | (1 << l)] = dk;
    if (k == 1) return;
    double *R = st->buf + st->off[l];
    const int k1 = k - 1;
    const double ip = 1.0 / p;
    for (int r = 0; r < k1; ++r) {
        const double f = M[(r + 1) * ld] * ip;
        const double *src = M + (r + 1) * ld + 1;
        const double *top = M + 1;
        double *dst = R + r * k1;
        for (int q = 0; q < k1; ++q) dst[q] = src[q] - f * top[q];
    }
    fs_node(st, l + 1, mask | (1 << l), dk, R, k1);
}

/* The connected sums: c[S] = a[S] - sum over T proper subset of S containing
 * the lowest element of S of c[T] a[S \ T]; c[0] = 0. */
static void fs_cdet(int n, const double *a, double *c) {
    const int N = 1 << n;
    c[0] = 0.0;
    for (int S = 1; S < N; ++S) {
        const int j = S & -S, rest = S ^ j;
        double acc = a[S];
        if (rest) {
            /* T = j | U, U a proper subset of rest (U = rest would give T = S) */
            for (int U = (rest - 1) & rest;; U = (U - 1) & rest) {
                const int T = j | U;
                acc -= c[T] * a[S ^ T];
                if (U == 0) break;
            }
        }
        c[S] = acc;
    }
}

/* minors[b][2^n] and c[b][2^n] for the batch; status[b] bit 0 = corrected,
 * bit 1 = more corrections than recorded (row left as computed). */
void fpm_sc_batch(const double *A, int n, int64_t batch, double *minors, double *c, double thr, double shift,
                  int *status, int nthreads) {
    const int N = 1 << n;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        fs_state st;
        st.n = n;
        size_t total = 0;
        st.off = (size_t *)malloc(sizeof(size_t) * (size_t)(n + 1));
        for (int l = 0; l < n; ++l) {
            st.off[l] = total;
            total += (size_t)(n - l - 1) * (size_t)(n - l - 1);
        }
        st.buf = (double *)malloc(sizeof(double) * (total + 1));
        st.capcorr = 4 * N;
        st.corr = (fs_corr *)malloc(sizeof(fs_corr) * (size_t)st.capcorr);
        double *a = (double *)malloc(sizeof(double) * (size_t)N);
#pragma omp for schedule(dynamic, 16)
        for (int64_t b = 0; b < batch; ++b) {
            const double *M = A + b * n * n;
            double amax = 0.0;
            for (int e = 0; e < n * n; ++e) amax = fmax(amax, fabs(M[e]));
            const double sc = amax > 0.0 ? amax : 1.0;
            st.thr = thr * sc;
            st.shift = shift * sc;
            st.minors = minors + b * N;
            st.ncorr = 0;
            st.overflow = 0;
            st.minors[0] = 1.0;
            fs_node(&st, 0, 0, 1.0, M, n);
            /* back-propagation, deepest level first */
            for (int l = n - 1; l >= 0; --l) {
                for (int i = 0; i < st.ncorr; ++i) {
                    if (st.corr[i].level != l) continue;
                    const int S = st.corr[i].mask, low = (2 << l) - 1, bit = 1 << l;
                    const double C = st.corr[i].C;
                    /* every m with m & low == S: S plus any set of elements above l */
                    const int hi = (N - 1) & ~low;
                    for (int H = hi;; H = (H - 1) & hi) {
                        const int m = S | H;
                        st.minors[m] -= C * st.minors[m ^ bit];
                        if (H == 0) break;
                    }
                }
            }
            for (int S = 0; S < N; ++S) a[S] = st.minors[S] * st.minors[S];
            fs_cdet(n, a, c + b * N);
            if (status) status[b] = (st.ncorr ? 1 : 0) | (st.overflow ? 2 : 0);
        }
        free(a);
        free(st.corr);
        free(st.buf);
        free(st.off);
    }
}

int fpm_sc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
