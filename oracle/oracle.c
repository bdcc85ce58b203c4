/*
 * Plain FP64 CPU oracle for the all-principal-minor path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the product path links, loads or calls
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline
 * leg do. It shares no code, header, table or helper with the CUDA library.
 *
 * Every routine is the direct definition of what it computes, written for
 * obviousness rather than speed:
 *   - principal minors:  one Gaussian elimination with partial pivoting per
 *                        subset (the naive O(n^3 2^n) method that Section II improves on);
 *   - permanents:        Ryser's inclusion-exclusion formula (Eq. ryser,
 *                        Section IV) applied to each principal submatrix, with
 *                        the global sign (-1)^|S| that makes it the permanent;
 *   - connected sums:    the CDet recursion (Eq. recursion, Section V.A) as
 *                        plain loops, and independently the set-partition
 *                        Moebius formula c[S] = sum_pi (-1)^{|pi|-1}(|pi|-1)!
 *                        prod_{B in pi} a[B];
 *   - Keldysh sums:      the sum over all 2^n Keldysh index assignments of a
 *                        separate complex determinant each (Section V.D);
 *   - XNOR minors:       for a 2n x 2n matrix of 2 x 2 blocks, the determinant
 *                        of every submatrix keeping both rows and columns of
 *                        a subset of the blocks (Section III.B, the minors of
 *                        the Nambu CDet of Section V.B), one elimination each;
 *   - NAND minors:       the 3^n submatrices keeping one or neither row and
 *                        column of each block (Section III.C) and their sums
 *                        over the two types of each kept vertex (Section V.C);
 *   - two-spin Keldysh:  the sum over the 2^n assignments shared by both spins
 *                        of the product of the two determinants (Section V.D
 *                        with the two determinants of Eq. CTINT).
 *
 * Subsets are bit masks: element k (0-based) <-> bit k (Section II, the
 * subset labelling S_i by the binary digits of i). Matrices are row-major.
 * Batches are parallelised over matrices with OpenMP; nthreads <= 0 means the
 * OpenMP default.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXN 24

static int popcount_u32(uint32_t x) {
    int c = 0;
    while (x) { c += (int)(x & 1u); x >>= 1; }
    return c;
}

static int threads_for(int nthreads) {
#ifdef _OPENMP
    return nthreads > 0 ? nthreads : omp_get_max_threads();
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_max_threads(void) { return threads_for(0); }

/* Determinant of the k x k row-major matrix M (destroyed) by Gaussian
 * elimination with partial (row) pivoting. det of the empty matrix is 1
 * (Section II). */
static double det_partial_pivot(double *M, int k) {
    double det = 1.0;
    for (int col = 0; col < k; ++col) {
        int piv = col;
        double best = fabs(M[col * k + col]);
        for (int r = col + 1; r < k; ++r) {
            double v = fabs(M[r * k + col]);
            if (v > best) { best = v; piv = r; }
        }
        if (best == 0.0) return 0.0;
        if (piv != col) {
            for (int q = 0; q < k; ++q) {
                double t = M[col * k + q];
                M[col * k + q] = M[piv * k + q];
                M[piv * k + q] = t;
            }
            det = -det;
        }
        double p = M[col * k + col];
        det *= p;
        for (int r = col + 1; r < k; ++r) {
            double f = M[r * k + col] / p;
            for (int q = col + 1; q < k; ++q) M[r * k + q] -= f * M[col * k + q];
        }
    }
    return det;
}

/* Complex version of the above. */
static double complex cdet_partial_pivot(double complex *M, int k) {
    double complex det = 1.0;
    for (int col = 0; col < k; ++col) {
        int piv = col;
        double best = cabs(M[col * k + col]);
        for (int r = col + 1; r < k; ++r) {
            double v = cabs(M[r * k + col]);
            if (v > best) { best = v; piv = r; }
        }
        if (best == 0.0) return 0.0;
        if (piv != col) {
            for (int q = 0; q < k; ++q) {
                double complex t = M[col * k + q];
                M[col * k + q] = M[piv * k + q];
                M[piv * k + q] = t;
            }
            det = -det;
        }
        double complex p = M[col * k + col];
        det *= p;
        for (int r = col + 1; r < k; ++r) {
            double complex f = M[r * k + col] / p;
            for (int q = col + 1; q < k; ++q) M[r * k + q] -= f * M[col * k + q];
        }
    }
    return det;
}

/* All 2^n principal minors det(A[S]) of each n x n matrix, each by its own
 * partial-pivot elimination (Section II, the trivial method); minors[0] = 1. */
void oracle_minors_lu(const double *A, int n, int64_t batch, double *minors, int nthreads) {
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads_for(nthreads))
    for (int64_t b = 0; b < batch; ++b) {
        const double *Ab = A + b * (int64_t)n * n;
        double *out = minors + b * N;
        double M[MAXN * MAXN];
        int idx[MAXN];
        for (int64_t S = 0; S < N; ++S) {
            int k = 0;
            for (int e = 0; e < n; ++e)
                if ((S >> e) & 1) idx[k++] = e;
            for (int r = 0; r < k; ++r)
                for (int q = 0; q < k; ++q) M[r * k + q] = Ab[idx[r] * n + idx[q]];
            out[S] = det_partial_pivot(M, k);
        }
    }
}

/* All 2^n principal permanents perm(A[S]) (mode 0), perm(|A[S]|) (mode 1), or
 * the sum of the absolute values of the Ryser terms (mode 2, the rounding-error
 * scale of any evaluation of Ryser's formula).
 * Ryser's formula (Eq. ryser) on the submatrix A[S] with k = |S| rows:
 *     perm(A[S]) = (-1)^k sum_{T subset of S} (-1)^{|T|} prod_{i in S} sum_{j in T} A_ij.
 * (As printed, Eq. ryser lacks the (-1)^k; with it the formula gives the
 * permanent, e.g. perm of the all-ones k x k matrix = k!.) The inner column
 * sums are rebuilt from scratch for every T; the empty subset gives 1. */
void oracle_perm_ryser(const double *A, int n, int64_t batch, double *perms, int mode,
                       int nthreads) {
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads_for(nthreads))
    for (int64_t b = 0; b < batch; ++b) {
        const double *Ab = A + b * (int64_t)n * n;
        double *out = perms + b * N;
        int idx[MAXN];
        for (int64_t S = 0; S < N; ++S) {
            int k = 0;
            for (int e = 0; e < n; ++e)
                if ((S >> e) & 1) idx[k++] = e;
            double total = 0.0;
            for (int64_t T = 0; T < ((int64_t)1 << k); ++T) {
                double prod = 1.0;
                for (int r = 0; r < k; ++r) {
                    double rs = 0.0;
                    for (int q = 0; q < k; ++q)
                        if ((T >> q) & 1) {
                            double v = Ab[idx[r] * n + idx[q]];
                            rs += mode == 1 ? fabs(v) : v;
                        }
                    prod *= rs;
                }
                if (mode == 2) total += fabs(prod);
                else total += (popcount_u32((uint32_t)T) & 1) ? -prod : prod;
            }
            out[S] = (mode != 2 && (k & 1)) ? -total : total;
        }
    }
}

/* Connected sums by the CDet recursion (Eq. recursion), plain loops:
 *     c[S] = a[S] - sum_{T proper subset of S, j in T} c[T] a[S \ T],
 * with j = the lowest element of S, S taken in increasing numeric order (every
 * proper subset T of S is numerically smaller, so c[T] is final). c[0] = 0.
 * The proper subsets T of S containing j are enumerated as T = {j} u U with U
 * running over the submasks of S \ {j} other than S \ {j} itself. */
void oracle_cdet_recursion(const double *a, int n, int64_t batch, double *c, int nthreads) {
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads_for(nthreads))
    for (int64_t b = 0; b < batch; ++b) {
        const double *ab = a + b * N;
        double *cb = c + b * N;
        cb[0] = 0.0;
        for (int64_t S = 1; S < N; ++S) {
            int64_t j = S & (-S);
            int64_t rest = S ^ j;
            double acc = ab[S];
            if (rest != 0) {
                /* submasks U of rest, U != rest, in decreasing order down to 0 */
                for (int64_t U = (rest - 1) & rest;; U = (U - 1) & rest) {
                    acc -= cb[j | U] * ab[rest ^ U];
                    if (U == 0) break;
                }
            }
            cb[S] = acc;
        }
    }
}

/* The same recursion on absolute values with every sign positive: the sum of
 * the absolute values of all terms that the recursion combines (the error scale
 * for connected sums). ahat >= 0 expected. */
void oracle_cdet_scale(const double *ahat, int n, int64_t batch, double *chat, int nthreads) {
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads_for(nthreads))
    for (int64_t b = 0; b < batch; ++b) {
        const double *ab = ahat + b * N;
        double *cb = chat + b * N;
        cb[0] = 0.0;
        for (int64_t S = 1; S < N; ++S) {
            int64_t j = S & (-S);
            int64_t rest = S ^ j;
            double acc = fabs(ab[S]);
            if (rest != 0) {
                for (int64_t U = (rest - 1) & rest;; U = (U - 1) & rest) {
                    acc += cb[j | U] * fabs(ab[rest ^ U]);
                    if (U == 0) break;
                }
            }
            cb[S] = acc;
        }
    }
}

/* Set-partition (Moebius) route to the connected sums, independent of the
 * recursion: c[S] = sum over set partitions pi of S of
 * (-1)^{|pi|-1} (|pi|-1)! prod_{B in pi} a[B].
 * Partitions are generated element by element: each element of S joins one of
 * the blocks opened so far or opens a new one. */
static void partitions_rec(const double *a, const int *elems, int k, int pos, int64_t *blocks,
                           int nb, double *acc) {
    if (pos == k) {
        double prod = 1.0;
        for (int i = 0; i < nb; ++i) prod *= a[blocks[i]];
        double coef = 1.0;
        for (int i = 2; i < nb; ++i) coef *= (double)i; /* (nb-1)! */
        *acc += ((nb - 1) & 1) ? -coef * prod : coef * prod;
        return;
    }
    int64_t bit = (int64_t)1 << elems[pos];
    for (int i = 0; i < nb; ++i) {
        blocks[i] |= bit;
        partitions_rec(a, elems, k, pos + 1, blocks, nb, acc);
        blocks[i] &= ~bit;
    }
    blocks[nb] = bit;
    partitions_rec(a, elems, k, pos + 1, blocks, nb + 1, acc);
    blocks[nb] = 0;
}

void oracle_cdet_partition(const double *a, int n, int64_t batch, double *c, int nthreads) {
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads_for(nthreads))
    for (int64_t b = 0; b < batch; ++b) {
        const double *ab = a + b * N;
        double *cb = c + b * N;
        cb[0] = 0.0;
        for (int64_t S = 1; S < N; ++S) {
            int elems[MAXN];
            int64_t blocks[MAXN + 1];
            int k = 0;
            for (int e = 0; e < n; ++e)
                if ((S >> e) & 1) elems[k++] = e;
            memset(blocks, 0, sizeof(blocks));
            double acc = 0.0;
            partitions_rec(ab, elems, k, 0, blocks, 0, &acc);
            cb[S] = acc;
        }
    }
}

/* Real-time Keldysh sum (Section V.D): the 2n x 2n complex block matrix Mt has
 * the block of vertices (i,j) at rows 2i,2i+1 and columns 2j,2j+1 (row 2i+0 is
 * Keldysh index +, 2i+1 is -). For every assignment alpha in {+,-}^n the n x n
 * matrix (M_alpha)_ij = Mt[2i+alpha_i][2j+alpha_j] is built and its determinant
 * taken by its own complex partial-pivot elimination. With signed != 0 each
 * assignment is weighted by (-1)^{number of - indices}.
 *   sum[b]        = sum over alpha of (weight) det M_alpha          (complex)
 *   partial[b][d] = the same sum over the 2^d assignments of the first d
 *                   vertices of det of the leading d x d block (d = 0..n;
 *                   partial[.][0] = 1, partial[.][n] = sum). May be NULL.
 * Complex numbers are stored interleaved (re, im). */
void oracle_keldysh(const double *Mt, int n, int64_t batch, int signed_, double *sum,
                    double *partial, int nthreads) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads_for(nthreads))
    for (int64_t b = 0; b < batch; ++b) {
        const double complex *Mb = (const double complex *)Mt + b * (int64_t)(2 * n) * (2 * n);
        double complex M[MAXN * MAXN];
        for (int d = (partial ? 0 : n); d <= n; ++d) {
            double complex acc = 0.0;
            for (int64_t al = 0; al < ((int64_t)1 << d); ++al) {
                for (int i = 0; i < d; ++i)
                    for (int j = 0; j < d; ++j) {
                        int ri = 2 * i + (int)((al >> i) & 1);
                        int cj = 2 * j + (int)((al >> j) & 1);
                        M[i * d + j] = Mb[ri * (2 * n) + cj];
                    }
                double complex det = cdet_partial_pivot(M, d);
                if (signed_ && (popcount_u32((uint32_t)al) & 1)) det = -det;
                acc += det;
            }
            if (partial) {
                partial[(b * (n + 1) + d) * 2 + 0] = creal(acc);
                partial[(b * (n + 1) + d) * 2 + 1] = cimag(acc);
            }
            if (d == n) {
                sum[b * 2 + 0] = creal(acc);
                sum[b * 2 + 1] = cimag(acc);
            }
        }
    }
}

/* Error scale for the Keldysh sum: sum over alpha of perm(|M_alpha|) (the sum of
 * the absolute values of all Leibniz terms) when use_perm != 0, else the cheaper
 * bound sum over alpha of prod_i sum_j |(M_alpha)_ij|. perm by Ryser on |M_alpha|. */
void oracle_keldysh_scale(const double *Mt, int n, int64_t batch, int use_perm, double *scale,
                          int nthreads) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads_for(nthreads))
    for (int64_t b = 0; b < batch; ++b) {
        const double complex *Mb = (const double complex *)Mt + b * (int64_t)(2 * n) * (2 * n);
        double M[MAXN * MAXN];
        double acc = 0.0;
        for (int64_t al = 0; al < ((int64_t)1 << n); ++al) {
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    int ri = 2 * i + (int)((al >> i) & 1);
                    int cj = 2 * j + (int)((al >> j) & 1);
                    M[i * n + j] = cabs(Mb[ri * (2 * n) + cj]);
                }
            if (use_perm) {
                double total = 0.0;
                for (int64_t T = 0; T < ((int64_t)1 << n); ++T) {
                    double prod = 1.0;
                    for (int r = 0; r < n; ++r) {
                        double rs = 0.0;
                        for (int q = 0; q < n; ++q)
                            if ((T >> q) & 1) rs += M[r * n + q];
                        prod *= rs;
                    }
                    total += (popcount_u32((uint32_t)T) & 1) ? -prod : prod;
                }
                acc += (n & 1) ? -total : total;
            } else {
                double prod = 1.0;
                for (int r = 0; r < n; ++r) {
                    double rs = 0.0;
                    for (int q = 0; q < n; ++q) rs += M[r * n + q];
                    prod *= rs;
                }
                acc += prod;
            }
        }
        scale[b] = acc;
    }
}

/* All 2^n XNOR principal minors of each 2n x 2n matrix M (Section III.B): for
 * every vertex subset S, the determinant of the submatrix that keeps both rows
 * and both columns 2i, 2i+1 of each vertex i in S and none of the others, each
 * by its own partial-pivot elimination; minors[0] = 1. n <= 16. */
void oracle_xnor_minors(const double *M, int n, int64_t batch, double *minors, int nthreads) {
    const int m = 2 * n;
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads_for(nthreads))
    for (int64_t b = 0; b < batch; ++b) {
        const double *Mb = M + b * (int64_t)m * m;
        double *out = minors + b * N;
        double sub[32 * 32];
        int idx[32];
        for (int64_t S = 0; S < N; ++S) {
            int k = 0;
            for (int v = 0; v < n; ++v)
                if ((S >> v) & 1) {
                    idx[k++] = 2 * v;
                    idx[k++] = 2 * v + 1;
                }
            for (int r = 0; r < k; ++r)
                for (int q = 0; q < k; ++q) sub[r * k + q] = Mb[idx[r] * m + idx[q]];
            out[S] = det_partial_pivot(sub, k);
        }
    }
}

/* Rounding scale of each XNOR minor: perm(|M[S]|) of its 2|S| x 2|S| submatrix
 * (the sum of the absolute values of all Leibniz terms, by Ryser on the
 * absolute values) when use_perm != 0, else the bound prod_r sum_q |M_rq| over
 * the submatrix. scale[0] = 1. */
void oracle_xnor_scale(const double *M, int n, int64_t batch, int use_perm, double *scale, int nthreads) {
    const int m = 2 * n;
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads_for(nthreads))
    for (int64_t b = 0; b < batch; ++b) {
        const double *Mb = M + b * (int64_t)m * m;
        double *out = scale + b * N;
        double sub[32 * 32];
        int idx[32];
        for (int64_t S = 0; S < N; ++S) {
            int k = 0;
            for (int v = 0; v < n; ++v)
                if ((S >> v) & 1) {
                    idx[k++] = 2 * v;
                    idx[k++] = 2 * v + 1;
                }
            for (int r = 0; r < k; ++r)
                for (int q = 0; q < k; ++q) sub[r * k + q] = fabs(Mb[idx[r] * m + idx[q]]);
            double acc;
            if (use_perm) {
                double total = 0.0;
                for (int64_t T = 0; T < ((int64_t)1 << k); ++T) {
                    double prod = 1.0;
                    for (int r = 0; r < k; ++r) {
                        double rs = 0.0;
                        for (int q = 0; q < k; ++q)
                            if ((T >> q) & 1) rs += sub[r * k + q];
                        prod *= rs;
                    }
                    total += (popcount_u32((uint32_t)T) & 1) ? -prod : prod;
                }
                acc = (k & 1) ? -total : total;
            } else {
                acc = 1.0;
                for (int r = 0; r < k; ++r) {
                    double rs = 0.0;
                    for (int q = 0; q < k; ++q) rs += sub[r * k + q];
                    acc *= rs;
                }
            }
            out[S] = acc;
        }
    }
}

/* NAND principal minors of each 2n x 2n matrix M (Section III.C): for every
 * ternary assignment sigma (vertex i <-> base-3 digit i of the index: 0 keeps
 * neither row/column 2i nor 2i+1, 1 keeps row and column 2i, 2 keeps row and
 * column 2i+1), the determinant of the kept submatrix, each by its own
 * partial-pivot elimination. With out3 != NULL all 3^n minors are written
 * (out3[0] = 1); with abar != NULL, abar[S] = the sum of the minors of the
 * 2^|S| assignments whose kept vertices are exactly S (the weights of the CDet
 * summed over two vertex types, Section V.C); with scale != NULL, scale[S] =
 * the sum over the same assignments of prod_r sum_q |sub_rq| (a bound on the
 * absolute Leibniz terms). n <= 13. */
void oracle_nand(const double *M, int n, int64_t batch, double *out3, double *abar, double *scale,
                 int nthreads) {
    const int m = 2 * n;
    int64_t N3 = 1;
    for (int i = 0; i < n; ++i) N3 *= 3;
    const int64_t N = (int64_t)1 << n;
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads_for(nthreads))
    for (int64_t b = 0; b < batch; ++b) {
        const double *Mb = M + b * (int64_t)m * m;
        double sub[16 * 16];
        int idx[16];
        if (abar)
            for (int64_t S = 0; S < N; ++S) abar[b * N + S] = 0.0;
        if (scale)
            for (int64_t S = 0; S < N; ++S) scale[b * N + S] = 0.0;
        for (int64_t t = 0; t < N3; ++t) {
            int k = 0;
            int64_t S = 0, r3 = t;
            for (int v = 0; v < n; ++v, r3 /= 3) {
                const int dgt = (int)(r3 % 3);
                if (dgt) {
                    idx[k++] = 2 * v + (dgt - 1);
                    S |= (int64_t)1 << v;
                }
            }
            double bound = 1.0;
            for (int r = 0; r < k; ++r) {
                double rs = 0.0;
                for (int q = 0; q < k; ++q) {
                    sub[r * k + q] = Mb[idx[r] * m + idx[q]];
                    rs += fabs(sub[r * k + q]);
                }
                bound *= rs;
            }
            const double det = det_partial_pivot(sub, k);
            if (out3) out3[b * N3 + t] = det;
            if (abar) abar[b * N + S] += det;
            if (scale) scale[b * N + S] += bound;
        }
    }
}

/* Two-spin Keldysh sum (Section V.D with the two determinants of Eq. CTINT):
 * sum over the 2^n assignments alpha shared by both spins of
 * det(M_up,alpha) det(M_dn,alpha), each determinant by its own complex
 * partial-pivot elimination; partial[d] (if not NULL) is the same sum over the
 * first d vertices only (leading blocks), partial[0] = 1. signed_ weights each
 * assignment by (-1)^{number of - indices} once. */
void oracle_keldysh2(const double *Mu, const double *Md, int n, int64_t batch, int signed_, double *sum,
                     double *partial, int nthreads) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads_for(nthreads))
    for (int64_t b = 0; b < batch; ++b) {
        const double complex *U = (const double complex *)Mu + b * (int64_t)(2 * n) * (2 * n);
        const double complex *Dn = (const double complex *)Md + b * (int64_t)(2 * n) * (2 * n);
        double complex A[MAXN * MAXN], B[MAXN * MAXN];
        for (int d = (partial ? 0 : n); d <= n; ++d) {
            double complex acc = 0.0;
            for (int64_t al = 0; al < ((int64_t)1 << d); ++al) {
                for (int i = 0; i < d; ++i)
                    for (int j = 0; j < d; ++j) {
                        int ri = 2 * i + (int)((al >> i) & 1);
                        int cj = 2 * j + (int)((al >> j) & 1);
                        A[i * d + j] = U[ri * (2 * n) + cj];
                        B[i * d + j] = Dn[ri * (2 * n) + cj];
                    }
                double complex v = cdet_partial_pivot(A, d) * cdet_partial_pivot(B, d);
                if (signed_ && (popcount_u32((uint32_t)al) & 1)) v = -v;
                acc += v;
            }
            if (partial) {
                partial[(b * (n + 1) + d) * 2 + 0] = creal(acc);
                partial[(b * (n + 1) + d) * 2 + 1] = cimag(acc);
            }
            if (d == n) {
                sum[b * 2 + 0] = creal(acc);
                sum[b * 2 + 1] = cimag(acc);
            }
        }
    }
}

/* Error scale for the two-spin sum: sum over alpha of the product of the two
 * row-sum bounds prod_i sum_j |(M_sigma,alpha)_ij| (>= the absolute Leibniz
 * terms of the product of the two determinants). */
void oracle_keldysh2_scale(const double *Mu, const double *Md, int n, int64_t batch, double *scale,
                           int nthreads) {
#pragma omp parallel for schedule(dynamic, 1) num_threads(threads_for(nthreads))
    for (int64_t b = 0; b < batch; ++b) {
        const double complex *U = (const double complex *)Mu + b * (int64_t)(2 * n) * (2 * n);
        const double complex *Dn = (const double complex *)Md + b * (int64_t)(2 * n) * (2 * n);
        double acc = 0.0;
        for (int64_t al = 0; al < ((int64_t)1 << n); ++al) {
            double pu = 1.0, pd = 1.0;
            for (int i = 0; i < n; ++i) {
                double su = 0.0, sd = 0.0;
                const int ri = 2 * i + (int)((al >> i) & 1);
                for (int j = 0; j < n; ++j) {
                    const int cj = 2 * j + (int)((al >> j) & 1);
                    su += cabs(U[ri * (2 * n) + cj]);
                    sd += cabs(Dn[ri * (2 * n) + cj]);
                }
                pu *= su;
                pd *= sd;
            }
            acc += pu * pd;
        }
        scale[b] = acc;
    }
}
