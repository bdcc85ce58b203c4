/*
 * apm.h -- C ABI of the all-principal-minor library (libapm.so) for GB300.
 *
 * What the library computes (Simkovic & Ferrero, "Fast Principal Minor
 * Algorithms for Quantum Many Body Systems", arXiv:2104.07638):
 *   - all 2^n principal minors of n x n matrices by the Schur-complement tree
 *     with pivot correction (Section II, Eq. minor, Alg. 1);
 *   - the connected sums of the CDet recursion over all subsets (Section V.A,
 *     Eq. recursion), fused with the minors;
 *   - the real-time Keldysh sum over 2^n index assignments as the sum of XOR
 *     principal minors of the 2n x 2n block matrix (Sections III.D and V.D);
 *   - all 2^n permanent principal minors in O(3^n) (Section IV).
 *
 * Conventions shared by every call
 *   Subsets are bit masks: element k (0-based) <-> bit k, so an array indexed by
 *   mask S in [0, 2^n) holds the value for the subset S (Section II labels the
 *   subset S_i by the binary digits of i). minors[0] = det(empty) = 1,
 *   perms[0] = 1, c[0] = 0.
 *   Matrices are row-major and stored back to back ("batch-major"): matrix b of a
 *   fixed-order batch starts at element b*n*n.
 *   All data pointers are DEVICE pointers owned by the caller, 16-byte aligned.
 *   The library allocates no device memory in any call: where scratch is needed
 *   the caller passes it (apm_workspace_size tells how much).
 *   Calls are asynchronous on `stream` (NULL = the legacy default stream).
 *   Argument errors are detected on the host, before any launch, and return
 *   APM_ERR_ARG / APM_ERR_UNSUPPORTED_N / APM_ERR_WORKSPACE with nothing written.
 *   A launch failure returns APM_ERR_CUDA (apm_last_cuda_error gives the code).
 *   Numerical trouble never aborts a launch: it sets bits in the optional
 *   per-matrix `status` array (device memory, one uint32 per matrix, written by
 *   every call that takes it) and, where the result cannot be trusted, fills that
 *   matrix's outputs with NaN. apm_status_reduce() collects the bits on the host.
 */
#ifndef APM_H
#define APM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A cudaStream_t. */
typedef struct CUstream_st *apm_stream_t;

typedef enum {
    APM_OK = 0,
    APM_ERR_ARG = 1,            /* null/misaligned pointer, negative batch, bad flags */
    APM_ERR_UNSUPPORTED_N = 2,  /* order outside the supported range of the call */
    APM_ERR_CUDA = 3,           /* a CUDA runtime call or launch failed */
    APM_ERR_NUMERIC = 4,        /* apm_status_reduce: some matrix has an error bit */
    APM_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
    APM_ERR_WORKSPACE = 6       /* scratch missing or smaller than apm_workspace_size */
} apm_status_t;

/* Per-matrix status bits. */
#define APM_ST_PIVOT_CORRECTED     0x01u /* a pivot correction was applied and back-propagated */
#define APM_ST_NONFINITE_INPUT     0x02u /* the input held a NaN or an infinity */
#define APM_ST_ZERO_PIVOT          0x04u /* Keldysh, XNOR, NAND: a zero or non-finite pivot; outputs NaN */
#define APM_ST_CORRECTION_OVERFLOW 0x08u /* more pivot corrections than the per-matrix records
                                            hold (256 for the FPM tree); outputs set to NaN */
#define APM_ST_BAD_ORDER           0x10u /* uneven batch: order outside 1..n_max; matrix skipped */
#define APM_ST_ERROR_MASK          (APM_ST_NONFINITE_INPUT | APM_ST_ZERO_PIVOT | APM_ST_CORRECTION_OVERFLOW | \
                                    APM_ST_BAD_ORDER)

/* Largest supported orders. */
#define APM_MAX_N_MINORS   16
#define APM_MAX_N_ALL_MINORS 24 /* apm_all_minors alone (2^24 minors per matrix) */
#define APM_MAX_N_KELDYSH  16
#define APM_MAX_N_PERM     16
#define APM_MAX_N_XNOR     16
#define APM_MAX_N_NAND_MINORS 13 /* 3^n doubles per matrix */
#define APM_MAX_N_TWO_TYPE 16

/*
 * Pivot correction (Section II, the paragraph after Eq. minor and Alg. 1): when
 * a pivot p of the Schur-complement tree satisfies |p| <= piv_threshold*||A||max
 * it is replaced by p + C with C = sign(p)*piv_shift*||A||max (sign(0) = +1),
 * the node's minor is stored with the shifted pivot, and after the tree the
 * shift is removed exactly by det(A[S]) = det(A~[S]) - C det(A[S \ {l}]),
 * applied to the node's whole right subtree, deepest level first; the node's
 * own minor is written as det(A[S \ {l}]) p with the unshifted pivot.
 * Any choice gives the same exact result; the threshold trades stability. An
 * uncorrected pivot p amplifies the rounding of the minors below it by about
 * ||A||max / |p|, so the default 1e-4 keeps that factor under 10^4 (about
 * 2e-12 relative to the sum of absolute terms); the minors of the Hubbard
 * Green's-function matrices of Section V meet no pivot below 1e-2 ||A||max.
 * NULL selects the defaults below (||A||max = 0 is treated as 1).
 */
typedef struct {
    double piv_threshold; /* default 1e-4 */
    double piv_shift;     /* default 1.0 */
} apm_pivot_opts;

#define APM_DEFAULT_PIV_THRESHOLD 1e-4
#define APM_DEFAULT_PIV_SHIFT 1.0

/*
 * apm_all_minors -- all 2^n principal minors of each matrix.
 * Section II (Eq. dets_schur, Eq. lemma1/lemma2, Eq. minor, Alg. 1): the minor of
 * subset S_i is the minor of S_i \ {l} times the (1,1) entry of the Schur
 * complement reached along the tree path of S_i.
 *   A       [batch][n][n] float64, input.
 *   n       1..APM_MAX_N_ALL_MINORS.
 *   batch   >= 0 (0 launches nothing).
 *   minors  [batch][2^n] float64, output, minors[b][S] = det(A_b[S]).
 *   opt     pivot-correction options or NULL.
 *   status  [batch] uint32 or NULL.
 *   workspace / workspace_bytes: scratch for n >= 9 (see apm_workspace_size),
 *           256-byte aligned; may be NULL/0 for n <= 8.
 * For n = 9..16 one warp takes a matrix (elements decided from the last one
 * down: above the last 12 depth first, then 5 levels breadth first in shared
 * memory, then each lane finishes one of the 32 nodes left, in registers, down
 * to 3 x 3 nodes whose 8 minors it writes in closed form); it shifts no pivot, and the matrices that meet a pivot with |p| <= piv_threshold
 * ||A||max are computed again, with the correction, by the one-CTA-per-matrix
 * kernel of apm_cdet_connected, launched after it on those matrices only.
 * For n = 17..24 the tree is cut in two: its upper n - 12 levels (elements n-1
 * down to 12) run breadth first over the batch, one launch per level, and each
 * of the 2^(n-12) leaves, the 12 x 12 Schur complement M_T of the kept upper
 * set T, goes through the n = 12 path above, whose 4096 minors fill the row at
 * T * 4096 and are scaled by det(A[T]): det(A[T u U]) = det(A[T]) det(M_T[U]).
 * Upper-level pivots are corrected as above (at most 256 per matrix, more set
 * APM_ST_CORRECTION_OVERFLOW), and so are the leaves' own: threshold and shift
 * of both are relative to ||A||max of the whole matrix (a leaf's entries can be
 * inflated by a small upper pivot; its pivots are pivots of the same tree). An
 * error bit anywhere makes the matrix's whole row NaN.
 */
apm_status_t apm_all_minors(const double *A, int n, int64_t batch, double *minors,
                            const apm_pivot_opts *opt, uint32_t *status, void *workspace,
                            size_t workspace_bytes, apm_stream_t stream);

/* flags for apm_cdet_connected */
#define APM_CDET_SINGLE_DET 0x1 /* a[S] = det(A_up[S]) instead of det(A_up[S]) det(A_dn[S]) */

/*
 * apm_cdet_connected -- connected sums c[S] for all subsets S, fused with the
 * minors that define the weights.
 * Section V.A: a[S] = det(M_up[S]) det(M_dn[S]); Eq. recursion:
 *     c[S] = a[S] - sum_{T proper subset of S, j in T} c[T] a[S \ T],
 * with j = the lowest element of S (the paper lets j be any element of S).
 *   A_up       [batch][n][n] float64.
 *   A_dn       [batch][n][n] float64 or NULL; NULL means the spin-symmetric case
 *              M_dn = M_up, so a[S] = det(A_up[S])^2.
 *   flags      0 or APM_CDET_SINGLE_DET (then A_dn must be NULL).
 *   c          [batch][2^n] float64 output.
 *   minors_out [batch][2^n] float64 (minors of A_up) or NULL; when A_dn is given,
 *              [batch][2][2^n] (minors of A_up, then of A_dn).
 *   opt, status, workspace: as for apm_all_minors (for n = 16 the workspace
 *              also holds the ranked arrays below: apm_workspace_size with
 *              APM_OP_CDET).
 * At n = 16 the connected sums come from the same weights by the fast subset
 * convolution of apm_cdet_from_weights_fsc (a second launch on `stream`, in
 * place on c), which is faster there; the results agree with the recursion up
 * to rounding.
 * For n >= 13 with A_dn NULL the minors come first from the one-warp-per-matrix
 * tree of apm_all_minors (a launch on `stream` before the fused kernel, writing
 * them to minors_out, or to c when minors_out is NULL); the fused kernel forms
 * the weights from them and computes the tree itself, with the pivot
 * correction, only for the matrices that tree flagged (a pivot at or below the
 * threshold, a non-finite entry). The workspace then also holds one flag byte
 * per matrix (apm_workspace_size with APM_OP_CDET includes it).
 */
apm_status_t apm_cdet_connected(const double *A_up, const double *A_dn, int n, int64_t batch,
                                int flags, double *c, double *minors_out,
                                const apm_pivot_opts *opt, uint32_t *status, void *workspace,
                                size_t workspace_bytes, apm_stream_t stream);

/* Most streams apm_cdet_connected_host runs its chunks on. */
#define APM_HOST_MAX_STREAMS 8

/*
 * apm_cdet_connected_host -- apm_cdet_connected (Section V.A, Eq. recursion:
 * the same arithmetic, bit for bit) on matrices and outputs in HOST memory. The
 * transfer pipeline has no counterpart in the paper: the batch is cut into
 * chunks of `chunk` matrices (the last two chunks' worth into halving pieces,
 * down to chunk/16, so that the copy-out left exposed at the end is short)
 * that go in turn to `nstreams` slots of the device workspace, each with a
 * stream the call creates; a slot copies its chunk in, runs the kernels of
 * apm_cdet_connected on it and copies the outputs back, so the copies of one
 * chunk overlap the kernels of the others. The kernels
 * only ever touch device memory. The exceptions to the conventions at the top
 * of this header: A_up, A_dn, c, minors_out and status are host pointers (any
 * alignment), and the call is blocking.
 *   A_up, A_dn, n, batch, flags, opt: as apm_cdet_connected (host memory).
 *   c, minors_out, status: host outputs, laid out as apm_cdet_connected's.
 *   chunk      matrices per chunk, >= 1 (a value above batch acts as batch).
 *   nstreams   1..APM_HOST_MAX_STREAMS.
 *   workspace  device memory of the current device, 256-byte aligned, at least
 *              apm_cdet_connected_host_workspace_size(n, chunk, nstreams,
 *              A_dn != NULL) bytes: per slot the chunk's inputs, outputs and
 *              status words and the kernels' scratch.
 *   stream     work already queued on it is complete before the call touches
 *              the workspace (NULL = the legacy default stream).
 * Page-locked host memory (cudaHostAlloc, cudaHostRegister) lets the copies
 * run asynchronously; pageable memory gives the same results with the copies
 * serialised. Returns when every output is in host memory. Argument errors
 * return before any copy; a CUDA error stops the pipeline, waits for the work
 * already issued and returns APM_ERR_CUDA (outputs then partly written).
 */
apm_status_t apm_cdet_connected_host(const double *A_up, const double *A_dn, int n, int64_t batch,
                                     int flags, double *c, double *minors_out,
                                     const apm_pivot_opts *opt, uint32_t *status, int64_t chunk,
                                     int nstreams, void *workspace, size_t workspace_bytes,
                                     apm_stream_t stream);

/* Device workspace bytes of apm_cdet_connected_host for these arguments
 * (two_mats: 1 when A_dn is given). */
apm_status_t apm_cdet_connected_host_workspace_size(int n, int64_t chunk, int nstreams, int two_mats,
                                                    size_t *bytes);

/*
 * apm_cdet_from_weights -- the CDet recursion (Eq. recursion) applied to given
 * weights a[S] (e.g. permanent minors for the bosonic connected sum of
 * Section V.F, or products of two minor arrays).
 *   a  [batch][2^n] float64 input (a[0] is ignored).   c  [batch][2^n] output.
 */
apm_status_t apm_cdet_from_weights(const double *a, int n, int64_t batch, double *c,
                                   void *workspace, size_t workspace_bytes, apm_stream_t stream);

/*
 * apm_cdet_from_weights_fsc -- the same connected sums as apm_cdet_from_weights,
 * by the fast subset convolution the paper mentions for Eq. recursion
 * (Section V.A, O(n^2 2^n) instead of O(3^n)): ranked zeta transform of a
 * (a[0] taken as 1), logarithm of the power series in the rank variable at
 * every mask, ranked Mobius transform, c[S] read at rank |S|. Results agree
 * with the recursion up to rounding (a different order of operations).
 *   a  [batch][2^n] float64 input (a[0] is ignored).   c  [batch][2^n] output.
 *   n  1..APM_MAX_N_MINORS.
 *   workspace  apm_workspace_size(APM_OP_CDET_FSC, n, batch): the ranked arrays
 *              (n 2^n doubles per resident CTA) for n > 9, none below.
 */
apm_status_t apm_cdet_from_weights_fsc(const double *a, int n, int64_t batch, double *c, void *workspace,
                                       size_t workspace_bytes, apm_stream_t stream);

/*
 * apm_xnor_minors -- all 2^n XNOR principal minors of 2n x 2n matrices made of
 * 2 x 2 blocks (Section III.B): minors[S] = det of the submatrix that keeps both
 * rows and both columns 2i, 2i+1 of every vertex i in S and none of the others;
 * minors[0] = 1. Binary tree of Schur complements with respect to 2 x 2 pivot
 * blocks, O(2^n); no pivot correction is possible (Section III.B).
 *   M        [batch][2n][2n] float64, row-major; block (i, j) at rows 2i, 2i+1
 *            and columns 2j, 2j+1.
 *   n        1..APM_MAX_N_XNOR.
 *   minors   [batch][2^n] float64 output.
 *   status   [batch] or NULL; APM_ST_ZERO_PIVOT marks a singular or non-finite
 *            2 x 2 pivot block met on the way, APM_ST_NONFINITE_INPUT a NaN or
 *            infinity in the input; either makes that matrix's row NaN.
 *   workspace / workspace_bytes: scratch for the depth-first part of the tree,
 *            needed for n > 9 (apm_workspace_size with APM_OP_XNOR_MINORS).
 */
apm_status_t apm_xnor_minors(const double *M, int n, int64_t batch, double *minors, uint32_t *status,
                             void *workspace, size_t workspace_bytes, apm_stream_t stream);

/*
 * apm_nambu_cdet -- the CDet connected sums for expansions around BCS theory
 * (Section V.B): the weights a[S] are the XNOR minors of the 2n x 2n Nambu
 * matrix (apm_xnor_minors, written to minors), and c[S] follows from them by
 * the CDet recursion (Eq. recursion), exactly as apm_cdet_from_weights.
 *   minors   [batch][2^n] float64 output (the weights), c [batch][2^n] output.
 *   Other arguments as for apm_xnor_minors; the workspace size is
 *   apm_workspace_size with APM_OP_NAMBU_CDET (zero for n <= 9).
 */
apm_status_t apm_nambu_cdet(const double *M, int n, int64_t batch, double *minors, double *c, uint32_t *status,
                            void *workspace, size_t workspace_bytes, apm_stream_t stream);

/*
 * apm_nand_minors -- all 3^n NAND principal minors of 2n x 2n matrices made of
 * 2 x 2 blocks (Section III.C): for every ternary assignment sigma (vertex i <->
 * base-3 digit i of the index: 0 keeps neither row/column 2i nor 2i+1, 1 keeps
 * row and column 2i, 2 keeps row and column 2i+1) the determinant of the kept
 * submatrix; minors3[0] = 1. Ternary tree of Schur complements with scalar
 * pivots, O(3^n), with the pivot correction the paper allows here (Section
 * III.C: as in the FPM tree, back-propagated at the end): a pivot p with
 * |p| <= piv_threshold ||M||max becomes p + C, C = sign(p) piv_shift ||M||max,
 * and afterwards det(M[S]) = det(M~[S]) - C det(M[S \ {row}]) is applied over
 * the kept child's subtree, deepest vertex first.
 *   M        [batch][2n][2n] float64, row-major.
 *   n        1..APM_MAX_N_NAND_MINORS.
 *   minors3  [batch][3^n] float64 output.
 *   opt      pivot-correction options or NULL (the defaults of apm_pivot_opts).
 *   status   [batch] or NULL; APM_ST_PIVOT_CORRECTED when a pivot was shifted;
 *            APM_ST_ZERO_PIVOT (a zero or non-finite pivot left after the
 *            shift), APM_ST_NONFINITE_INPUT, or APM_ST_CORRECTION_OVERFLOW
 *            (more than 256 corrected pivots above the last 6 vertices) make
 *            that matrix's row NaN.
 *   workspace / workspace_bytes: per resident warp the depth-first part of the
 *            tree and the correction records (apm_workspace_size with
 *            APM_OP_NAND_MINORS; needed for every n).
 */
apm_status_t apm_nand_minors(const double *M, int n, int64_t batch, double *minors3, const apm_pivot_opts *opt,
                             uint32_t *status, void *workspace, size_t workspace_bytes, apm_stream_t stream);

/*
 * apm_two_type_cdet -- the CDet summed over two vertex types (Section V.C):
 * abar[S] = the sum over the 2^|S| type assignments of the vertices of S of the
 * NAND minors (apm_nand_minors), abar[0] = 1, then c[S] from abar by the CDet
 * recursion (Eq. recursion; summing over types block by block is exact because
 * the recursion is a sum over set partitions of products of block weights).
 *   abar, c  [batch][2^n] float64 outputs.   n  1..APM_MAX_N_TWO_TYPE.
 *   Other arguments as for apm_nand_minors (corrections above the last 6
 *   vertices enter the sums through a list of at most 16 target sets per tree
 *   path; more set APM_ST_CORRECTION_OVERFLOW); workspace: apm_workspace_size
 *   with APM_OP_TWO_TYPE_CDET.
 */
apm_status_t apm_two_type_cdet(const double *M, int n, int64_t batch, double *abar, double *c,
                               const apm_pivot_opts *opt, uint32_t *status,
                               void *workspace, size_t workspace_bytes, apm_stream_t stream);

/* flags for apm_keldysh_sum and apm_keldysh_sum_noalloc */
#define APM_KELDYSH_SIGNED 0x1 /* weight each assignment by (-1)^{number of - indices} */

/*
 * apm_keldysh_sum -- sum over all 2^n Keldysh index assignments alpha of
 * det[G^{alpha_i alpha_j}(X_i - X_j)] (Section V.D), computed as the sum of the
 * XOR principal minors of the 2n x 2n block matrix (Section III.D) by a binary
 * tree of Schur complements in O(2^n); no pivot correction is possible there.
 *   Mt       [batch][2n][2n] complex128, interleaved (re, im); the 2x2 block of
 *            vertices (i, j) is at rows 2i (index +), 2i+1 (index -) and columns
 *            2j, 2j+1.
 *   n        1..APM_MAX_N_KELDYSH.
 *   flags    0 or APM_KELDYSH_SIGNED.
 *   sum      [batch][2] float64 output (re, im).
 *   partial  [batch][n+1][2] float64 or NULL: partial[b][d] = the same sum over
 *            the first d vertices only (the lower orders obtained on the way,
 *            Section V.D); partial[b][0] = 1, partial[b][n] = sum[b].
 *   status   [batch] or NULL; APM_ST_ZERO_PIVOT marks a zero or non-finite pivot,
 *            and then sum (and partial) of that matrix are NaN.
 *   workspace / workspace_bytes: scratch for the depth-first part of the tree,
 *            needed for n > 8 (apm_workspace_size with APM_OP_KELDYSH says how
 *            much): the per-warp path matrices and, when the batch is too
 *            small to occupy every warp, one slot of n+1 sums per chunk of a
 *            matrix (the matrix's leaves are then split over several warps and
 *            the chunks added in a fixed order, so results stay reproducible).
 */
apm_status_t apm_keldysh_sum(const double *Mt, int n, int64_t batch, int flags, double *sum,
                             double *partial, uint32_t *status, void *workspace,
                             size_t workspace_bytes, apm_stream_t stream);

/*
 * apm_keldysh2_sum -- the Keldysh sum for two spins under one shared assignment
 * (Section V.D with the two determinants per configuration of Eq. CTINT):
 *   sum[b] = sum over alpha in {+,-}^n of det(Mu_b,alpha) det(Md_b,alpha),
 * one binary tree of Schur complements walked for both matrices at once.
 *   Mu, Md   [batch][2n][2n] complex128 each (up and down spin), laid out as
 *            for apm_keldysh_sum.
 *   n        1..APM_MAX_N_KELDYSH.     flags  0 or APM_KELDYSH_SIGNED (the
 *            weight (-1)^{number of -} is applied once per assignment).
 *   sum      [batch][2] float64 output; partial [batch][n+1][2] or NULL: the same
 *            sum over the first d vertices (the lower orders), partial[b][0] = 1.
 *   status   [batch] or NULL; APM_ST_ZERO_PIVOT marks a zero or non-finite pivot
 *            in either spin, and then that pair's results are NaN.
 *   workspace / workspace_bytes: scratch for the depth-first part (both spins'
 *            path matrices), needed for n > 7 (apm_workspace_size with
 *            APM_OP_KELDYSH2).
 */
apm_status_t apm_keldysh2_sum(const double *Mu, const double *Md, int n, int64_t batch, int flags, double *sum,
                              double *partial, uint32_t *status, void *workspace, size_t workspace_bytes,
                              apm_stream_t stream);

/*
 * apm_keldysh_sum_noalloc -- the same sum as apm_keldysh_sum, for callers that
 * cannot allocate device memory around the call: programs that hand all device
 * memory to their own pool allocator and forbid cudaMalloc inside their
 * Monte Carlo step (cudaMalloc can synchronise the device, and fails once the
 * pool owns the memory), and plugin hosts that only pass device pointers in.
 * There is no counterpart in the paper; it is a packaging of the same kernel.
 *   Instead of a caller workspace, the depth-first stack uses a fixed array in
 *   device memory that belongs to the library: 600 warp slots (50 CTAs of 12
 *   warps) for orders up to 14, 26.1 MB, held on every GPU that loads the
 *   library until the process exits; matrices are never split over warps here. Orders above 14 are rejected with APM_ERR_UNSUPPORTED_N (use
 *   apm_keldysh_sum with a workspace). The call allocates nothing.
 *   The first call on a device, even one with batch 0, looks up the array's
 *   device address (once per device, with that device current), which also
 *   loads the library's device code, array included, if lazy module loading
 *   has not yet done so; make that first call before any stream capture and
 *   before a pool allocator takes the device's free memory. The address is kept
 *   for the life of the process: after cudaDeviceReset on that device (which
 *   destroys the context the array lived in) this entry point must not be
 *   called again. Every call shares the one array: calls that overlap on the GPU (for
 *   example on two streams) race and give wrong results; serialise them. The
 *   array keeps whatever the last call left there; nothing in it needs to start
 *   at zero, because every entry is written before it is read.
 *   Arguments and results as for apm_keldysh_sum (n in 1..14).
 */
apm_status_t apm_keldysh_sum_noalloc(const double *Mt, int n, int64_t batch, int flags, double *sum,
                                     double *partial, uint32_t *status, apm_stream_t stream);

/*
 * apm_perm_minors -- all 2^n permanent principal minors perm(A[S]) in O(3^n)
 * (Section IV): for every column subset T the row sums r_i(T) = sum_{j in T} A_ij,
 * the products over supersets S of T built one element at a time, and
 *     perm(A[S]) = (-1)^|S| sum_{T subset of S} (-1)^|T| prod_{i in S} r_i(T).
 *   A      [batch][n][n] float64.    perms  [batch][2^n] float64 output.
 *   n      1..APM_MAX_N_PERM.
 *   workspace / workspace_bytes: unused (pass NULL, 0); kept for a uniform
 *          signature with the other batched calls.
 *   The output rows double as accumulators; the summation order is fixed, so
 *   repeated calls give bit-identical results.
 */
apm_status_t apm_perm_minors(const double *A, int n, int64_t batch, double *perms,
                             void *workspace, size_t workspace_bytes, apm_stream_t stream);

/* operation codes for apm_workspace_size */
#define APM_OP_ALL_MINORS 1
#define APM_OP_CDET 2
#define APM_OP_CDET_FROM_WEIGHTS 3
#define APM_OP_PERM_MINORS 4
#define APM_OP_CDET_VARLEN 5
#define APM_OP_KELDYSH 6
#define APM_OP_KELDYSH_VARLEN 7
#define APM_OP_XNOR_MINORS 8
#define APM_OP_NAMBU_CDET 9
#define APM_OP_NAND_MINORS 10
#define APM_OP_TWO_TYPE_CDET 11
#define APM_OP_KELDYSH2 12
#define APM_OP_CDET_FSC 13

/*
 * apm_cdet_connected_varlen -- apm_cdet_connected for a batch of matrices of
 * uneven orders in one persistent launch (no counterpart in the paper; the
 * per-matrix arithmetic is that of apm_cdet_connected, bit for bit).
 *   A       packed input matrices; matrix b is n[b] x n[b] row-major at A + a_off[b].
 *   A_dn    NULL, or packed like A (same offsets) for a separate second matrix.
 *   a_off   [batch] int64 element offsets.     n  [batch] int32 orders in 1..n_max.
 *   n_max   largest order present (1..16); sizes the scratch.
 *   flags   as apm_cdet_connected.
 *   c       packed outputs: c[S] of matrix b at c + c_off[b] (2^n[b] doubles).
 *   minors_out NULL or packed like c (with A_dn: 2 x 2^n[b] doubles at 2*c_off[b]).
 *   c_off   [batch] int64 element offsets (multiples of 2 for 16-byte alignment).
 *   workspace  apm_workspace_size(APM_OP_CDET_VARLEN, n_max, batch, two_mats).
 * Scheduling: a one-block counting sort puts the matrices in decreasing order
 * of n (longest first) into the workspace; every CTA then takes the next matrix
 * from a global counter (an atomic increment, no waiting). Orders up to 12 keep
 * a[] and c[] in shared memory, larger ones in the CTA's slot of the workspace.
 * The lane-group mapping per order is the one installed by apm_cdet_tune_set.
 * Order-16 matrices (the first ones of that order, counted by the sort) leave
 * their weights in c and a third launch finishes them in place by the fast
 * subset convolution, as apm_cdet_connected does at n = 16. Without A_dn, the
 * matrices of orders 13..16 take their minors, as apm_cdet_connected does, from
 * one warp-per-matrix launch per order before the persistent kernel.
 * A matrix whose n[b] is outside 1..n_max is skipped with APM_ST_BAD_ORDER.
 * The call allocates nothing and does not synchronise: it can be captured in a
 * CUDA graph once the first (non-captured) call on the device has run.
 */
apm_status_t apm_cdet_connected_varlen(const double *A, const double *A_dn, const int64_t *a_off,
                                       const int32_t *n, int64_t batch, int n_max, int flags, double *c,
                                       double *minors_out, const int64_t *c_off,
                                       const apm_pivot_opts *opt, uint32_t *status, void *workspace,
                                       size_t workspace_bytes, apm_stream_t stream);

/*
 * apm_keldysh_sum_varlen -- apm_keldysh_sum for uneven orders in one launch,
 * longest first (same scheduling as apm_cdet_connected_varlen).
 *   Mt       packed complex128 matrices, matrix b (2n[b] x 2n[b]) at Mt + 2*m_off[b]
 *            doubles (m_off counts complex entries).
 *   sum      [batch][2].   partial  NULL or [batch][17][2] (entries 0..n[b] used).
 *   workspace  apm_workspace_size(APM_OP_KELDYSH_VARLEN, n_max, batch, 0).
 */
apm_status_t apm_keldysh_sum_varlen(const double *Mt, const int64_t *m_off, const int32_t *n, int64_t batch,
                                    int n_max, int flags, double *sum, double *partial, uint32_t *status,
                                    void *workspace, size_t workspace_bytes, apm_stream_t stream);

/*
 * apm_cdet_tune_set -- install per-order lane-group tables for the connected-sum
 * recursion (found by an autotuner; no counterpart in the paper). table[n] for
 * n = 0..16 packs, for each popcount layer k, 3 bits at bit 3k: log2 of the number
 * of lanes that share one set S (0..5, at most k-1). An entry 0 (or table NULL)
 * restores the built-in cost model. Used by every later fixed-order and uneven
 * launch in this process. Returns APM_ERR_ARG for an invalid entry.
 * apm_cdet_tune_get -- the table in effect for order n.
 */
apm_status_t apm_cdet_tune_set(const uint64_t *table);
apm_status_t apm_cdet_tune_get(int n, uint64_t *packed);

/*
 * apm_tune_options_set -- the other knobs an autotuner sets (no counterpart in
 * the paper; process-wide, for every device):
 *   fsc_from_n        orders >= this take their connected sums through the fast
 *                     subset convolution instead of the recursion, in
 *                     apm_cdet_connected and apm_cdet_connected_varlen: 13..16,
 *                     17 for never, 0 for the default 16.
 *   cdet_ctas_per_sm  resident CTAs per SM of the persistent uneven-batch kernel
 *                     of apm_cdet_connected_varlen: 1..3, 0 for as many as fit (3).
 *   keldysh_warps     warps per CTA of apm_keldysh_sum_varlen: 4..12, 0 for 12
 *                     (fewer warps per CTA let more CTAs share an SM).
 * Workspace sizes depend on the first two: query apm_workspace_size after
 * setting them (a smaller workspace than the options need is rejected with
 * APM_ERR_WORKSPACE). Results differ between hand-off orders by rounding only.
 * Returns APM_ERR_ARG for values out of range (nothing is changed then).
 */
apm_status_t apm_tune_options_set(int fsc_from_n, int cdet_ctas_per_sm, int keldysh_warps);
apm_status_t apm_tune_options_get(int *fsc_from_n, int *cdet_ctas_per_sm, int *keldysh_warps);

/* ------------------------------------------------------------------------
 * Learned Monte Carlo proposal (no counterpart in the paper: the paper's
 * Monte Carlo context is the power series of Section V, Eq. series, sampled
 * over vertex configurations with single-vertex moves, Section V.E).
 *
 * Walkers: X is [W][n][3] int32 vertices (x, y, m): a site of a win x win window
 * and an imaginary-time grid index m in [0, mtau). The weight of a walker is
 * |c_n(X)|, the full-set connected sum of apm_cdet_connected on the matrix
 * M_ij = G0(r_i - r_j, tau_i - tau_j) built by apm_mc_build_matrices.
 * Uniform random numbers are inputs (generated by the caller).
 * ------------------------------------------------------------------------ */

/* Xp = X with, for each walker w, vertex floor(u[w][0] n) redrawn uniformly
 * from (u[w][1], u[w][2], u[w][3]). u: [W][4] float in [0,1). */
apm_status_t apm_mc_propose(const int32_t *X, int W, int n, int win, int mtau, const float *u, int32_t *Xp,
                            apm_stream_t stream);

/* A[k] (n x n, FP64) = G0 matrix of walker idx[k] (idx NULL: walker k), k < count:
 * A_ij = g0[|x_i-x_j|][|y_i-y_j|][m_i - m_j + mtau - 1]; g0 is [win][win][2 mtau - 1]
 * FP64 (the table value at m_i = m_j is the tau -> 0^- limit). */
apm_status_t apm_mc_build_matrices(const int32_t *X, const int32_t *idx, int count, int n, int win, int mtau,
                                   const double *g0, double *A, apm_stream_t stream);

/* Network inputs F [Bp][64] BF16 (raw uint16 storage) of walkers idx[k] (or k),
 * k < count; rows count..Bp-1 are zero. Vertices sorted by time, shifted by the
 * first, scaled by 1/win and 1/mtau: 3 values per vertex in 14 slots (0..41),
 * n/14 (42), then in 14 slots (43..56) the ascending values of
 * 0.25 log10 sum_{j != i} |G0(X_i - X_j)| (g0 table as above). n <= 14. */
apm_status_t apm_mc_features(const int32_t *X, const int32_t *idx, int count, int n, int win, int mtau,
                             const double *g0, uint16_t *F, int Bp, apm_stream_t stream);

/* Delayed acceptance, stage 1: walker w survives with probability
 * min(1, exp(s_new[w] - s_old[w])) (u1[w] uniform); the survivors' indices are
 * appended to idx (order unspecified) and their number written to *count
 * (device int32, zeroed by the call). */
apm_status_t apm_mc_stage1(const float *s_new, const float *s_old, const float *u1, int W, int32_t *idx,
                           int32_t *count, apm_stream_t stream);

/* Acceptance of the exactly evaluated candidates k < count (walker idx[k], or k
 * when idx is NULL); c_full[k*stride] is the proposal's exact connected sum.
 * Plain Metropolis (s_new NULL): accept if u2[w] < |c|/weight[w]. Delayed
 * acceptance, stage 2: accept if u2[w] < |c| exp(s_cur[w]) / (weight[w] exp(s_new[w])).
 * On acceptance X[w] = Xp[w], weight[w] = |c|, sign[w] = sign(c), s_cur[w] = s_new[w],
 * and *accepted (device int32) is incremented. */
apm_status_t apm_mc_accept(int32_t *X, const int32_t *Xp, double *weight, double *sign, float *s_cur,
                           const float *s_new, const double *c_full, int64_t stride, const int32_t *idx, int count,
                           const float *u2, int n, int32_t *accepted, apm_stream_t stream);

/* Surrogate network: in 64 -> 256 -> 256 -> 256 -> 1 with ReLU, BF16 weights
 * and activations, FP32 accumulation (tcgen05 tensor-core GEMMs fed by TMA),
 * FP32 master weights and Adam moments. Parameter layout (APM_MLP_PARAMS floats):
 * W1 [256][64], b1 [256], W2 [256][256], b2, W3 [256][256], b3, w4 [256], b4 [1],
 * 7 floats padding; weight matrices stored [out][in]. All buffers device memory
 * owned by the caller. */
#define APM_MLP_IN 64
#define APM_MLP_HIDDEN 256
#define APM_MLP_PARAMS 148488
typedef struct {
    float *param;          /* [APM_MLP_PARAMS] FP32 master copy */
    uint16_t *param_bf16;  /* [APM_MLP_PARAMS] BF16 copy read by the forward pass */
    float *grad;           /* [APM_MLP_PARAMS] */
    float *adam_m;         /* [APM_MLP_PARAMS] */
    float *adam_v;         /* [APM_MLP_PARAMS] */
} apm_mlp;

/* scratch for a batch of batch_padded rows (a multiple of 64). Its first four
 * bytes are a status word that the GEMMs OR flags into: zero them before the
 * first use (apm_mlp_status reads and clears them). */
apm_status_t apm_mlp_workspace_size(int batch_padded, size_t *bytes);
/* Synchronises `stream`, stores the workspace's status word in *flags (host,
 * nullable) and clears it. Bit 0: a bounded wait inside a tensor-core GEMM gave
 * up after one second (its tile was not written); returns APM_ERR_TIMEOUT then,
 * else APM_OK. */
apm_status_t apm_mlp_status(void *workspace, size_t workspace_bytes, uint32_t *flags, apm_stream_t stream);
/* The network's GEMM on its own: C[M][N] = A[M][K] * Bt[N][K]^T (+ bias[N])
 * (ReLU if relu), BF16 operands (K contiguous in both), FP32 accumulation;
 * writes C32 (FP32) and/or Cb (BF16) when not NULL. N and K multiples of 64,
 * M >= 1, every pointer 16-byte aligned device memory; the workspace is one
 * sized for any batch (its status word and split-K partials are used).
 * A product with a plain FP32 result and a long K may split K: its slices are
 * added in a fixed order (same result on every call). */
apm_status_t apm_mlp_gemm_tn(const uint16_t *A, const uint16_t *Bt, const float *bias, float *C32, uint16_t *Cb,
                             int M, int N, int K, int relu, void *workspace, size_t workspace_bytes,
                             apm_stream_t stream);
/* refresh param_bf16 from param (after the caller initialises param) */
apm_status_t apm_mlp_sync_bf16(const apm_mlp *net, apm_stream_t stream);
/* y[b] (FP32) = network(X[b]) for b < batch_padded; X [batch_padded][64] BF16 */
apm_status_t apm_mlp_forward(const apm_mlp *net, const uint16_t *X, int batch_padded, float *y, void *workspace,
                             size_t workspace_bytes, apm_stream_t stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr, step >= 1
 * for the bias correction) on the mean squared error over the first batch_valid
 * rows; adds the loss to *loss_acc (device float). */
apm_status_t apm_mlp_train_step(const apm_mlp *net, const uint16_t *X, const float *target, int batch_padded,
                                int batch_valid, float lr, int step, float *loss_acc, void *workspace,
                                size_t workspace_bytes, apm_stream_t stream);
/* The two halves of apm_mlp_train_step, for data-parallel training across
 * processes (no counterpart in the paper): apm_mlp_gradient writes the gradient
 * of the mean squared error over the first batch_valid rows into net->grad (and
 * adds the loss to *loss_acc); the caller may then replace net->grad by its
 * average over the processes; apm_mlp_adam_step applies one Adam step from
 * net->grad and refreshes param_bf16. Together they do exactly what
 * apm_mlp_train_step does, bit for bit. */
apm_status_t apm_mlp_gradient(const apm_mlp *net, const uint16_t *X, const float *target, int batch_padded,
                              int batch_valid, float *loss_acc, void *workspace, size_t workspace_bytes,
                              apm_stream_t stream);
apm_status_t apm_mlp_adam_step(const apm_mlp *net, float lr, int step, apm_stream_t stream);

/*
 * apm_order_sums -- per-order sums of the connected sums of whole vertex sets,
 * the data of the power-series estimator (Section V, Eq. series: the order-m
 * term is the integral of c_m over the configurations of m vertices; a sample of
 * configurations estimates it by their mean, its sign problem by the ratio of
 * sum c to sum |c|). A data-parallel job reduces its rows on each device with
 * this call and adds the few resulting numbers across processes on the host.
 *   c      connected-sum rows (device): with n_arr NULL, row b has 2^n_fixed
 *          doubles at c + b 2^n_fixed; else row b has 2^n_arr[b] doubles at
 *          c + c_off[b] (the layout of apm_cdet_connected_varlen).
 *   n_arr, c_off  both NULL (fixed order n_fixed in 1..n_max) or both set.
 *   n_max  1..16.
 *   out    [n_max+1][4] device doubles, overwritten: out[m] = (count, sum c,
 *          sum |c|, sum c^2) over the rows of order m of c_m = c[2^m - 1], the
 *          connected sum of the whole vertex set; out[0] = 0, and rows whose
 *          order lies outside 1..n_max count nowhere.
 * One CTA adds in a fixed order: repeated calls give bit-identical results.
 * Asynchronous on `stream`; allocates nothing.
 */
apm_status_t apm_order_sums(const double *c, int n_fixed, const int32_t *n_arr, const int64_t *c_off,
                            int64_t batch, int n_max, double *out, apm_stream_t stream);

/*
 * apm_workspace_size -- bytes of device scratch the call `op` needs for orders up
 * to n_max and `batch` matrices on the current device (0 when none is needed).
 * two_mats != 0 sizes APM_OP_CDET for a separate A_dn.
 */
apm_status_t apm_workspace_size(int op, int n_max, int64_t batch, int two_mats, size_t *bytes);

/*
 * apm_status_reduce -- OR of the per-matrix status words; synchronises `stream`.
 *   status_dev [batch] device array written by an earlier call on `stream`.
 *   or_bits    host output.
 * Returns APM_ERR_NUMERIC when any APM_ST_ERROR_MASK bit is set, else APM_OK.
 */
apm_status_t apm_status_reduce(const uint32_t *status_dev, int64_t batch, uint32_t *or_bits,
                               apm_stream_t stream);

/* Human-readable name of a status code (static storage). */
const char *apm_status_string(apm_status_t s);

/* The cudaError_t of the last APM_ERR_CUDA on this thread (0 if none). */
int apm_last_cuda_error(void);

/* Library version, e.g. 100 for 0.1.0. */
int apm_version(void);

/*
 * apm_fp64_fma_probe -- FP64 throughput microbenchmark (no counterpart in the
 * paper; it measures the roofline denominator of the FP64-bound kernels).
 * Launches `blocks` x `threads` threads, each running `iters` rounds of 16
 * independent dependent-chain FP64 fused multiply-adds; writes one double per
 * thread to `sink` (device, blocks*threads doubles) so nothing is optimised away.
 * FLOPs = 32 * blocks * threads * iters.
 */
apm_status_t apm_fp64_fma_probe(double *sink, int blocks, int threads, int iters,
                                apm_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* APM_H */
