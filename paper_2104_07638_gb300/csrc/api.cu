// C-ABI entry points of libapm.so: argument validation on the host, then one
// asynchronous launch on the caller's stream. See include/apm.h.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdint.h>
#include <stdlib.h>

#include <vector>

#include "apm_internal.cuh"

namespace {

thread_local int t_last_cuda = 0;

apm_status_t cuda_fail(int e) {
    t_last_cuda = e;
    return APM_ERR_CUDA;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

apm_status_t check_ptr(const void *p, int64_t batch) {
    if (batch == 0) return APM_OK;
    if (!p || !aligned16(p)) return APM_ERR_ARG;
    return APM_OK;
}

apm_status_t check_opt_ptr(const void *p) {
    if (p && !aligned16(p)) return APM_ERR_ARG;
    return APM_OK;
}

void pivot_values(const apm_pivot_opts *opt, double *thr, double *shift) {
    *thr = opt ? opt->piv_threshold : APM_DEFAULT_PIV_THRESHOLD;
    *shift = opt ? opt->piv_shift : APM_DEFAULT_PIV_SHIFT;
}

apm_status_t cdet_common(apm::CdetArgs &a, void *workspace, size_t workspace_bytes,
                         cudaStream_t s) {
    if (a.batch == 0) return APM_OK;
    const bool two = a.two_mats != 0;
    const bool smem_arrays = a.n <= apm::cdet_smem_max_n(two);
    if (!smem_arrays) {
        int err = 0;
        const int grid = apm::cdet_grid(a.n, a.batch, two, false, &err);
        if (err) return cuda_fail(err);
        size_t need = static_cast<size_t>(grid) * apm::cdet_slot_doubles(a.n) * sizeof(double);
        if (a.mode == apm::kModeCdet && a.n >= apm::cdet_fsc_from_n()) {
            const size_t f = apm::fsc_workspace_bytes(a.n, a.batch, &err);
            if (err) return cuda_fail(err);
            if (f > need) need = f;
        }
        // connected sums of one matrix per item: the minors come from the
        // warp-per-matrix kernel (its flags first, its stacks in the slots' region)
        const bool route = a.mode == apm::kModeCdet && !two && a.n >= apm::kWarpRouteFromN;
        size_t flag_bytes = 0;
        if (route) {
            const size_t st = apm::fpm_warp_route_stack_bytes(a.n, a.batch, &err);
            if (err) return cuda_fail(err);
            if (st > need) need = st;
            flag_bytes = (static_cast<size_t>(a.batch) + 255) & ~static_cast<size_t>(255);
        }
        if (!workspace || workspace_bytes < flag_bytes + need || !aligned16(workspace)) return APM_ERR_WORKSPACE;
        if (route) {
            a.wflag = static_cast<uint8_t *>(workspace);
            a.warp_from_n = apm::kWarpRouteFromN;
        }
        a.gscratch = reinterpret_cast<double *>(static_cast<unsigned char *>(workspace) + flag_bytes);
    }
    const int e = apm::launch_fpm_cdet(a, s);
    return e ? cuda_fail(e) : APM_OK;
}

size_t round256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

// One slot of the host pipeline's workspace: byte sizes of its parts, each a
// multiple of 256 so that every part stays aligned.
struct HostSlot {
    size_t a_up, a_dn, c, m, st, ws, total;
};

apm_status_t host_slot_layout(int n, int64_t chunk, bool two, HostSlot *L) {
    const size_t N = static_cast<size_t>(1) << n, nn = static_cast<size_t>(n) * n;
    const size_t cb = static_cast<size_t>(chunk), mats = two ? 2 : 1;
    L->a_up = round256(cb * nn * sizeof(double));
    L->a_dn = two ? L->a_up : 0;
    L->c = round256(cb * N * sizeof(double));
    L->m = round256(cb * mats * N * sizeof(double));
    L->st = round256(cb * sizeof(uint32_t));
    size_t ws = 0;
    const apm_status_t s = apm_workspace_size(APM_OP_CDET, n, chunk, two ? 1 : 0, &ws);
    if (s) return s;
    L->ws = round256(ws);
    L->total = L->a_up + L->a_dn + L->c + L->m + L->st + L->ws;
    return APM_OK;
}

}  // namespace

extern "C" {

apm_status_t apm_all_minors(const double *A, int n, int64_t batch, double *minors,
                            const apm_pivot_opts *opt, uint32_t *status, void *workspace,
                            size_t workspace_bytes, apm_stream_t stream) {
    if (n < 1 || n > APM_MAX_N_ALL_MINORS) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0) return APM_ERR_ARG;
    apm_status_t st;
    if ((st = check_ptr(A, batch)) || (st = check_ptr(minors, batch)) || (st = check_opt_ptr(status)))
        return st;
    if (n > APM_MAX_N_MINORS) {  // the upper levels breadth first, the 12 x 12 leaves by warps
        if (batch == 0) return APM_OK;
        if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return APM_ERR_WORKSPACE;
        int err = 0;
        const size_t need = apm::fpm_big_workspace_bytes(n, batch, &err);
        if (err) return cuda_fail(err);
        if (workspace_bytes < need) return APM_ERR_WORKSPACE;
        double thr, shift;
        pivot_values(opt, &thr, &shift);
        const int e = apm::launch_fpm_big(A, n, batch, minors, thr, shift, status, workspace,
                                          reinterpret_cast<cudaStream_t>(stream));
        return e ? cuda_fail(e) : APM_OK;
    }
    if (n >= apm::kWarpMinorsFromN) {  // one warp per matrix; small pivots redone by the fused kernel
        if (batch == 0) return APM_OK;
        if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255u)) return APM_ERR_WORKSPACE;
        int err = 0;
        const size_t need = apm::fpm_warp_workspace_bytes(n, batch, &err);
        if (err) return cuda_fail(err);
        if (workspace_bytes < need) return APM_ERR_WORKSPACE;
        double thr, shift;
        pivot_values(opt, &thr, &shift);
        const int e = apm::launch_fpm_warp(A, n, batch, minors, thr, shift, status, workspace,
                                           reinterpret_cast<cudaStream_t>(stream));
        return e ? cuda_fail(e) : APM_OK;
    }
    apm::CdetArgs a = {};
    a.A_up = A;
    a.minors_out = minors;
    a.status = status;
    a.batch = batch;
    a.n = n;
    a.mode = apm::kModeMinors;
    pivot_values(opt, &a.piv_thr, &a.piv_shift);
    return cdet_common(a, workspace, workspace_bytes, reinterpret_cast<cudaStream_t>(stream));
}

apm_status_t apm_cdet_connected(const double *A_up, const double *A_dn, int n, int64_t batch,
                                int flags, double *c, double *minors_out,
                                const apm_pivot_opts *opt, uint32_t *status, void *workspace,
                                size_t workspace_bytes, apm_stream_t stream) {
    if (n < 1 || n > APM_MAX_N_MINORS) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0 || (flags & ~APM_CDET_SINGLE_DET)) return APM_ERR_ARG;
    if ((flags & APM_CDET_SINGLE_DET) && A_dn) return APM_ERR_ARG;
    apm_status_t st;
    if ((st = check_ptr(A_up, batch)) || (st = check_opt_ptr(A_dn)) || (st = check_ptr(c, batch)) ||
        (st = check_opt_ptr(minors_out)) || (st = check_opt_ptr(status)))
        return st;
    apm::CdetArgs a = {};
    a.A_up = A_up;
    a.A_dn = A_dn;
    a.minors_out = minors_out;
    a.c_out = c;
    a.status = status;
    a.batch = batch;
    a.n = n;
    a.mode = apm::kModeCdet;
    a.single_det = (flags & APM_CDET_SINGLE_DET) ? 1 : 0;
    a.two_mats = A_dn ? 1 : 0;
    pivot_values(opt, &a.piv_thr, &a.piv_shift);
    return cdet_common(a, workspace, workspace_bytes, reinterpret_cast<cudaStream_t>(stream));
}

apm_status_t apm_cdet_connected_host_workspace_size(int n, int64_t chunk, int nstreams, int two_mats,
                                                    size_t *bytes) {
    if (!bytes) return APM_ERR_ARG;
    *bytes = 0;
    if (n < 1 || n > APM_MAX_N_MINORS) return APM_ERR_UNSUPPORTED_N;
    if (chunk < 1 || nstreams < 1 || nstreams > APM_HOST_MAX_STREAMS) return APM_ERR_ARG;
    HostSlot L;
    const apm_status_t st = host_slot_layout(n, chunk, two_mats != 0, &L);
    if (st) return st;
    *bytes = L.total * static_cast<size_t>(nstreams);
    return APM_OK;
}

apm_status_t apm_cdet_connected_host(const double *A_up, const double *A_dn, int n, int64_t batch, int flags,
                                     double *c, double *minors_out, const apm_pivot_opts *opt,
                                     uint32_t *status, int64_t chunk, int nstreams, void *workspace,
                                     size_t workspace_bytes, apm_stream_t stream) {
    if (n < 1 || n > APM_MAX_N_MINORS) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0 || chunk < 1 || nstreams < 1 || nstreams > APM_HOST_MAX_STREAMS ||
        (flags & ~APM_CDET_SINGLE_DET))
        return APM_ERR_ARG;
    if ((flags & APM_CDET_SINGLE_DET) && A_dn) return APM_ERR_ARG;
    if (batch == 0) return APM_OK;
    if (!A_up || !c) return APM_ERR_ARG;
    if (chunk > batch) chunk = batch;  // the workspace size does not grow as the chunk shrinks
    const bool two = A_dn != nullptr;
    HostSlot L;
    apm_status_t res = host_slot_layout(n, chunk, two, &L);
    if (res) return res;
    if (!workspace || workspace_bytes < L.total * static_cast<size_t>(nstreams) ||
        (reinterpret_cast<uintptr_t>(workspace) & 255u))
        return APM_ERR_WORKSPACE;

    const size_t N = static_cast<size_t>(1) << n, nn = static_cast<size_t>(n) * n, mats = two ? 2 : 1;

    cudaStream_t ss[APM_HOST_MAX_STREAMS] = {};
    int made = 0;
    cudaError_t err = cudaSuccess;
    cudaEvent_t ready = nullptr;
    err = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
    if (err == cudaSuccess) err = cudaEventRecord(ready, reinterpret_cast<cudaStream_t>(stream));
    for (; err == cudaSuccess && made < nstreams; ++made) {
        err = cudaStreamCreateWithFlags(&ss[made], cudaStreamNonBlocking);
        if (err != cudaSuccess) break;
        err = cudaStreamWaitEvent(ss[made], ready, 0);  // the caller's earlier work on the workspace
    }
    // Pieces of `chunk` matrices while more than two chunks remain, then
    // halving pieces down to chunk / 16: the copy-out of the last piece is the
    // one part of the pipeline nothing overlaps, so it is kept short. Piece k
    // goes to slot k % nstreams: a slot's buffers are reused only by pieces on
    // its own stream, so stream order keeps them apart.
    const int64_t min_piece = chunk / 16 > 0 ? chunk / 16 : 1;
    int64_t b0 = 0;
    for (int64_t k = 0; err == cudaSuccess && res == APM_OK && b0 < batch; ++k) {
        const int q = static_cast<int>(k % nstreams);
        const int64_t rem = batch - b0;
        int64_t cb = rem > 2 * chunk ? chunk : (rem + 1) / 2;
        if (cb < min_piece || rem <= min_piece) cb = rem;
        if (cb > chunk) cb = chunk;
        const size_t ub = static_cast<size_t>(b0), ucb = static_cast<size_t>(cb);
        char *base = static_cast<char *>(workspace) + static_cast<size_t>(q) * L.total;
        double *dA = reinterpret_cast<double *>(base);
        double *dB = two ? reinterpret_cast<double *>(base + L.a_up) : nullptr;
        double *dc = reinterpret_cast<double *>(base + L.a_up + L.a_dn);
        double *dm = reinterpret_cast<double *>(base + L.a_up + L.a_dn + L.c);
        uint32_t *dst = reinterpret_cast<uint32_t *>(base + L.a_up + L.a_dn + L.c + L.m);
        void *dws = L.ws ? static_cast<void *>(base + L.a_up + L.a_dn + L.c + L.m + L.st) : nullptr;
        err = cudaMemcpyAsync(dA, A_up + ub * nn, ucb * nn * sizeof(double), cudaMemcpyHostToDevice, ss[q]);
        if (err == cudaSuccess && two)
            err = cudaMemcpyAsync(dB, A_dn + ub * nn, ucb * nn * sizeof(double), cudaMemcpyHostToDevice, ss[q]);
        if (err != cudaSuccess) break;
        res = apm_cdet_connected(dA, dB, n, cb, flags, dc, minors_out ? dm : nullptr, opt, status ? dst : nullptr,
                                 dws, L.ws, reinterpret_cast<apm_stream_t>(ss[q]));
        if (res != APM_OK) break;
        err = cudaMemcpyAsync(c + ub * N, dc, ucb * N * sizeof(double), cudaMemcpyDeviceToHost, ss[q]);
        if (err == cudaSuccess && minors_out)
            err = cudaMemcpyAsync(minors_out + ub * mats * N, dm, ucb * mats * N * sizeof(double),
                                  cudaMemcpyDeviceToHost, ss[q]);
        if (err == cudaSuccess && status)
            err = cudaMemcpyAsync(status + ub, dst, ucb * sizeof(uint32_t), cudaMemcpyDeviceToHost, ss[q]);
        b0 += cb;
    }
    for (int i = 0; i < made; ++i) {  // wait for everything issued, even after an error
        const cudaError_t e = cudaStreamSynchronize(ss[i]);
        if (err == cudaSuccess) err = e;
        cudaStreamDestroy(ss[i]);
    }
    if (ready) cudaEventDestroy(ready);
    if (res != APM_OK) return res;
    return err != cudaSuccess ? cuda_fail(static_cast<int>(err)) : APM_OK;
}

apm_status_t apm_cdet_from_weights(const double *a_in, int n, int64_t batch, double *c,
                                   void *workspace, size_t workspace_bytes, apm_stream_t stream) {
    if (n < 1 || n > APM_MAX_N_MINORS) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0) return APM_ERR_ARG;
    apm_status_t st;
    if ((st = check_ptr(a_in, batch)) || (st = check_ptr(c, batch))) return st;
    apm::CdetArgs a = {};
    a.a_in = a_in;
    a.c_out = c;
    a.batch = batch;
    a.n = n;
    a.mode = apm::kModeWeights;
    return cdet_common(a, workspace, workspace_bytes, reinterpret_cast<cudaStream_t>(stream));
}

apm_status_t apm_cdet_from_weights_fsc(const double *a, int n, int64_t batch, double *c, void *workspace,
                                       size_t workspace_bytes, apm_stream_t stream) {
    if (n < 1 || n > APM_MAX_N_MINORS) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0) return APM_ERR_ARG;
    apm_status_t st;
    if ((st = check_ptr(a, batch)) || (st = check_ptr(c, batch))) return st;
    if (batch == 0) return APM_OK;
    size_t need = 0;
    if ((st = apm_workspace_size(APM_OP_CDET_FSC, n, batch, 0, &need))) return st;
    if (need > 0 && (!workspace || workspace_bytes < need || !aligned16(workspace))) return APM_ERR_WORKSPACE;
    const int e = apm::launch_fsc(a, n, batch, c, workspace, reinterpret_cast<cudaStream_t>(stream));
    return e ? cuda_fail(e) : APM_OK;
}

apm_status_t apm_xnor_minors(const double *M, int n, int64_t batch, double *minors, uint32_t *status,
                             void *workspace, size_t workspace_bytes, apm_stream_t stream) {
    if (n < 1 || n > APM_MAX_N_XNOR) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0) return APM_ERR_ARG;
    apm_status_t st;
    if ((st = check_ptr(M, batch)) || (st = check_ptr(minors, batch)) || (st = check_opt_ptr(status))) return st;
    if (batch == 0) return APM_OK;
    size_t need = 0;
    if ((st = apm_workspace_size(APM_OP_XNOR_MINORS, n, batch, 0, &need))) return st;
    if (need > 0 && (!workspace || workspace_bytes < need || !aligned16(workspace))) return APM_ERR_WORKSPACE;
    const int e = apm::launch_xnor(M, n, batch, minors, status, workspace, reinterpret_cast<cudaStream_t>(stream));
    return e ? cuda_fail(e) : APM_OK;
}

apm_status_t apm_nambu_cdet(const double *M, int n, int64_t batch, double *minors, double *c, uint32_t *status,
                            void *workspace, size_t workspace_bytes, apm_stream_t stream) {
    if (n < 1 || n > APM_MAX_N_XNOR) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0) return APM_ERR_ARG;
    apm_status_t st;
    if ((st = check_ptr(M, batch)) || (st = check_ptr(minors, batch)) || (st = check_ptr(c, batch)) ||
        (st = check_opt_ptr(status)))
        return st;
    if (batch == 0) return APM_OK;
    size_t need = 0;
    if ((st = apm_workspace_size(APM_OP_NAMBU_CDET, n, batch, 0, &need))) return st;
    if (need > 0 && (!workspace || workspace_bytes < need || !aligned16(workspace))) return APM_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int e = apm::launch_xnor(M, n, batch, minors, status, workspace, s);
    if (e) return cuda_fail(e);
    // the same scratch serves the recursion: the two launches run in order on s
    apm::CdetArgs a = {};
    a.a_in = minors;
    a.c_out = c;
    a.batch = batch;
    a.n = n;
    a.mode = apm::kModeWeights;
    return cdet_common(a, workspace, workspace_bytes, s);
}

apm_status_t apm_nand_minors(const double *M, int n, int64_t batch, double *minors3, const apm_pivot_opts *opt,
                             uint32_t *status, void *workspace, size_t workspace_bytes, apm_stream_t stream) {
    if (n < 1 || n > APM_MAX_N_NAND_MINORS) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0) return APM_ERR_ARG;
    apm_status_t st;
    if ((st = check_ptr(M, batch)) || (st = check_ptr(minors3, batch)) || (st = check_opt_ptr(status))) return st;
    if (batch == 0) return APM_OK;
    size_t need = 0;
    if ((st = apm_workspace_size(APM_OP_NAND_MINORS, n, batch, 0, &need))) return st;
    if (need > 0 && (!workspace || workspace_bytes < need || !aligned16(workspace))) return APM_ERR_WORKSPACE;
    double thr, shift;
    pivot_values(opt, &thr, &shift);
    const int e = apm::launch_nand(M, n, batch, minors3, false, thr, shift, status, workspace,
                                   reinterpret_cast<cudaStream_t>(stream));
    return e ? cuda_fail(e) : APM_OK;
}

apm_status_t apm_two_type_cdet(const double *M, int n, int64_t batch, double *abar, double *c,
                               const apm_pivot_opts *opt, uint32_t *status, void *workspace,
                               size_t workspace_bytes, apm_stream_t stream) {
    if (n < 1 || n > APM_MAX_N_TWO_TYPE) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0) return APM_ERR_ARG;
    apm_status_t st;
    if ((st = check_ptr(M, batch)) || (st = check_ptr(abar, batch)) || (st = check_ptr(c, batch)) ||
        (st = check_opt_ptr(status)))
        return st;
    if (batch == 0) return APM_OK;
    size_t need = 0;
    if ((st = apm_workspace_size(APM_OP_TWO_TYPE_CDET, n, batch, 0, &need))) return st;
    if (need > 0 && (!workspace || workspace_bytes < need || !aligned16(workspace))) return APM_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double thr, shift;
    pivot_values(opt, &thr, &shift);
    const int e = apm::launch_nand(M, n, batch, abar, true, thr, shift, status, workspace, s);
    if (e) return cuda_fail(e);
    // the same scratch serves the recursion: the two launches run in order on s
    apm::CdetArgs a = {};
    a.a_in = abar;
    a.c_out = c;
    a.batch = batch;
    a.n = n;
    a.mode = apm::kModeWeights;
    return cdet_common(a, workspace, workspace_bytes, s);
}

apm_status_t apm_keldysh2_sum(const double *Mu, const double *Md, int n, int64_t batch, int flags, double *sum,
                              double *partial, uint32_t *status, void *workspace, size_t workspace_bytes,
                              apm_stream_t stream) {
    if (n < 1 || n > APM_MAX_N_KELDYSH) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0 || (flags & ~APM_KELDYSH_SIGNED)) return APM_ERR_ARG;
    apm_status_t st;
    if ((st = check_ptr(Mu, batch)) || (st = check_ptr(Md, batch)) || (st = check_ptr(sum, batch)) ||
        (st = check_opt_ptr(partial)) || (st = check_opt_ptr(status)))
        return st;
    if (batch == 0) return APM_OK;
    size_t need = 0;
    if ((st = apm_workspace_size(APM_OP_KELDYSH2, n, batch, 0, &need))) return st;
    if (need > 0 && (!workspace || workspace_bytes < need || !aligned16(workspace))) return APM_ERR_WORKSPACE;
    const int e = apm::launch_keldysh2(Mu, Md, n, batch, (flags & APM_KELDYSH_SIGNED) ? 1 : 0, sum, partial, status,
                                       workspace, reinterpret_cast<cudaStream_t>(stream));
    return e ? cuda_fail(e) : APM_OK;
}

apm_status_t apm_keldysh_sum(const double *Mt, int n, int64_t batch, int flags, double *sum,
                             double *partial, uint32_t *status, void *workspace,
                             size_t workspace_bytes, apm_stream_t stream) {
    if (n < 1 || n > APM_MAX_N_KELDYSH) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0 || (flags & ~APM_KELDYSH_SIGNED)) return APM_ERR_ARG;
    apm_status_t st;
    if ((st = check_ptr(Mt, batch)) || (st = check_ptr(sum, batch)) || (st = check_opt_ptr(partial)) ||
        (st = check_opt_ptr(status)))
        return st;
    if (batch == 0) return APM_OK;
    size_t need = 0;
    if ((st = apm_workspace_size(APM_OP_KELDYSH, n, batch, 0, &need))) return st;
    if (need > 0 && (!workspace || workspace_bytes < need || !aligned16(workspace)))
        return APM_ERR_WORKSPACE;
    const int e = apm::launch_keldysh(Mt, n, batch, (flags & APM_KELDYSH_SIGNED) ? 1 : 0, sum, partial,
                                      status, workspace, reinterpret_cast<cudaStream_t>(stream));
    return e ? cuda_fail(e) : APM_OK;
}

apm_status_t apm_perm_minors(const double *A, int n, int64_t batch, double *perms, void *workspace,
                             size_t workspace_bytes, apm_stream_t stream) {
    (void)workspace;
    (void)workspace_bytes;
    if (n < 1 || n > APM_MAX_N_PERM) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0) return APM_ERR_ARG;
    apm_status_t st;
    if ((st = check_ptr(A, batch)) || (st = check_ptr(perms, batch))) return st;
    if (batch == 0) return APM_OK;
    const int e = apm::launch_ppm(A, n, batch, perms, reinterpret_cast<cudaStream_t>(stream));
    return e ? cuda_fail(e) : APM_OK;
}

apm_status_t apm_cdet_connected_varlen(const double *A, const double *A_dn, const int64_t *a_off,
                                       const int32_t *n, int64_t batch, int n_max, int flags, double *c,
                                       double *minors_out, const int64_t *c_off,
                                       const apm_pivot_opts *opt, uint32_t *status, void *workspace,
                                       size_t workspace_bytes, apm_stream_t stream) {
    if (n_max < 1 || n_max > APM_MAX_N_MINORS) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0 || batch > INT32_MAX || (flags & ~APM_CDET_SINGLE_DET)) return APM_ERR_ARG;
    if ((flags & APM_CDET_SINGLE_DET) && A_dn) return APM_ERR_ARG;
    if (batch == 0) return APM_OK;
    apm_status_t st;
    if ((st = check_ptr(A, batch)) || (st = check_opt_ptr(A_dn)) || (st = check_ptr(a_off, batch)) ||
        (st = check_ptr(n, batch)) || (st = check_ptr(c, batch)) || (st = check_opt_ptr(minors_out)) ||
        (st = check_ptr(c_off, batch)) || (st = check_opt_ptr(status)))
        return st;
    size_t need = 0;
    if ((st = apm_workspace_size(APM_OP_CDET_VARLEN, n_max, batch, A_dn ? 1 : 0, &need))) return st;
    if (!workspace || workspace_bytes < need || !aligned16(workspace)) return APM_ERR_WORKSPACE;
    apm::CdetArgs a = {};
    a.A_up = A;
    a.A_dn = A_dn;
    a.minors_out = minors_out;
    a.c_out = c;
    a.status = status;
    a.batch = batch;
    a.n = n_max;
    a.mode = apm::kModeCdet;
    a.single_det = (flags & APM_CDET_SINGLE_DET) ? 1 : 0;
    a.two_mats = A_dn ? 1 : 0;
    pivot_values(opt, &a.piv_thr, &a.piv_shift);
    const int e = apm::launch_cdet_varlen(a, a_off, n, c_off, n_max, workspace,
                                          reinterpret_cast<cudaStream_t>(stream));
    return e ? cuda_fail(e) : APM_OK;
}

apm_status_t apm_keldysh_sum_varlen(const double *Mt, const int64_t *m_off, const int32_t *n, int64_t batch,
                                    int n_max, int flags, double *sum, double *partial, uint32_t *status,
                                    void *workspace, size_t workspace_bytes, apm_stream_t stream) {
    if (n_max < 1 || n_max > APM_MAX_N_KELDYSH) return APM_ERR_UNSUPPORTED_N;
    if (batch < 0 || batch > INT32_MAX || (flags & ~APM_KELDYSH_SIGNED)) return APM_ERR_ARG;
    if (batch == 0) return APM_OK;
    apm_status_t st;
    if ((st = check_ptr(Mt, batch)) || (st = check_ptr(m_off, batch)) || (st = check_ptr(n, batch)) ||
        (st = check_ptr(sum, batch)) || (st = check_opt_ptr(partial)) || (st = check_opt_ptr(status)))
        return st;
    size_t need = 0;
    if ((st = apm_workspace_size(APM_OP_KELDYSH_VARLEN, n_max, batch, 0, &need))) return st;
    if (!workspace || workspace_bytes < need || !aligned16(workspace)) return APM_ERR_WORKSPACE;
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    const size_t order_bytes = ((static_cast<size_t>(batch) * 4) + 255) & ~size_t(255);
    unsigned *ctr = reinterpret_cast<unsigned *>(ws);
    int *order = reinterpret_cast<int *>(ws + 256);
    void *stack = apm::keldysh_stack_entries(n_max) ? ws + 256 + order_bytes : nullptr;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int e = apm::launch_order(n, batch, n_max, order, ctr, s);
    if (!e)
        e = apm::launch_keldysh_varlen(Mt, m_off, n, batch, n_max, (flags & APM_KELDYSH_SIGNED) ? 1 : 0, sum,
                                       partial, status, stack, order, ctr, s);
    return e ? cuda_fail(e) : APM_OK;
}

apm_status_t apm_tune_options_set(int fsc_from_n, int cdet_ctas_per_sm, int keldysh_warps) {
    if (fsc_from_n == 0) fsc_from_n = apm::kFscFromN;
    if (fsc_from_n < apm::kFscMinFrom || fsc_from_n > 17 || cdet_ctas_per_sm < 0 || cdet_ctas_per_sm > 3 ||
        keldysh_warps < 0 || (keldysh_warps && (keldysh_warps < 4 || keldysh_warps > 12)))
        return APM_ERR_ARG;
    apm::cdet_tune_options_set(fsc_from_n, cdet_ctas_per_sm);
    apm::keldysh_varlen_warps_set(keldysh_warps);
    return APM_OK;
}

apm_status_t apm_tune_options_get(int *fsc_from_n, int *cdet_ctas_per_sm, int *keldysh_warps) {
    if (fsc_from_n) *fsc_from_n = apm::cdet_fsc_from_n();
    if (cdet_ctas_per_sm) *cdet_ctas_per_sm = apm::cdet_varlen_ctas_per_sm();
    if (keldysh_warps) *keldysh_warps = apm::keldysh_varlen_warps();
    return APM_OK;
}

apm_status_t apm_cdet_tune_set(const uint64_t *table) {
    if (table) {
        for (int n = 0; n <= 16; ++n) {
            const uint64_t t = table[n];
            if (!t) continue;
            for (int k = 0; k <= 16; ++k) {
                const int r = static_cast<int>((t >> (3 * k)) & 7u);
                if (r > 5 || (k <= n && k >= 1 && r > k - 1) || (k > n && r != 0) || (k < 2 && r != 0))
                    return APM_ERR_ARG;
            }
        }
    }
    apm::cdet_tune_set(reinterpret_cast<const unsigned long long *>(table));
    return APM_OK;
}

apm_status_t apm_cdet_tune_get(int n, uint64_t *packed) {
    if (!packed || n < 0 || n > 16) return APM_ERR_ARG;
    *packed = apm::cdet_gsel_packed(n);
    return APM_OK;
}

apm_status_t apm_workspace_size(int op, int n_max, int64_t batch, int two_mats, size_t *bytes) {
    if (!bytes || batch < 0) return APM_ERR_ARG;
    *bytes = 0;
    switch (op) {
        case APM_OP_ALL_MINORS:
        case APM_OP_CDET:
        case APM_OP_CDET_FROM_WEIGHTS: {
            if (op == APM_OP_ALL_MINORS && n_max > APM_MAX_N_MINORS && n_max <= APM_MAX_N_ALL_MINORS) {
                int err = 0;
                *bytes = apm::fpm_big_workspace_bytes(n_max, batch, &err);
                return err ? cuda_fail(err) : APM_OK;
            }
            if (op == APM_OP_ALL_MINORS && n_max >= apm::kWarpMinorsFromN && n_max <= APM_MAX_N_MINORS) {
                int err = 0;
                *bytes = apm::fpm_warp_workspace_bytes(n_max, batch, &err);
                return err ? cuda_fail(err) : APM_OK;
            }
            if (n_max < 1 || n_max > APM_MAX_N_MINORS) return APM_ERR_UNSUPPORTED_N;
            const bool two = op == APM_OP_CDET && two_mats;
            if (n_max <= apm::cdet_smem_max_n(two) || batch == 0) return APM_OK;
            int err = 0;
            const int grid = apm::cdet_grid(n_max, batch, two, false, &err);
            if (err) return cuda_fail(err);
            *bytes = static_cast<size_t>(grid) * apm::cdet_slot_doubles(n_max) * sizeof(double);
            if (op == APM_OP_CDET && n_max >= apm::cdet_fsc_from_n()) {  // then the ranked arrays
                const size_t f = apm::fsc_workspace_bytes(n_max, batch, &err);
                if (err) return cuda_fail(err);
                if (f > *bytes) *bytes = f;
            }
            if (op == APM_OP_CDET && !two && n_max >= apm::kWarpRouteFromN) {
                // the warp-per-matrix minors: its stacks in the same region, its flags before it
                const size_t st = apm::fpm_warp_route_stack_bytes(n_max, batch, &err);
                if (err) return cuda_fail(err);
                if (st > *bytes) *bytes = st;
                *bytes += (static_cast<size_t>(batch) + 255) & ~static_cast<size_t>(255);
            }
            return APM_OK;
        }
        case APM_OP_KELDYSH: {
            if (n_max < 1 || n_max > APM_MAX_N_KELDYSH) return APM_ERR_UNSUPPORTED_N;
            if (apm::keldysh_stack_entries(n_max) == 0 || batch == 0) return APM_OK;
            apm::KeldyshPlan p;
            const int err = apm::keldysh_plan(n_max, batch, &p);
            if (err) return cuda_fail(err);
            *bytes = p.total;
            return APM_OK;
        }
        case APM_OP_XNOR_MINORS:
        case APM_OP_NAMBU_CDET: {
            if (n_max < 1 || n_max > APM_MAX_N_XNOR) return APM_ERR_UNSUPPORTED_N;
            if (batch == 0) return APM_OK;
            int err = 0;
            size_t need = apm::xnor_workspace_bytes(n_max, batch, &err);
            if (err) return cuda_fail(err);
            if (op == APM_OP_NAMBU_CDET && n_max > apm::cdet_smem_max_n(false)) {
                const int grid = apm::cdet_grid(n_max, batch, false, false, &err);
                if (err) return cuda_fail(err);
                const size_t rec = static_cast<size_t>(grid) * apm::cdet_slot_doubles(n_max) * sizeof(double);
                if (rec > need) need = rec;
            }
            *bytes = need;
            return APM_OK;
        }
        case APM_OP_NAND_MINORS:
        case APM_OP_TWO_TYPE_CDET: {
            const int nmax = op == APM_OP_NAND_MINORS ? APM_MAX_N_NAND_MINORS : APM_MAX_N_TWO_TYPE;
            if (n_max < 1 || n_max > nmax) return APM_ERR_UNSUPPORTED_N;
            if (batch == 0) return APM_OK;
            int err = 0;
            size_t need = apm::nand_workspace_bytes(n_max, batch, &err);
            if (err) return cuda_fail(err);
            if (op == APM_OP_TWO_TYPE_CDET && n_max > apm::cdet_smem_max_n(false)) {
                const int grid = apm::cdet_grid(n_max, batch, false, false, &err);
                if (err) return cuda_fail(err);
                const size_t rec = static_cast<size_t>(grid) * apm::cdet_slot_doubles(n_max) * sizeof(double);
                if (rec > need) need = rec;
            }
            *bytes = need;
            return APM_OK;
        }
        case APM_OP_KELDYSH2: {
            if (n_max < 1 || n_max > APM_MAX_N_KELDYSH) return APM_ERR_UNSUPPORTED_N;
            if (batch == 0) return APM_OK;
            int err = 0;
            *bytes = apm::keldysh2_workspace_bytes(n_max, batch, &err);
            return err ? cuda_fail(err) : APM_OK;
        }
        case APM_OP_CDET_FSC: {
            if (n_max < 1 || n_max > APM_MAX_N_MINORS) return APM_ERR_UNSUPPORTED_N;
            if (batch == 0) return APM_OK;
            int err = 0;
            *bytes = apm::fsc_workspace_bytes(n_max, batch, &err);
            return err ? cuda_fail(err) : APM_OK;
        }
        case APM_OP_PERM_MINORS:
            if (n_max < 1 || n_max > APM_MAX_N_PERM) return APM_ERR_UNSUPPORTED_N;
            return APM_OK;
        case APM_OP_CDET_VARLEN: {
            if (n_max < 1 || n_max > APM_MAX_N_MINORS) return APM_ERR_UNSUPPORTED_N;
            if (batch == 0) return APM_OK;
            int err = 0;
            *bytes = apm::cdet_varlen_workspace(n_max, batch, two_mats != 0, &err);
            return err ? cuda_fail(err) : APM_OK;
        }
        case APM_OP_KELDYSH_VARLEN: {
            if (n_max < 1 || n_max > APM_MAX_N_KELDYSH) return APM_ERR_UNSUPPORTED_N;
            if (batch == 0) return APM_OK;
            const size_t order_bytes = ((static_cast<size_t>(batch) * 4) + 255) & ~size_t(255);
            size_t stack = 0;
            const size_t per = apm::keldysh_stack_entries(n_max);
            if (per) {
                int err = 0;
                const int grid = apm::keldysh_grid(batch, &err);
                if (err) return cuda_fail(err);
                stack = static_cast<size_t>(grid) * apm::keldysh_warps_per_block() * per * 2 * sizeof(double);
            }
            *bytes = 256 + order_bytes + stack;
            return APM_OK;
        }
        default:
            return APM_ERR_ARG;
    }
}

apm_status_t apm_status_reduce(const uint32_t *status_dev, int64_t batch, uint32_t *or_bits,
                               apm_stream_t stream) {
    if (!or_bits || batch < 0 || (batch > 0 && !status_dev)) return APM_ERR_ARG;
    *or_bits = 0;
    if (batch == 0) return APM_OK;
    std::vector<uint32_t> host(static_cast<size_t>(batch));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(host.data(), status_dev, host.size() * sizeof(uint32_t),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e);
    uint32_t acc = 0;
    for (uint32_t v : host) acc |= v;
    *or_bits = acc;
    return (acc & APM_ST_ERROR_MASK) ? APM_ERR_NUMERIC : APM_OK;
}

const char *apm_status_string(apm_status_t s) {
    switch (s) {
        case APM_OK: return "APM_OK";
        case APM_ERR_ARG: return "APM_ERR_ARG: invalid argument (null, misaligned, negative or bad flags)";
        case APM_ERR_UNSUPPORTED_N: return "APM_ERR_UNSUPPORTED_N: order outside the supported range";
        case APM_ERR_CUDA: return "APM_ERR_CUDA: a CUDA call failed";
        case APM_ERR_NUMERIC: return "APM_ERR_NUMERIC: a matrix has an error status bit";
        case APM_ERR_TIMEOUT: return "APM_ERR_TIMEOUT: a bounded device wait gave up";
        case APM_ERR_WORKSPACE: return "APM_ERR_WORKSPACE: workspace missing or too small";
    }
    return "APM_UNKNOWN";
}

int apm_last_cuda_error(void) { return t_last_cuda; }

int apm_version(void) { return 100; }

apm_status_t apm_fp64_fma_probe(double *sink, int blocks, int threads, int iters,
                                apm_stream_t stream) {
    if (!sink || blocks < 1 || threads < 32 || threads > 1024 || iters < 1) return APM_ERR_ARG;
    const int e = apm::launch_fp64_probe(sink, blocks, threads, iters,
                                         reinterpret_cast<cudaStream_t>(stream));
    return e ? cuda_fail(e) : APM_OK;
}

}  // extern "C"
