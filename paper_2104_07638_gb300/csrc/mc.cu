// Monte Carlo walkers over vertex configurations and the C ABI of the
// surrogate network.
//
// A walker holds n vertices X_i = (x_i, y_i, m_i): a site of a win x win
// window and an imaginary-time grid index m in [0, mtau). Its weight is
// |c_n(X)|, the connected sum over all n vertices of the CDet recursion
// (Section V.A) on M_ij = G0(r_i - r_j, tau_i - tau_j), computed exactly by the
// FP64 minor / connected-sum kernels. The Section V.E single-vertex move is the
// plain proposal (one vertex redrawn uniformly). The learned proposal filters
// those moves with a surrogate s(X) ~ log|c_n(X)| first (delayed acceptance):
//   stage 1: pass with probability min(1, exp(s(X') - s(X)))
//   stage 2: accept with probability min(1, |c(X')| exp(s(X)) / (|c(X)| exp(s(X'))))
// which leaves the exact |c_n| distribution invariant; only stage-1 survivors
// are evaluated exactly. Uniform random numbers come in as inputs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "apm_internal.cuh"

namespace apm {

__global__ void mc_propose_kernel(const int *__restrict__ X, int W, int n, int win, int mtau,
                                  const float *__restrict__ u, int *Xp) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const int *src = X + static_cast<size_t>(w) * n * 3;
    int *dst = Xp + static_cast<size_t>(w) * n * 3;
    for (int i = 0; i < 3 * n; ++i) dst[i] = src[i];
    const float *uw = u + 4 * static_cast<size_t>(w);
    const int v = min(n - 1, static_cast<int>(uw[0] * n));
    dst[3 * v + 0] = min(win - 1, static_cast<int>(uw[1] * win));
    dst[3 * v + 1] = min(win - 1, static_cast<int>(uw[2] * win));
    dst[3 * v + 2] = min(mtau - 1, static_cast<int>(uw[3] * mtau));
}

// A[k] = G0 matrix of walker idx[k] (or k), from the table g0[|dx|][|dy|][dm + mtau - 1]
__global__ void mc_build_kernel(const int *__restrict__ X, const int *__restrict__ idx, int count, int n, int win,
                                int mtau, const double *__restrict__ g0, double *A) {
    const int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nn = static_cast<int64_t>(n) * n;
    if (e >= count * nn) return;
    const int k = static_cast<int>(e / nn);
    const int rem = static_cast<int>(e - k * nn);
    const int i = rem / n, j = rem - i * n;
    const int w = idx ? idx[k] : k;
    const int *xw = X + static_cast<size_t>(w) * n * 3;
    const int dx = abs(xw[3 * i] - xw[3 * j]);
    const int dy = abs(xw[3 * i + 1] - xw[3 * j + 1]);
    const int dm = xw[3 * i + 2] - xw[3 * j + 2] + mtau - 1;
    A[e] = g0[(static_cast<size_t>(dx) * win + dy) * (2 * mtau - 1) + dm];
}

// network input of walker idx[k] (or k): vertices sorted by time, shifted by
// the first one, scaled to [-1, 1] (14 vertex slots x 3); then n/14; then, in
// 14 slots sorted ascending, log10 of each vertex's coupling to the others,
// sum_{j != i} |G0(X_i - X_j)| (a weakly coupled vertex makes the connected sum
// small); zero padding.
__global__ void mc_features_kernel(const int *__restrict__ X, const int *__restrict__ idx, int count, int n,
                                   int win, int mtau, const double *__restrict__ g0, __nv_bfloat16 *F, int Bp) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= Bp) return;
    __nv_bfloat16 *f = F + static_cast<size_t>(k) * kMlpIn;
    for (int q = 0; q < kMlpIn; ++q) f[q] = __float2bfloat16_rn(0.f);
    if (k >= count) return;
    const int w = idx ? idx[k] : k;
    const int *xw = X + static_cast<size_t>(w) * n * 3;
    int ord[16];
    for (int i = 0; i < n; ++i) ord[i] = i;
    for (int i = 1; i < n; ++i) {  // insertion sort by time index
        const int o = ord[i];
        int j = i - 1;
        while (j >= 0 && xw[3 * ord[j] + 2] > xw[3 * o + 2]) {
            ord[j + 1] = ord[j];
            --j;
        }
        ord[j + 1] = o;
    }
    const int x0 = xw[3 * ord[0]], y0 = xw[3 * ord[0] + 1], m0 = xw[3 * ord[0] + 2];
    const float sw = 1.f / win, sm = 1.f / mtau;
    for (int i = 0; i < n && i < 14; ++i) {
        const int o = ord[i];
        f[3 * i + 0] = __float2bfloat16_rn((xw[3 * o] - x0) * sw);
        f[3 * i + 1] = __float2bfloat16_rn((xw[3 * o + 1] - y0) * sw);
        f[3 * i + 2] = __float2bfloat16_rn((xw[3 * o + 2] - m0) * sm);
    }
    f[42] = __float2bfloat16_rn(n / 14.f);
    float cpl[16];
    for (int i = 0; i < n; ++i) {
        double sum = 0.0;
        for (int j = 0; j < n; ++j) {
            if (j == i) continue;
            const int dx = abs(xw[3 * i] - xw[3 * j]), dy = abs(xw[3 * i + 1] - xw[3 * j + 1]);
            const int dm = xw[3 * i + 2] - xw[3 * j + 2] + mtau - 1;
            sum += fabs(g0[(static_cast<size_t>(dx) * win + dy) * (2 * mtau - 1) + dm]);
        }
        cpl[i] = log10f(static_cast<float>(sum) + 1e-30f);
    }
    for (int i = 1; i < n; ++i) {  // ascending
        const float v = cpl[i];
        int j = i - 1;
        while (j >= 0 && cpl[j] > v) {
            cpl[j + 1] = cpl[j];
            --j;
        }
        cpl[j + 1] = v;
    }
    for (int i = 0; i < n && i < 14; ++i) f[43 + i] = __float2bfloat16_rn(0.25f * cpl[i]);
}

// stage 1 of delayed acceptance: compacted list of surviving walkers
__global__ void mc_stage1_kernel(const float *__restrict__ s_new, const float *__restrict__ s_old,
                                 const float *__restrict__ u1, int W, int *idx, int *count) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    const float d = s_new[w] - s_old[w];
    if (d >= 0.f || u1[w] < expf(d)) idx[atomicAdd(count, 1)] = w;
}

// accept / reject candidates k < count (walker idx[k] or k); c_full[k * stride]
// is the exact connected sum of the proposal. Plain Metropolis when s_new is NULL.
__global__ void mc_accept_kernel(int *X, const int *__restrict__ Xp, double *weight, double *sign,
                                 float *s_cur, const float *__restrict__ s_new, const double *__restrict__ c_full,
                                 int64_t stride, const int *__restrict__ idx, int count, const float *__restrict__ u2,
                                 int n, int *accepted) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int w = idx ? idx[k] : k;
    const double c = c_full[static_cast<int64_t>(k) * stride];
    const double wn = fabs(c), wo = weight[w];
    double ratio = wo > 0.0 ? wn / wo : 1.0;
    if (s_new) ratio *= exp(static_cast<double>(s_cur[w]) - static_cast<double>(s_new[w]));
    if (isfinite(ratio) && static_cast<double>(u2[w]) < ratio) {
        const int *src = Xp + static_cast<size_t>(w) * n * 3;
        int *dst = X + static_cast<size_t>(w) * n * 3;
        for (int i = 0; i < 3 * n; ++i) dst[i] = src[i];
        weight[w] = wn;
        sign[w] = c >= 0.0 ? 1.0 : -1.0;
        if (s_new) s_cur[w] = s_new[w];
        atomicAdd(accepted, 1);
    }
}

}  // namespace apm

using namespace apm;

extern "C" {

apm_status_t apm_mc_propose(const int32_t *X, int W, int n, int win, int mtau, const float *u, int32_t *Xp,
                            apm_stream_t stream) {
    if (W < 0 || n < 1 || n > 16 || win < 1 || mtau < 1) return APM_ERR_ARG;
    if (W == 0) return APM_OK;
    if (!X || !u || !Xp) return APM_ERR_ARG;
    mc_propose_kernel<<<(W + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(X, W, n, win, mtau, u, Xp);
    return cudaGetLastError() == cudaSuccess ? APM_OK : APM_ERR_CUDA;
}

apm_status_t apm_mc_build_matrices(const int32_t *X, const int32_t *idx, int count, int n, int win, int mtau,
                                   const double *g0, double *A, apm_stream_t stream) {
    if (count < 0 || n < 1 || n > 16 || win < 1 || mtau < 1) return APM_ERR_ARG;
    if (count == 0) return APM_OK;
    if (!X || !g0 || !A) return APM_ERR_ARG;
    const int64_t total = static_cast<int64_t>(count) * n * n;
    mc_build_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        X, idx, count, n, win, mtau, g0, A);
    return cudaGetLastError() == cudaSuccess ? APM_OK : APM_ERR_CUDA;
}

apm_status_t apm_mc_features(const int32_t *X, const int32_t *idx, int count, int n, int win, int mtau,
                             const double *g0, uint16_t *F, int Bp, apm_stream_t stream) {
    if (count < 0 || Bp < count || n < 1 || n > 14 || win < 1 || mtau < 1) return APM_ERR_ARG;
    if (Bp == 0) return APM_OK;
    if (!X || !F || !g0) return APM_ERR_ARG;
    mc_features_kernel<<<(Bp + 127) / 128, 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        X, idx, count, n, win, mtau, g0, reinterpret_cast<__nv_bfloat16 *>(F), Bp);
    return cudaGetLastError() == cudaSuccess ? APM_OK : APM_ERR_CUDA;
}

apm_status_t apm_mc_stage1(const float *s_new, const float *s_old, const float *u1, int W, int32_t *idx,
                           int32_t *count, apm_stream_t stream) {
    if (W < 0 || !count) return APM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(count, 0, sizeof(int32_t), s) != cudaSuccess) return APM_ERR_CUDA;
    if (W == 0) return APM_OK;
    if (!s_new || !s_old || !u1 || !idx) return APM_ERR_ARG;
    mc_stage1_kernel<<<(W + 255) / 256, 256, 0, s>>>(s_new, s_old, u1, W, idx, count);
    return cudaGetLastError() == cudaSuccess ? APM_OK : APM_ERR_CUDA;
}

apm_status_t apm_mc_accept(int32_t *X, const int32_t *Xp, double *weight, double *sign, float *s_cur,
                           const float *s_new, const double *c_full, int64_t stride, const int32_t *idx, int count,
                           const float *u2, int n, int32_t *accepted, apm_stream_t stream) {
    if (count < 0 || n < 1 || n > 16 || stride < 1) return APM_ERR_ARG;
    if (count == 0) return APM_OK;
    if (!X || !Xp || !weight || !sign || !c_full || !u2 || !accepted || (s_new && !s_cur)) return APM_ERR_ARG;
    mc_accept_kernel<<<(count + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        X, Xp, weight, sign, s_cur, s_new, c_full, stride, idx, count, u2, n, accepted);
    return cudaGetLastError() == cudaSuccess ? APM_OK : APM_ERR_CUDA;
}

apm_status_t apm_mlp_workspace_size(int batch_padded, size_t *bytes) {
    if (!bytes || batch_padded < 0 || batch_padded % 64) return APM_ERR_ARG;
    *bytes = mlp_workspace_bytes(batch_padded);
    return APM_OK;
}

apm_status_t apm_mlp_sync_bf16(const apm_mlp *net, apm_stream_t stream) {
    if (!net || !net->param || !net->param_bf16) return APM_ERR_ARG;
    MlpParams P;
    mlp_bind(net, P);
    return mlp_refresh_bf16(P, reinterpret_cast<cudaStream_t>(stream)) ? APM_ERR_CUDA : APM_OK;
}

apm_status_t apm_mlp_forward(const apm_mlp *net, const uint16_t *X, int batch_padded, float *y, void *workspace,
                             size_t workspace_bytes, apm_stream_t stream) {
    if (!net || !net->param || !net->param_bf16 || batch_padded < 0 || batch_padded % 64) return APM_ERR_ARG;
    if (batch_padded == 0) return APM_OK;
    if (!X || !y) return APM_ERR_ARG;
    if (!workspace || workspace_bytes < mlp_workspace_bytes(batch_padded)) return APM_ERR_WORKSPACE;
    MlpParams P;
    mlp_bind(net, P);
    MlpWork w;
    mlp_work(workspace, batch_padded, w);
    return mlp_forward(P, reinterpret_cast<const __nv_bfloat16 *>(X), batch_padded, y, w,
                       reinterpret_cast<cudaStream_t>(stream))
               ? APM_ERR_CUDA
               : APM_OK;
}

apm_status_t apm_mlp_train_step(const apm_mlp *net, const uint16_t *X, const float *target, int batch_padded,
                                int batch_valid, float lr, int step, float *loss_acc, void *workspace,
                                size_t workspace_bytes, apm_stream_t stream) {
    if (!net || !net->param || !net->param_bf16 || !net->grad || !net->adam_m || !net->adam_v) return APM_ERR_ARG;
    if (batch_padded <= 0 || batch_padded % 64 || batch_valid < 1 || batch_valid > batch_padded || step < 1)
        return APM_ERR_ARG;
    if (!X || !target || !loss_acc) return APM_ERR_ARG;
    if (!workspace || workspace_bytes < mlp_workspace_bytes(batch_padded)) return APM_ERR_WORKSPACE;
    MlpParams P;
    mlp_bind(net, P);
    MlpWork w;
    mlp_work(workspace, batch_padded, w);
    return mlp_train_step(P, reinterpret_cast<const __nv_bfloat16 *>(X), target, batch_padded, batch_valid, w, lr,
                          step, loss_acc, reinterpret_cast<cudaStream_t>(stream))
               ? APM_ERR_CUDA
               : APM_OK;
}

apm_status_t apm_mlp_gradient(const apm_mlp *net, const uint16_t *X, const float *target, int batch_padded,
                              int batch_valid, float *loss_acc, void *workspace, size_t workspace_bytes,
                              apm_stream_t stream) {
    if (!net || !net->param || !net->param_bf16 || !net->grad) return APM_ERR_ARG;
    if (batch_padded <= 0 || batch_padded % 64 || batch_valid < 1 || batch_valid > batch_padded) return APM_ERR_ARG;
    if (!X || !target || !loss_acc) return APM_ERR_ARG;
    if (!workspace || workspace_bytes < mlp_workspace_bytes(batch_padded)) return APM_ERR_WORKSPACE;
    MlpParams P;
    mlp_bind(net, P);
    MlpWork w;
    mlp_work(workspace, batch_padded, w);
    return mlp_gradient(P, reinterpret_cast<const __nv_bfloat16 *>(X), target, batch_padded, batch_valid, w,
                        loss_acc, reinterpret_cast<cudaStream_t>(stream))
               ? APM_ERR_CUDA
               : APM_OK;
}

apm_status_t apm_mlp_adam_step(const apm_mlp *net, float lr, int step, apm_stream_t stream) {
    if (!net || !net->param || !net->param_bf16 || !net->grad || !net->adam_m || !net->adam_v || step < 1)
        return APM_ERR_ARG;
    MlpParams P;
    mlp_bind(net, P);
    return mlp_adam(P, lr, step, reinterpret_cast<cudaStream_t>(stream)) ? APM_ERR_CUDA : APM_OK;
}

apm_status_t apm_mlp_status(void *workspace, size_t workspace_bytes, uint32_t *flags, apm_stream_t stream) {
    if (!workspace || workspace_bytes < mlp_workspace_bytes(0)) return APM_ERR_WORKSPACE;
    uint32_t v = 0;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&v, workspace, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemsetAsync(workspace, 0, sizeof(v), s) != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return APM_ERR_CUDA;
    if (flags) *flags = v;
    return v ? APM_ERR_TIMEOUT : APM_OK;
}

apm_status_t apm_mlp_gemm_tn(const uint16_t *A, const uint16_t *Bt, const float *bias, float *C32, uint16_t *Cb,
                             int M, int N, int K, int relu, void *workspace, size_t workspace_bytes,
                             apm_stream_t stream) {
    if (!A || !Bt || (!C32 && !Cb) || M < 1 || N < 64 || K < 64 || N % 64 || K % 64) return APM_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(Bt) |
         reinterpret_cast<uintptr_t>(C32) | reinterpret_cast<uintptr_t>(Cb)) &
        15)
        return APM_ERR_ARG;
    if (!workspace || workspace_bytes < mlp_workspace_bytes(0)) return APM_ERR_WORKSPACE;
    MlpWork w;
    mlp_work(workspace, 0, w);
    return launch_tc_gemm_tn(reinterpret_cast<const __nv_bfloat16 *>(A), reinterpret_cast<const __nv_bfloat16 *>(Bt),
                             bias, C32, reinterpret_cast<__nv_bfloat16 *>(Cb), M, N, K, relu, w.part,
                             tc_gemm_split_floats(), w.err, reinterpret_cast<cudaStream_t>(stream))
               ? APM_ERR_CUDA
               : APM_OK;
}

}  // extern "C"
