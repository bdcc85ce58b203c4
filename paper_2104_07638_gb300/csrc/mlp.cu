// Surrogate network of the learned Monte Carlo proposal: a 4-layer MLP
// (in 64 -> 256 -> 256 -> 256 -> 1, ReLU) with BF16 weights and activations,
// FP32 accumulation and FP32 master weights trained by Adam.
//
// GEMMs are "TN": C[M x N] = A[M x K] * Bt[N x K]^T with both operands
// K-contiguous BF16, on the tensor cores (tcgen05, tc_gemm.cu); the forms that
// need a transposed operand get it from transpose_bf16_kernel. M a multiple of
// 64, N of 64, K of 64. The network is tiny next to the FP64 minor kernels.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "apm_internal.cuh"

namespace apm {

// bf16 transpose: out[c][r] = in[r][c], in is R x C
__global__ void transpose_bf16_kernel(const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *out, int R, int C) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < R && c < C) tile[i][threadIdx.x] = in[static_cast<size_t>(r) * C + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < R && c < C) out[static_cast<size_t>(c) * R + r] = tile[threadIdx.x][i];
    }
}

// last layer: y[b] = sum_i H[b][i] w[i] + b0 (one warp per row, 256 inputs)
__global__ void head_forward_kernel(const __nv_bfloat16 *__restrict__ H, const __nv_bfloat16 *__restrict__ w,
                                    const float *__restrict__ b0, float *y, int B, int D) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= B) return;
    float s = 0.f;
    for (int i = lane; i < D; i += 32)
        s = fmaf(__bfloat162float(H[static_cast<size_t>(row) * D + i]), __bfloat162float(w[i]), s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) y[row] = s + b0[0];
}

// dy = 2 (y - target) / B_valid for rows < B_valid (0 for padding rows); loss partial sums
__global__ void mse_grad_kernel(const float *__restrict__ y, const float *__restrict__ target, float *dy,
                                int Bp, int B_valid, float *loss_part) {
    // dy = 2 (y - t) / B_valid on the valid rows; the block's share of the loss
    // into loss_part[block] (added in a fixed order later: deterministic)
    __shared__ float red[256];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    float d = 0.f, l = 0.f;
    if (i < B_valid) {
        const float e = y[i] - target[i];
        d = 2.f * e / static_cast<float>(B_valid);
        l = e * e / static_cast<float>(B_valid);
    }
    if (i < Bp) dy[i] = d;
    red[threadIdx.x] = l;
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0];
}

// head backward: dZ[b][i] = (H[b][i] > 0) ? dy[b] * w[i] : 0 (fp32 and bf16);
// per block of rows the partial sums of dw[i] = sum_b dy[b] H[b][i],
// dbz[i] = sum_b dZ[b][i] and db = sum_b dy[b] (added over the blocks in a
// fixed order by col_sum_kernel: no atomics, so training is deterministic)
__global__ void head_backward_kernel(const __nv_bfloat16 *__restrict__ H, const __nv_bfloat16 *__restrict__ w,
                                     const float *__restrict__ dy, float *dZ32, __nv_bfloat16 *dZb, float *pw,
                                     float *pb, float *pz, int Bp, int D, int rows_per_block) {
    const int i = threadIdx.x;  // column, blockDim.x == D
    const int r0 = blockIdx.x * rows_per_block;
    float accw = 0.f, accb = 0.f, accz = 0.f;
    const float wi = __bfloat162float(w[i]);
    for (int r = r0; r < r0 + rows_per_block && r < Bp; ++r) {
        const float h = __bfloat162float(H[static_cast<size_t>(r) * D + i]);
        const float g = dy[r];
        const float z = h > 0.f ? g * wi : 0.f;
        dZ32[static_cast<size_t>(r) * D + i] = z;
        dZb[static_cast<size_t>(r) * D + i] = __float2bfloat16_rn(z);
        accw = fmaf(g, h, accw);
        accb += g;
        accz += z;
    }
    pw[static_cast<size_t>(blockIdx.x) * D + i] = accw;
    pz[static_cast<size_t>(blockIdx.x) * D + i] = accz;
    if (i == 0) pb[blockIdx.x] = accb;
}

// dZ = dH * (H > 0) (fp32 in, fp32 + bf16 out); per block of rows the partial
// column sums (the bias gradient) into pdb[block][i]
__global__ void relu_backward_kernel(const float *__restrict__ dH, const __nv_bfloat16 *__restrict__ H,
                                     float *dZ32, __nv_bfloat16 *dZb, float *pdb, int Bp, int D,
                                     int rows_per_block) {
    const int i = threadIdx.x;
    const int r0 = blockIdx.x * rows_per_block;
    float acc = 0.f;
    for (int r = r0; r < r0 + rows_per_block && r < Bp; ++r) {
        const size_t o = static_cast<size_t>(r) * D + i;
        const float z = __bfloat162float(H[o]) > 0.f ? dH[o] : 0.f;
        dZ32[o] = z;
        dZb[o] = __float2bfloat16_rn(z);
        acc += z;
    }
    pdb[static_cast<size_t>(blockIdx.x) * D + i] = acc;
}

// out[i] (+)= sum over the blocks k = 0 .. nblk-1, in that order, of part[k][i]
__global__ void col_sum_kernel(const float *__restrict__ part, float *out, int nblk, int D, int accumulate) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= D) return;
    float acc = 0.f;
    for (int k = 0; k < nblk; ++k) acc += part[static_cast<size_t>(k) * D + i];
    out[i] = accumulate ? out[i] + acc : acc;
}

// Adam on the flat fp32 parameter vector; refreshes the bf16 copy
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, __nv_bfloat16 *pb, int count, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
}

__global__ void f32_to_bf16_kernel(const float *in, __nv_bfloat16 *out, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] = __float2bfloat16_rn(in[i]);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

static size_t al(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kMlpRowsPerBlock = 64;  // rows per block of the backward column sums

// layout: status word (offset 0), split-K partials, activations and gradients,
// per-block partial column sums of the backward pass
size_t mlp_workspace_bytes(int Bp) {
    const size_t act = static_cast<size_t>(Bp) * kMlpH;
    const size_t nblk = static_cast<size_t>(Bp + kMlpRowsPerBlock - 1) / kMlpRowsPerBlock + 1;
    return al(sizeof(uint32_t)) + al(tc_gemm_split_floats() * 4) + 3 * al(act * 2) + 2 * al(static_cast<size_t>(Bp) * 4) + 2 * al(act * 4) + al(act * 2) +
           2 * al(act * 2) + al(static_cast<size_t>(kMlpH) * kMlpH * 2) + 2 * al(nblk * kMlpH * 4) +
           2 * al(static_cast<size_t>(Bp / 256 + 1 > nblk ? Bp / 256 + 1 : nblk) * 4);
}

void mlp_work(void *ws, int Bp, MlpWork &w) {
    unsigned char *p = static_cast<unsigned char *>(ws);
    const size_t act = static_cast<size_t>(Bp) * kMlpH;
    auto take = [&](size_t bytes) {
        unsigned char *q = p;
        p += al(bytes);
        return q;
    };
    w.err = reinterpret_cast<uint32_t *>(take(sizeof(uint32_t)));
    w.part = reinterpret_cast<float *>(take(tc_gemm_split_floats() * 4));
    w.h1 = reinterpret_cast<__nv_bfloat16 *>(take(act * 2));
    w.h2 = reinterpret_cast<__nv_bfloat16 *>(take(act * 2));
    w.h3 = reinterpret_cast<__nv_bfloat16 *>(take(act * 2));
    w.y = reinterpret_cast<float *>(take(static_cast<size_t>(Bp) * 4));
    w.dy = reinterpret_cast<float *>(take(static_cast<size_t>(Bp) * 4));
    w.dz32 = reinterpret_cast<float *>(take(act * 4));
    w.dh32 = reinterpret_cast<float *>(take(act * 4));
    w.dzb = reinterpret_cast<__nv_bfloat16 *>(take(act * 2));
    w.t1 = reinterpret_cast<__nv_bfloat16 *>(take(act * 2));
    w.t2 = reinterpret_cast<__nv_bfloat16 *>(take(act * 2));
    w.wt = reinterpret_cast<__nv_bfloat16 *>(take(static_cast<size_t>(kMlpH) * kMlpH * 2));
    const size_t nblk = static_cast<size_t>(Bp + kMlpRowsPerBlock - 1) / kMlpRowsPerBlock + 1;
    const size_t np = static_cast<size_t>(Bp / 256 + 1 > nblk ? Bp / 256 + 1 : nblk);
    w.pcol = reinterpret_cast<float *>(take(nblk * kMlpH * 4));
    w.pcol2 = reinterpret_cast<float *>(take(nblk * kMlpH * 4));
    w.pvec = reinterpret_cast<float *>(take(np * 4));
    w.pvec2 = reinterpret_cast<float *>(take(np * 4));
}

void mlp_bind(const apm_mlp *net, MlpParams &P) {
    P.param = net->param;
    P.grad = net->grad;
    P.m = net->adam_m;
    P.v = net->adam_v;
    P.pb = reinterpret_cast<__nv_bfloat16 *>(net->param_bf16);
    P.w1b = P.pb + kOffW1;
    P.w2b = P.pb + kOffW2;
    P.w3b = P.pb + kOffW3;
    P.w4b = P.pb + kOffW4;
    P.b1 = P.param + kOffB1;
    P.b2 = P.param + kOffB2;
    P.b3 = P.param + kOffB3;
    P.b4 = P.param + kOffB4;
}

static int gemm_tn(const __nv_bfloat16 *A, const __nv_bfloat16 *Bt, const float *bias, float *C32,
                   __nv_bfloat16 *Cb, int M, int N, int K, int relu, MlpWork &w, cudaStream_t s) {
    return launch_tc_gemm_tn(A, Bt, bias, C32, Cb, M, N, K, relu, w.part, tc_gemm_split_floats(), w.err, s);
}

static int transpose(const __nv_bfloat16 *in, __nv_bfloat16 *out, int R, int C, cudaStream_t s) {
    dim3 grid((C + 31) / 32, (R + 31) / 32);
    transpose_bf16_kernel<<<grid, dim3(32, 8), 0, s>>>(in, out, R, C);
    return static_cast<int>(cudaGetLastError());
}

int mlp_forward(const MlpParams &P, const __nv_bfloat16 *X, int Bp, float *y, MlpWork &w, cudaStream_t s) {
    int e;
    if ((e = gemm_tn(X, P.w1b, P.b1, nullptr, w.h1, Bp, kMlpH, kMlpIn, 1, w, s))) return e;
    if ((e = gemm_tn(w.h1, P.w2b, P.b2, nullptr, w.h2, Bp, kMlpH, kMlpH, 1, w, s))) return e;
    if ((e = gemm_tn(w.h2, P.w3b, P.b3, nullptr, w.h3, Bp, kMlpH, kMlpH, 1, w, s))) return e;
    head_forward_kernel<<<(Bp + 7) / 8, 256, 0, s>>>(w.h3, P.w4b, P.b4, y, Bp, kMlpH);
    return static_cast<int>(cudaGetLastError());
}

// The gradient of the mean squared error over the first B_valid rows into
// P.grad (forward pass, then backpropagation layer by layer).
int mlp_gradient(MlpParams &P, const __nv_bfloat16 *X, const float *target, int Bp, int B_valid, MlpWork &w,
                 float *loss_acc, cudaStream_t s) {
    int e;
    if ((e = mlp_forward(P, X, Bp, w.y, w, s))) return e;
    cudaMemsetAsync(P.grad, 0, sizeof(float) * kMlpParams, s);
    const int nl = (Bp + 255) / 256;
    mse_grad_kernel<<<nl, 256, 0, s>>>(w.y, target, w.dy, Bp, B_valid, w.pvec2);
    col_sum_kernel<<<1, 32, 0, s>>>(w.pvec2, loss_acc, nl, 1, 1);
    const int rpb = kMlpRowsPerBlock;
    const int nblk = (Bp + rpb - 1) / rpb;
    float *g = P.grad;
    float *gw1 = g + kOffW1, *gb1 = g + kOffB1, *gw2 = g + kOffW2, *gb2 = g + kOffB2;
    float *gw3 = g + kOffW3, *gb3 = g + kOffB3, *gw4 = g + kOffW4, *gb4 = g + kOffB4;
    // head: dZ3 = dH3 * (H3 > 0), dw4, db4, db3 = column sums of dZ3
    head_backward_kernel<<<nblk, kMlpH, 0, s>>>(w.h3, P.w4b, w.dy, w.dz32, w.dzb, w.pcol, w.pvec, w.pcol2, Bp,
                                                kMlpH, rpb);
    col_sum_kernel<<<1, kMlpH, 0, s>>>(w.pcol, gw4, nblk, kMlpH, 0);
    col_sum_kernel<<<1, kMlpH, 0, s>>>(w.pcol2, gb3, nblk, kMlpH, 0);
    col_sum_kernel<<<1, 32, 0, s>>>(w.pvec, gb4, nblk, 1, 0);
    // layer 3: dW3 = dZ3^T H2 ; dH2 = dZ3 W3
    if ((e = transpose(w.dzb, w.t1, Bp, kMlpH, s))) return e;  // dZ3^T [256 x Bp]
    if ((e = transpose(w.h2, w.t2, Bp, kMlpH, s))) return e;   // H2^T  [256 x Bp]
    if ((e = gemm_tn(w.t1, w.t2, nullptr, gw3, nullptr, kMlpH, kMlpH, Bp, 0, w, s))) return e;
    if ((e = transpose(P.w3b, w.wt, kMlpH, kMlpH, s))) return e;  // W3 stored [out x in] -> [in x out]
    if ((e = gemm_tn(w.dzb, w.wt, nullptr, w.dh32, nullptr, Bp, kMlpH, kMlpH, 0, w, s))) return e;
    // layer 2
    relu_backward_kernel<<<nblk, kMlpH, 0, s>>>(w.dh32, w.h2, w.dz32, w.dzb, w.pcol, Bp, kMlpH, rpb);
    col_sum_kernel<<<1, kMlpH, 0, s>>>(w.pcol, gb2, nblk, kMlpH, 0);
    if ((e = transpose(w.dzb, w.t1, Bp, kMlpH, s))) return e;  // dZ2^T
    if ((e = transpose(w.h1, w.t2, Bp, kMlpH, s))) return e;   // H1^T
    if ((e = gemm_tn(w.t1, w.t2, nullptr, gw2, nullptr, kMlpH, kMlpH, Bp, 0, w, s))) return e;
    if ((e = transpose(P.w2b, w.wt, kMlpH, kMlpH, s))) return e;
    if ((e = gemm_tn(w.dzb, w.wt, nullptr, w.dh32, nullptr, Bp, kMlpH, kMlpH, 0, w, s))) return e;
    // layer 1
    relu_backward_kernel<<<nblk, kMlpH, 0, s>>>(w.dh32, w.h1, w.dz32, w.dzb, w.pcol, Bp, kMlpH, rpb);
    col_sum_kernel<<<1, kMlpH, 0, s>>>(w.pcol, gb1, nblk, kMlpH, 0);
    if ((e = transpose(w.dzb, w.t1, Bp, kMlpH, s))) return e;  // dZ1^T [256 x Bp]
    if ((e = transpose(X, w.t2, Bp, kMlpIn, s))) return e;     // X^T   [64 x Bp]
    if ((e = gemm_tn(w.t1, w.t2, nullptr, gw1, nullptr, kMlpH, kMlpIn, Bp, 0, w, s))) return e;
    return static_cast<int>(cudaGetLastError());
}

// One Adam step from P.grad (step >= 1 for the bias correction); refreshes the
// BF16 copy of the weights.
int mlp_adam(MlpParams &P, float lr, int step, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, static_cast<float>(step)), c2 = 1.f - powf(b2, static_cast<float>(step));
    adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(P.param, P.grad, P.m, P.v, P.pb, kMlpParams, lr, b1, b2,
                                                         eps, c1, c2);
    return static_cast<int>(cudaGetLastError());
}

int mlp_train_step(MlpParams &P, const __nv_bfloat16 *X, const float *target, int Bp, int B_valid, MlpWork &w,
                   float lr, int step, float *loss_acc, cudaStream_t s) {
    const int e = mlp_gradient(P, X, target, Bp, B_valid, w, loss_acc, s);
    return e ? e : mlp_adam(P, lr, step, s);
}

int mlp_refresh_bf16(MlpParams &P, cudaStream_t s) {
    f32_to_bf16_kernel<<<(kMlpParams + 255) / 256, 256, 0, s>>>(P.param, P.pb, kMlpParams);
    return static_cast<int>(cudaGetLastError());
}

}  // namespace apm
