// Per-order sums of the connected sums of whole vertex sets: the data of the
// power-series estimator (Section V, Eq. series), which sums the order-m
// integrals of c_m over the configurations sampled at each order m. A rank
// reduces its own rows here; ranks then add these few numbers on the host.
//
// One CTA: for each order m, every thread sums its rows of that order in a
// fixed stride, and a shared-memory tree adds the threads' sums in a fixed
// pairing, so the result does not depend on scheduling.
#include <cuda_runtime.h>
#include <stdint.h>

#include "apm_internal.cuh"

namespace apm {

constexpr int kSumThreads = 512;

__global__ void __launch_bounds__(kSumThreads) order_sums_kernel(const double *__restrict__ c, int n_fixed,
                                                                 const int32_t *__restrict__ n_arr,
                                                                 const int64_t *__restrict__ c_off, int64_t batch,
                                                                 int n_max, double *out) {
    __shared__ double red[4][kSumThreads];
    const int t = threadIdx.x;
    for (int m = 0; m <= n_max; ++m) {
        double cnt = 0.0, s1 = 0.0, sa = 0.0, s2 = 0.0;
        if (m >= 1 && (n_arr || m == n_fixed)) {
            for (int64_t b = t; b < batch; b += kSumThreads) {
                const int nb = n_arr ? n_arr[b] : n_fixed;
                if (nb != m) continue;
                const int64_t row = c_off ? c_off[b] : b << m;
                const double v = c[row + (int64_t(1) << m) - 1];
                cnt += 1.0;
                s1 += v;
                sa += fabs(v);
                s2 = fma(v, v, s2);
            }
        }
        red[0][t] = cnt;
        red[1][t] = s1;
        red[2][t] = sa;
        red[3][t] = s2;
        __syncthreads();
        for (int h = kSumThreads / 2; h > 0; h >>= 1) {
            if (t < h)
#pragma unroll
                for (int k = 0; k < 4; ++k) red[k][t] += red[k][t + h];
            __syncthreads();
        }
        if (t < 4) out[4 * m + t] = red[t][0];
        __syncthreads();
    }
}

int launch_order_sums(const double *c, int n_fixed, const int32_t *n_arr, const int64_t *c_off, int64_t batch,
                      int n_max, double *out, cudaStream_t s) {
    order_sums_kernel<<<1, kSumThreads, 0, s>>>(c, n_fixed, n_arr, c_off, batch, n_max, out);
    return static_cast<int>(cudaGetLastError());
}

}  // namespace apm

extern "C" apm_status_t apm_order_sums(const double *c, int n_fixed, const int32_t *n_arr, const int64_t *c_off,
                                      int64_t batch, int n_max, double *out, apm_stream_t stream) {
    if (n_max < 1 || n_max > 16 || batch < 0 || !out) return APM_ERR_ARG;
    if ((n_arr == nullptr) != (c_off == nullptr)) return APM_ERR_ARG;
    if (!n_arr && (n_fixed < 1 || n_fixed > n_max)) return APM_ERR_ARG;
    if (batch > 0 && !c) return APM_ERR_ARG;
    const int e = apm::launch_order_sums(c, n_fixed, n_arr, c_off, batch, n_max, out,
                                         reinterpret_cast<cudaStream_t>(stream));
    return e ? APM_ERR_CUDA : APM_OK;
}
