// FP64 throughput microbenchmark: 16 independent fused-multiply-add chains per
// thread. It measures the denominator of the FP64 roofline of the minor and
// connected-sum kernels (the chip's published FP64 rate is a nominal figure).
#include <cuda_runtime.h>

#include "apm_internal.cuh"

namespace apm {

__global__ void fp64_probe_kernel(double *sink, int iters) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double x[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = 1e-9 * t + 1e-3 * k;
    const double a = 0.9999999, b = 1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 16; ++k) s += x[k];
    sink[t] = s;
}

int launch_fp64_probe(double *sink, int blocks, int threads, int iters, cudaStream_t s) {
    fp64_probe_kernel<<<blocks, threads, 0, s>>>(sink, iters);
    return static_cast<int>(cudaGetLastError());
}

}  // namespace apm
