// FP64 throughput microbenchmark: 8 independent fused-multiply-add chains per
// thread. It measures the denominator of the FP64 roofline of the minor and
// connected-sum kernels (the chip's published FP64 rate is a nominal figure).
#include <cuda_runtime.h>

#include "apm_internal.cuh"

namespace apm {

__global__ void fp64_probe_kernel(double *sink, int iters) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    double x0 = 1e-9 * t, x1 = x0 + 1e-3, x2 = x0 + 2e-3, x3 = x0 + 3e-3;
    double x4 = x0 + 4e-3, x5 = x0 + 5e-3, x6 = x0 + 6e-3, x7 = x0 + 7e-3;
    const double a = 0.9999999, b = 1e-7;
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b);
        x1 = fma(x1, a, b);
        x2 = fma(x2, a, b);
        x3 = fma(x3, a, b);
        x4 = fma(x4, a, b);
        x5 = fma(x5, a, b);
        x6 = fma(x6, a, b);
        x7 = fma(x7, a, b);
    }
    sink[t] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

int launch_fp64_probe(double *sink, int blocks, int threads, int iters, cudaStream_t s) {
    fp64_probe_kernel<<<blocks, threads, 0, s>>>(sink, iters);
    return static_cast<int>(cudaGetLastError());
}

}  // namespace apm
