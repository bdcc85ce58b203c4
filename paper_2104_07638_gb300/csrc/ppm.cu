// All permanent principal minors in O(3^n) (FP64).
//
// Paper: Section IV. Ryser's formula restricted to a subset S (Eq. ryser with
// the sum over column subsets T of S), the row sums r_i(T) = sum_{j in T} A_ij
// shared by every S containing T, and the products over S built one element at
// a time (Pi[S] = Pi[S \ {i}] * r_i(T)), O(3^n) in total. With the sign that
// makes Ryser's formula the permanent,
//     perm(A[S]) = sum_{T subset of S} prod_{i in S} u_i(T),
//     u_i(T) = r_i(T) for i in T, -r_i(T) for i not in T,
// (the factor (-1)^{|S|-|T|} distributed over the |S \ T| rows outside T).
//
// Mapping: one CTA per matrix (persistent), 16 warps. Each warp takes chunks of
// 64 consecutive column subsets T in Gray-code order (dynamic chunk counter),
// so r_i(T) (lane i) changes by one +-A_ij per step. For one T the warp expands
// all supersets S = T u R, R a subset of the free elements F = complement(T):
// lane t fixes membership of the 5 highest free elements by its bits (a
// product of at most 5 factors), then walks the subsets of the remaining free
// elements with one multiplication per subset (a fully unrolled binary
// recursion over up to 6 elements, an outer loop above that). Every product is
// added into perm[S] with a shared-memory atomic (the S of one T are distinct,
// different warps' T overlap); above n = 14 the accumulator is the output row in
// global memory.
#include <cuda_runtime.h>
#include <stdint.h>

#include "apm_internal.cuh"

namespace apm {

constexpr int kPpmWarps = 16;
constexpr int kPpmChunk = 64;
constexpr int kPpmSmemMaxN = 14;

template <int K, int G>
struct PpmExpand {
    static __device__ __forceinline__ void run(double *perm, double val, int S, const double (&ul)[6],
                                               const int (&el)[6]) {
        const double v2 = val * ul[K];
        atomicAdd(perm + (S | el[K]), v2);
        PpmExpand<K + 1, G>::run(perm, v2, S | el[K], ul, el);
        PpmExpand<K + 1, G>::run(perm, val, S, ul, el);
    }
};
template <int G>
struct PpmExpand<G, G> {
    static __device__ __forceinline__ void run(double *, double, int, const double (&)[6], const int (&)[6]) {}
};

__device__ __forceinline__ void ppm_expand(int G, double *perm, double val, int S, const double (&ul)[6],
                                           const int (&el)[6]) {
    switch (G) {
        case 1: PpmExpand<0, 1>::run(perm, val, S, ul, el); break;
        case 2: PpmExpand<0, 2>::run(perm, val, S, ul, el); break;
        case 3: PpmExpand<0, 3>::run(perm, val, S, ul, el); break;
        case 4: PpmExpand<0, 4>::run(perm, val, S, ul, el); break;
        case 5: PpmExpand<0, 5>::run(perm, val, S, ul, el); break;
        case 6: PpmExpand<0, 6>::run(perm, val, S, ul, el); break;
        default: break;
    }
}

// Contribution of one nonempty column subset T to every superset S.
__device__ __forceinline__ void ppm_one_T(double *perm, int n, int T, double r, int lane) {
    const bool inT = lane < n && ((T >> lane) & 1);
    const double u = lane < n ? (inT ? r : -r) : 1.0;
    // pre = prod_{i in T} u_i (lanes 0..15 hold the n <= 16 rows)
    double v = inT ? u : 1.0;
    v *= __shfl_xor_sync(0xffffffffu, v, 1);
    v *= __shfl_xor_sync(0xffffffffu, v, 2);
    v *= __shfl_xor_sync(0xffffffffu, v, 4);
    v *= __shfl_xor_sync(0xffffffffu, v, 8);
    const double pre = __shfl_sync(0xffffffffu, v, 0);
    int F = (~T) & ((1 << n) - 1);
    const int f = __popc(F);
    const int k = f < 5 ? f : 5;
    double val = pre;
    int Sb = T;
    for (int m = 0; m < k; ++m) {
        const int e = 31 - __clz(F);
        F ^= 1 << e;
        const double ue = __shfl_sync(0xffffffffu, u, e);
        if ((lane >> m) & 1) {
            val *= ue;
            Sb |= 1 << e;
        }
    }
    const bool active = lane < (1 << k);
    // remaining free elements F: the lowest G = min(|F|, 6) go to the unrolled
    // expansion, the rest (mid) to an outer loop
    const int g = __popc(F);
    const int G = g < 6 ? g : 6;
    double ul[6];
    int el[6];
    int Fl = F;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        int e = 0;
        if (q < G) {
            e = __ffs(Fl) - 1;
            Fl ^= 1 << e;
        }
        ul[q] = __shfl_sync(0xffffffffu, u, e);
        el[q] = 1 << e;
    }
    const int mid = Fl;  // elements above the lowest G
    const int nmid = __popc(mid);
    for (int t = 0; t < (1 << nmid); ++t) {
        double vm = val;
        int Sm = Sb;
        int mm = mid;
        for (int q = 0; q < nmid; ++q) {
            const int e = __ffs(mm) - 1;
            mm ^= 1 << e;
            const double ue = __shfl_sync(0xffffffffu, u, e);
            if ((t >> q) & 1) {
                vm *= ue;
                Sm |= 1 << e;
            }
        }
        if (active) {
            atomicAdd(perm + Sm, vm);
            ppm_expand(G, perm, vm, Sm, ul, el);
        }
    }
}

__global__ void __launch_bounds__(kPpmWarps * 32) ppm_kernel(const double *__restrict__ A, int n,
                                                             int64_t batch, double *perms,
                                                             int smem_arrays) {
    extern __shared__ __align__(16) double ppm_smem[];
    __shared__ int chunk_ctr;
    const int tid = threadIdx.x, lane = tid & 31;
    const int N = 1 << n;
    const int nn_pad = (n * n + 1) & ~1;
    double *sA = ppm_smem;
    for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
        double *perm = smem_arrays ? ppm_smem + nn_pad : perms + b * N;
        for (int t = tid; t < n * n; t += blockDim.x) sA[t] = __ldg(A + b * n * n + t);
        for (int t = tid; t < N; t += blockDim.x) perm[t] = t == 0 ? 1.0 : 0.0;
        if (tid == 0) chunk_ctr = 0;
        __syncthreads();
        const int nchunks = (N + kPpmChunk - 1) / kPpmChunk;
        while (true) {
            int k = 0;
            if (lane == 0) k = atomicAdd(&chunk_ctr, 1);
            k = __shfl_sync(0xffffffffu, k, 0);
            if (k >= nchunks) break;
            const int g0 = k * kPpmChunk;
            const int g1 = g0 + kPpmChunk < N ? g0 + kPpmChunk : N;
            int T = g0 ^ (g0 >> 1);
            double r = 0.0;
            if (lane < n)
                for (int j = 0; j < n; ++j)
                    if ((T >> j) & 1) r += sA[lane * n + j];
            for (int gi = g0; gi < g1; ++gi) {
                if (gi > g0) {
                    const int j = __ffs(gi) - 1;
                    T ^= 1 << j;
                    if (lane < n) r += ((T >> j) & 1) ? sA[lane * n + j] : -sA[lane * n + j];
                }
                if (T != 0) ppm_one_T(perm, n, T, r, lane);
            }
        }
        __syncthreads();
        if (smem_arrays) {
            double *out = perms + b * N;
            for (int t = tid; t < N; t += blockDim.x) out[t] = perm[t];
        }
        __syncthreads();
    }
}

int launch_ppm(const double *A, int n, int64_t batch, double *perms, cudaStream_t s) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int smem_arrays = n <= kPpmSmemMaxN ? 1 : 0;
    const size_t smem = sizeof(double) * (((n * n + 1) & ~1) + (smem_arrays ? (size_t(1) << n) : 0));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ppm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ppm_kernel, kPpmWarps * 32, smem);
    if (e != cudaSuccess) return static_cast<int>(e);
    if (per_sm < 1) return static_cast<int>(cudaErrorInvalidConfiguration);
    int64_t g = static_cast<int64_t>(sms) * per_sm;
    if (batch < g) g = batch;
    ppm_kernel<<<static_cast<int>(g), kPpmWarps * 32, smem, s>>>(A, n, batch, perms, smem_arrays);
    return static_cast<int>(cudaGetLastError());
}

}  // namespace apm
