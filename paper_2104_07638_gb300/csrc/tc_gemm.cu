// BF16 "TN" GEMM of the surrogate network on the fifth-generation tensor cores:
//     C[M x N] = A[M x K] * Bt[N x K]^T (+ bias[N]) (ReLU), FP32 accumulation,
// both operands K-contiguous BF16 (row-major activations times weights stored
// [out][in], and the transposed forms of the gradient products).
//
// One CTA of 128 threads per 128 x BN tile of C (BN = 128, or 64 when N is not
// a multiple of 128). Products whose K is long next to M x N (the weight
// gradients, K = batch) split K over gridDim.z slices; each slice stores an
// FP32 partial tile and a second kernel adds the slices in slice order, so the
// result does not depend on scheduling.
//  * Operands: TMA tiled loads (cp.async.bulk.tensor.2d) of 128 x 64 and BN x 64
//    BF16 boxes with the 128-byte swizzle into a ring of three shared-memory
//    stages; rows past M or N arrive as zeros.
//  * Products: one thread issues tcgen05.mma (kind::f16, M = 128, N = BN, K = 16
//    per instruction) with both operands read from shared memory through matrix
//    descriptors (K-major, 128-byte swizzle: 8-row atoms of 1024 bytes), into an
//    FP32 accumulator of BN columns in tensor memory; tcgen05.commit on a stage's
//    mbarrier frees its buffers for the next load.
//  * Epilogue: warp w owns accumulator rows 32w..32w+31 (its quarter of the
//    tensor-memory lanes), reads them with tcgen05.ld 16 columns at a time, adds
//    the bias, applies the ReLU and stores FP32 and/or BF16 rows.
// Every mbarrier wait gives up after one second of %globaltimer: the CTA then
// sets bit 0 of *err, waits (with the same limit) for the loads it has in
// flight and for its issued products, releases its tensor memory and returns
// without storing.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "apm_internal.cuh"

namespace apm {

constexpr int kTcM = 128;                                  // rows per tile = tensor-memory lanes
constexpr int kTcK = 64;                                   // K per stage: one 128-byte swizzle row
constexpr int kTcStages = 3;
constexpr int kTcThreads = 128;
constexpr uint32_t kTcABytes = kTcM * kTcK * 2;            // 16 KB
constexpr uint32_t kTcStageBytes = kTcABytes + 128 * kTcK * 2;  // A + B (BN <= 128)
constexpr size_t kTcSmemBytes = 1024 + kTcStages * kTcStageBytes + 128;  // alignment slack + barriers
constexpr unsigned long long kTcWaitNs = 1000000000ull;
constexpr int kTcMaxSplits = 32;

__device__ __forceinline__ uint32_t sh_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// true once the phase of the given parity has completed, false after the limit
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = global_ns();
    while (true) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        if (ok) return true;
        if (global_ns() - t0 > kTcWaitNs) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// shared-memory matrix descriptor: K-major operand in 128-byte-swizzled 8-row
// atoms (1024 bytes apart), start address in 16-byte units; the leading offset
// is not used by this layout
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    return static_cast<uint64_t>((addr & 0x3FFFF) >> 4) | (1ull << 16) | (static_cast<uint64_t>(1024 >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(n >> 3) << 17) |
           (static_cast<uint32_t>(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// the mbarrier gets one arrival once every product issued so far by this thread is done
__device__ __forceinline__ void tc_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}

struct TcGemmArgs {
    const float *bias;
    float *C32;           // [M][N] FP32 result, or the split partials [splits][M][N]
    __nv_bfloat16 *Cb;    // [M][N] BF16 result (single slice only)
    uint32_t *err;
    int M, N, BN, nk, kb_per_split, relu;
};

__global__ void __launch_bounds__(kTcThreads) tc_gemm_tn_kernel(const __grid_constant__ CUtensorMap mapA,
                                                                const __grid_constant__ CUtensorMap mapB,
                                                                const TcGemmArgs g) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    __shared__ uint32_t s_tmem;
    __shared__ int s_bad;
    const uint32_t raw = sh_addr(tc_smem_raw);
    const uint32_t sbase = (raw + 1023u) & ~1023u;  // swizzle atoms want 1024-byte alignment
    const uint32_t bar0 = sbase + kTcStages * kTcStageBytes;
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto empty = [&](int s) { return bar0 + 8u * (kTcStages + s); };
    const uint32_t done = bar0 + 8u * (2 * kTcStages);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int BN = g.BN;
    const int n0 = blockIdx.x * BN, m0 = blockIdx.y * kTcM;
    const int kb0 = blockIdx.z * g.kb_per_split;
    const int nk = min(g.kb_per_split, g.nk - kb0);
    const uint32_t stage_tx = kTcABytes + static_cast<uint32_t>(BN) * kTcK * 2;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(sh_addr(&s_tmem)),
                     "r"(BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        mbar_init(done, 1);
        s_bad = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;

    if (tid == 0) {
        const uint32_t idesc = idesc_bf16(kTcM, BN);
        int issued = 0, waited = 0;
        bool bad = false;
        auto load = [&](int kb) {
            const int s = kb % kTcStages;
            const uint32_t a = sbase + s * kTcStageBytes;
            mbar_expect_tx(full(s), stage_tx);
            tma_load_2d(a, &mapA, (kb0 + kb) * kTcK, m0, full(s));
            tma_load_2d(a + kTcABytes, &mapB, (kb0 + kb) * kTcK, n0, full(s));
        };
        for (; issued < nk && issued < kTcStages; ++issued) load(issued);
        for (int kb = 0; kb < nk; ++kb) {
            const int s = kb % kTcStages;
            if (!mbar_wait(full(s), (kb / kTcStages) & 1)) {
                bad = true;
                break;
            }
            waited = kb + 1;
            tc_fence_after();
            const uint32_t a = sbase + s * kTcStageBytes, b = a + kTcABytes;
#pragma unroll
            for (int kk = 0; kk < kTcK / 16; ++kk)
                tc_mma(tmem, smem_desc_sw128(a + 32 * kk), smem_desc_sw128(b + 32 * kk), idesc, (kb | kk) != 0);
            tc_commit(empty(s));
            // refill the stage of the previous k-block once its products are done
            if (kb >= 1 && issued < nk) {
                if (!mbar_wait(empty((kb - 1) % kTcStages), ((kb - 1) / kTcStages) & 1)) {
                    bad = true;
                    break;
                }
                load(issued++);
            }
        }
        if (bad) {
            for (int q = waited; q < issued; ++q) mbar_wait(full(q % kTcStages), (q / kTcStages) & 1);
            s_bad = 1;
        }
        tc_commit(done);  // all issued products done (at once when none was issued)
    }
    const bool ok = mbar_wait(done, 0);
    if (!ok) s_bad = 1;
    tc_fence_after();
    __syncthreads();
    if (!s_bad) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t trow = tmem + (static_cast<uint32_t>(warp * 32) << 16);
        const bool split = gridDim.z > 1;
        float *c32 = g.C32 ? g.C32 + (split ? static_cast<size_t>(blockIdx.z) * g.M * g.N : 0) : nullptr;
        for (int c = 0; c < BN; c += 16) {
            uint32_t r[16];
            tmem_ld16(trow + c, r);
            if (row < g.M) {
                float v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    v[j] = __uint_as_float(r[j]);
                    if (!split && g.bias) v[j] += g.bias[n0 + c + j];
                    if (!split && g.relu) v[j] = fmaxf(v[j], 0.f);
                }
                const size_t o = static_cast<size_t>(row) * g.N + n0 + c;
                if (c32) {
                    float4 *d = reinterpret_cast<float4 *>(c32 + o);
#pragma unroll
                    for (int q = 0; q < 4; ++q) d[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
                if (g.Cb && !split) {
                    uint4 pk[2];
                    uint32_t *w = reinterpret_cast<uint32_t *>(pk);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * q], v[2 * q + 1]);
                        w[q] = *reinterpret_cast<const uint32_t *>(&h);
                    }
                    uint4 *d = reinterpret_cast<uint4 *>(g.Cb + o);
                    d[0] = pk[0];
                    d[1] = pk[1];
                }
            }
        }
    }
    if (s_bad && tid == 0) atomicOr(g.err, 1u);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
    }
}

// C[i] = sum over the slices z (in order) of part[z][i]
__global__ void split_sum_kernel(const float *__restrict__ part, float *C, int count, int splits) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float s = part[i];
    for (int z = 1; z < splits; ++z) s += part[static_cast<size_t>(z) * count + i];
    C[i] = s;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

typedef CUresult (*TensorMapEncodeTiled)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                         const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                         CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                         CUtensorMapFloatOOBfill);

static TensorMapEncodeTiled encode_tiled() {
    static std::once_flag once;
    static TensorMapEncodeTiled fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<TensorMapEncodeTiled>(p);
    });
    return fn;
}

// rows x K BF16, row-major, boxes of box_rows x 64 with the 128-byte swizzle
static bool make_map(CUtensorMap *m, const __nv_bfloat16 *base, int rows, int K, int box_rows) {
    TensorMapEncodeTiled fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {static_cast<cuuint64_t>(K), static_cast<cuuint64_t>(rows)};
    const cuuint64_t strides[1] = {static_cast<cuuint64_t>(K) * 2};
    const cuuint32_t box[2] = {static_cast<cuuint32_t>(kTcK), static_cast<cuuint32_t>(box_rows)};
    const cuuint32_t estr[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(base), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t tc_gemm_split_floats() { return static_cast<size_t>(kTcMaxSplits) * kMlpH * kMlpH; }

int launch_tc_gemm_tn(const __nv_bfloat16 *A, const __nv_bfloat16 *Bt, const float *bias, float *C32,
                      __nv_bfloat16 *Cb, int M, int N, int K, int relu, float *part, size_t part_floats,
                      uint32_t *err, cudaStream_t s) {
    if (M <= 0 || N <= 0 || K <= 0 || N % 64 || K % kTcK || !A || !Bt || !err || (!C32 && !Cb))
        return static_cast<int>(cudaErrorInvalidValue);
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(Bt)) & 15)
        return static_cast<int>(cudaErrorMisalignedAddress);
    const int BN = N % 128 == 0 ? 128 : 64;
    const int nk = K / kTcK;
    const int tiles = ((M + kTcM - 1) / kTcM) * (N / BN);
    // split K where the tiles alone would leave most SMs idle (only for a plain
    // FP32 result: the bias, the ReLU and the BF16 copy need the whole sum)
    int splits = 1;
    if (part && C32 && !Cb && !bias && !relu && tiles < 64) {
        splits = nk / 8;
        if (splits > kTcMaxSplits) splits = kTcMaxSplits;
        while (splits > 1 && static_cast<size_t>(splits) * M * N > part_floats) --splits;
        if (splits < 1) splits = 1;
    }
    const int kb_per = (nk + splits - 1) / splits;
    splits = (nk + kb_per - 1) / kb_per;
    CUtensorMap mapA, mapB;
    if (!make_map(&mapA, A, M, K, kTcM) || !make_map(&mapB, Bt, N, K, BN))
        return static_cast<int>(cudaErrorInvalidValue);
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_tn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(kTcSmemBytes));
    if (e != cudaSuccess) return static_cast<int>(e);
    TcGemmArgs g{bias, splits > 1 ? part : C32, splits > 1 ? nullptr : Cb, err, M, N, BN, nk, kb_per, relu};
    dim3 grid(N / BN, (M + kTcM - 1) / kTcM, splits);
    tc_gemm_tn_kernel<<<grid, kTcThreads, kTcSmemBytes, s>>>(mapA, mapB, g);
    e = cudaGetLastError();
    if (e != cudaSuccess || splits == 1) return static_cast<int>(e);
    const int count = M * N;
    split_sum_kernel<<<(count + 255) / 256, 256, 0, s>>>(part, C32, count, splits);
    return static_cast<int>(cudaGetLastError());
}

}  // namespace apm
