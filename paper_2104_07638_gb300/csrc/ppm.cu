// All permanent principal minors in O(3^n) (FP64).
//
// Paper: Section IV. Ryser's formula restricted to a subset S (Eq. ryser with
// the sum over column subsets T of S), with the row sums r_i(T) = sum_{j in T}
// A_ij shared by every S containing T and the products over S built one
// element at a time, O(3^n) in total. With the sign that makes Ryser's formula
// the permanent:
//     perm(A[S]) = sum_{T subset of S} prod_{i in S} u_i(T),
//     u_i(T) = r_i(T) if i in T, -r_i(T) otherwise.
//
// Split every subset into a low part (elements 0..l-1, l = min(n,7)) and a high
// part (the other h = n-l elements): S = S_H u S_L, T = T_H u T_L. Then
//     perm[S_H u S_L] = sum_{T_H subset of S_H} sum_{T_L subset of S_L}
//                       alpha_{T_H,S_H}(T_L) * B_{T_H}(T_L, S_L),
//     alpha = prod_{i in S_H} u_i(T),   B = prod_{i in S_L} u_i(T),   T = T_H u T_L.
// For each T_H (outer loop, CTA-wide): the table U[T_L][i] = u_i(T_H u T_L) (one
// add per entry from precomputed row sums), then the 3^l entries of B, level by
// level over |S_L \ T_L|, one multiply each (B(T_L, S_L) = B(T_L, S_L \ {e})
// * u_e). For each S_H containing T_H (one warp per S_H): alpha for all T_L
// (|S_H| multiplies each), then for every S_L the sum over its submasks T_L, one
// FMA per (T, S) pair, with the 3^l terms cut into pieces of at most 24 and
// spread over the lanes by a precomputed longest-first assignment; the pieces of
// one S_L are added in a fixed order and the owning warp updates perm[S] in the
// output row (no two warps touch one S within a T_H step, and steps are
// separated by CTA barriers, so no atomics and a deterministic result).
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "apm_internal.cuh"

namespace apm {

constexpr int kPpmWarps = 8;
constexpr int kPpmMaxL = 7;
constexpr int kPpmPiece = 24;
constexpr int kPpmMaxPieces = 200;
constexpr int kPpmBpSlots = 2560;  // lane-interleaved B table: 32 x (longest lane <= 80)

// Schedules for l = 1..7, packed into one int array on the device.
struct PpmSched {
    int lvl;        // [l+2] start of each level in the entry list
    int ent;        // [3^l][2] entries: (dst | src << 16), (e | T << 8); src 0xffff at level 0
    int term;       // [maxlen][32] per lane term q: T_L | 0x80 if q starts a piece | S_L << 8; -1 past the end
    int lane;       // [33] first piece of each lane (pieces numbered lane by lane)
    int comb;       // [2^l + 1] CSR offsets of the pieces of each S_L
    int combidx;    // [npieces] piece ids per S_L
    int npieces;
    int maxlen;     // terms of the longest lane
};

__device__ __align__(16) int g_ppm_sched[60000];
static PpmSched h_sched[kPpmMaxL + 1];

static int popc(unsigned x) { return __builtin_popcount(x); }

static int pext_host(unsigned T, unsigned S) {
    int r = 0, k = 0;
    for (int b = 0; b < 32; ++b)
        if ((S >> b) & 1u) {
            if ((T >> b) & 1u) r |= 1 << k;
            ++k;
        }
    return r;
}

static void build_schedules(std::vector<int> &buf) {
    buf.clear();
    for (int l = 1; l <= kPpmMaxL; ++l) {
        PpmSched &s = h_sched[l];
        const int NL = 1 << l;
        // pieces of at most kPpmPiece consecutive submasks of one S_L, longest
        // first onto the least loaded lane
        struct P { int S, k0, cnt; };
        std::vector<P> pieces;
        for (int S = 0; S < NL; ++S) {
            const int terms = 1 << popc(S);
            for (int k0 = 0; k0 < terms; k0 += kPpmPiece)
                pieces.push_back({S, k0, terms - k0 < kPpmPiece ? terms - k0 : kPpmPiece});
        }
        std::vector<int> order(pieces.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = static_cast<int>(i);
        for (size_t i = 1; i < order.size(); ++i)  // stable insertion sort by decreasing count
            for (size_t j = i; j > 0 && pieces[order[j]].cnt > pieces[order[j - 1]].cnt; --j)
                std::swap(order[j], order[j - 1]);
        std::vector<std::vector<int>> per_lane(32);
        int load[32] = {};
        for (int id : order) {
            int best = 0;
            for (int ln = 1; ln < 32; ++ln)
                if (load[ln] < load[best]) best = ln;
            per_lane[best].push_back(id);
            load[best] += pieces[id].cnt;
        }
        int maxlen = 0;
        for (int ln = 0; ln < 32; ++ln) maxlen = load[ln] > maxlen ? load[ln] : maxlen;
        // B entry (S, rank k) lives at q*32 + lane, q = its position in the lane's term list
        std::vector<int> pos_of(3279 * 0 + (1 << (2 * l)), -1);  // indexed S * 2^l + k
        std::vector<int> term(static_cast<size_t>(maxlen) * 32, -1), lane_off(33), piece_id(pieces.size());
        int pid = 0;
        for (int ln = 0; ln < 32; ++ln) {
            lane_off[ln] = pid;
            int q = 0;
            for (int id : per_lane[ln]) {
                piece_id[id] = pid++;
                const P &pc = pieces[id];
                for (int k = pc.k0; k < pc.k0 + pc.cnt; ++k, ++q) {
                    // T_L = the k-th submask of S in increasing order
                    int T = 0, kk = k;
                    for (int m = pc.S; m; m &= m - 1) {
                        if (kk & 1) T |= m & (-m);
                        kk >>= 1;
                    }
                    term[static_cast<size_t>(q) * 32 + ln] = T | (k == pc.k0 ? 0x80 : 0) | (pc.S << 8);
                    pos_of[pc.S * NL + k] = q * 32 + ln;
                }
            }
        }
        lane_off[32] = pid;
        // B entries level by level over d = |S \ T|
        std::vector<int> lvl(l + 2, 0), ent;
        for (int d = 0; d <= l; ++d) {
            lvl[d] = static_cast<int>(ent.size() / 2);
            for (int S = 0; S < NL; ++S)
                for (int T = S;; T = (T - 1) & S) {
                    if (popc(S ^ T) == d) {
                        const int dst = pos_of[S * NL + pext_host(T, S)];
                        int src = 0xffff, e = 0;
                        if (d > 0) {
                            e = 31 - __builtin_clz(static_cast<unsigned>(S ^ T));
                            const int Sp = S ^ (1 << e);
                            src = pos_of[Sp * NL + pext_host(T, Sp)];
                        }
                        ent.push_back(dst | (src << 16));
                        ent.push_back(e | (T << 8));
                    }
                    if (T == 0) break;
                }
        }
        lvl[l + 1] = static_cast<int>(ent.size() / 2);
        std::vector<int> comb(NL + 1, 0), combidx;
        for (int S = 0; S < NL; ++S) {
            comb[S] = static_cast<int>(combidx.size());
            for (size_t id = 0; id < pieces.size(); ++id)
                if (pieces[id].S == S) combidx.push_back(piece_id[id]);
        }
        comb[NL] = static_cast<int>(combidx.size());
        s.lvl = static_cast<int>(buf.size());
        buf.insert(buf.end(), lvl.begin(), lvl.end());
        if (buf.size() & 1) buf.push_back(0);  // the entries are read as int2 (8-byte aligned)
        s.ent = static_cast<int>(buf.size());
        buf.insert(buf.end(), ent.begin(), ent.end());
        s.term = static_cast<int>(buf.size());
        buf.insert(buf.end(), term.begin(), term.end());
        s.lane = static_cast<int>(buf.size());
        buf.insert(buf.end(), lane_off.begin(), lane_off.end());
        s.comb = static_cast<int>(buf.size());
        buf.insert(buf.end(), comb.begin(), comb.end());
        s.combidx = static_cast<int>(buf.size());
        buf.insert(buf.end(), combidx.begin(), combidx.end());
        s.npieces = static_cast<int>(pieces.size());
        s.maxlen = maxlen;
    }
}

static bool schedules_fit() {
    for (int l = 1; l <= kPpmMaxL; ++l)
        if (h_sched[l].npieces > kPpmMaxPieces || h_sched[l].maxlen * 32 > kPpmBpSlots) return false;
    return true;
}

__device__ __forceinline__ int pdep_dev(int k, int S) {  // k-th submask of S (increasing order)
    int r = 0;
    for (int m = S; m; m &= m - 1) {
        if (k & 1) r |= m & (-m);
        k >>= 1;
    }
    return r;
}

struct PpmSmem {
    double U[16 * 128];   // [i][T_L]
    double RL[16 * 128];  // [i][T_L]
    double Bp[kPpmBpSlots];
    double PT[128];       // prod_{i in T_H} u_i(T_H u T_L)
    double alpha[kPpmWarps][128];
    double part[kPpmWarps][kPpmMaxPieces];
    double A[256];
    double RH[16];
};

__global__ void __launch_bounds__(kPpmWarps * 32) ppm_kernel(const double *__restrict__ Ag, int n, int64_t batch,
                                                             double *perms, const PpmSched sc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PpmSmem &sm = *reinterpret_cast<PpmSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, T = blockDim.x;
    const int l = n < kPpmMaxL ? n : kPpmMaxL, h = n - l, NL = 1 << l;
    const int N = 1 << n;
    const int *lvl = g_ppm_sched + sc.lvl;
    const int2 *ent = reinterpret_cast<const int2 *>(g_ppm_sched + sc.ent);
    const int *term = g_ppm_sched + sc.term;
    const int *lane_off = g_ppm_sched + sc.lane;
    const int *comb = g_ppm_sched + sc.comb;
    const int *combidx = g_ppm_sched + sc.combidx;
    const int maxlen = sc.maxlen;
    for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
        double *perm = perms + b * N;
        for (int t = tid; t < N; t += T) perm[t] = 0.0;
        for (int t = tid; t < n * n; t += T) sm.A[t] = __ldg(Ag + b * n * n + t);
        __syncthreads();
        // low row sums r_i(T_L), T_L over elements 0..l-1
        for (int t = tid; t < NL * n; t += T) {
            const int i = t / NL, TL = t - i * NL;
            double s = 0.0;
            for (int j = 0; j < l; ++j)
                if ((TL >> j) & 1) s += sm.A[i * n + j];
            sm.RL[i * 128 + TL] = s;
        }
        for (int TH = 0; TH < (1 << h); ++TH) {
            if (tid < n) {
                double s = 0.0;
                for (int j = 0; j < h; ++j)
                    if ((TH >> j) & 1) s += sm.A[tid * n + l + j];
                sm.RH[tid] = s;
            }
            __syncthreads();  // RH ready; previous step's U/Bp readers done
            for (int t = tid; t < NL * n; t += T) {
                const int i = t / NL, TL = t - i * NL;
                const double rr = sm.RH[i] + sm.RL[i * 128 + TL];
                const bool inT = i < l ? ((TL >> i) & 1) : ((TH >> (i - l)) & 1);
                sm.U[i * 128 + TL] = inT ? rr : -rr;
            }
            __syncthreads();
            // prefix product over the high column subset, shared by all its S_H
            for (int TL = tid; TL < NL; TL += T) {
                double v = 1.0;
                for (int i = 0; i < h; ++i)
                    if ((TH >> i) & 1) v *= sm.U[(l + i) * 128 + TL];
                sm.PT[TL] = v;
            }
            // B(T_L, S_L) = prod_{i in S_L} u_i, level by level over |S_L \ T_L|
            for (int d = 0; d <= l; ++d) {
                for (int e = lvl[d] + tid; e < lvl[d + 1]; e += T) {
                    const int2 w = ent[e];
                    const int dst = w.x & 0xffff, src = (w.x >> 16) & 0xffff;
                    const int el = w.y & 0xff, TL = w.y >> 8;
                    double v;
                    if (d == 0) {
                        v = 1.0;
                        for (int i = 0; i < l; ++i)
                            if ((TL >> i) & 1) v *= sm.U[i * 128 + TL];
                    } else {
                        v = sm.Bp[src] * sm.U[el * 128 + TL];
                    }
                    sm.Bp[dst] = v;
                }
                __syncthreads();
            }
            // one warp per S_H containing T_H
            const int freeH = ((1 << h) - 1) & ~TH;
            const int items = 1 << __popc(freeH);
            for (int it = warp; it < items; it += kPpmWarps) {
                const int R = pdep_dev(it, freeH);
                const int SH = TH | R;
                for (int TL = lane; TL < NL; TL += 32) {
                    double a = sm.PT[TL];
                    for (int m = R; m; m &= m - 1)
                        a *= sm.U[(l + __ffs(m) - 1) * 128 + TL];
                    sm.alpha[warp][TL] = a;
                }
                __syncwarp();
                // this lane's terms, lane-interleaved: conflict-free B reads
                int p = lane_off[lane];
                double acc = 0.0;
                for (int q = 0; q < maxlen; ++q) {
                    const int w = term[q * 32 + lane];
                    if (w < 0) break;
                    if ((w & 0x80) && q > 0) {
                        sm.part[warp][p++] = acc;
                        acc = 0.0;
                    }
                    acc = fma(sm.alpha[warp][w & 0x7f], sm.Bp[q * 32 + lane], acc);
                }
                if (lane_off[lane + 1] > lane_off[lane]) sm.part[warp][p] = acc;
                __syncwarp();
                for (int S = lane; S < NL; S += 32) {
                    double tot = 0.0;
                    for (int q = comb[S]; q < comb[S + 1]; ++q) tot += sm.part[warp][combidx[q]];
                    perm[(SH << l) | S] += tot;
                }
                __syncwarp();
            }
            __syncthreads();  // perm updates of this step visible before the next
        }
    }
}

static std::mutex g_sched_mu;
static int g_sched_dev_mask = 0;
static bool g_sched_built = false;
static std::vector<int> g_sched_buf;

static int ensure_ppm_schedules() {
    std::lock_guard<std::mutex> lk(g_sched_mu);
    if (!g_sched_built) {
        build_schedules(g_sched_buf);
        g_sched_built = true;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 32 && ((g_sched_dev_mask >> dev) & 1)) return 0;
    if (g_sched_buf.size() > 60000 || !schedules_fit()) return static_cast<int>(cudaErrorInvalidValue);
    e = cudaMemcpyToSymbol(g_ppm_sched, g_sched_buf.data(), g_sched_buf.size() * sizeof(int));
    if (e != cudaSuccess) return e;
    if (dev < 32) g_sched_dev_mask |= 1 << dev;
    return 0;
}

int launch_ppm(const double *A, int n, int64_t batch, double *perms, cudaStream_t s) {
    int err = ensure_ppm_schedules();
    if (err) return err;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = sizeof(PpmSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(ppm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ppm_kernel, kPpmWarps * 32, smem);
    if (e != cudaSuccess) return static_cast<int>(e);
    if (per_sm < 1) return static_cast<int>(cudaErrorInvalidConfiguration);
    int64_t g = static_cast<int64_t>(sms) * per_sm;
    if (batch < g) g = batch;
    const int l = n < kPpmMaxL ? n : kPpmMaxL;
    ppm_kernel<<<static_cast<int>(g), kPpmWarps * 32, smem, s>>>(A, n, batch, perms, h_sched[l]);
    return static_cast<int>(cudaGetLastError());
}

}  // namespace apm
