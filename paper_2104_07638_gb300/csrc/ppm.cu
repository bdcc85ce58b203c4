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
//
// One CTA per matrix, 8 warps, three CTAs per SM; the outer loop runs over the
// high column subsets T_H, two CTA barriers per step:
//  * tables (each warp alone, for the T_L it owns): U[i][T_L] = u_i(T_H u T_L)
//    (one add per entry from row sums kept per T_L and per T_H; the high row
//    sums of the next T_H take one add each, from a stack indexed by
//    popcount), the 8 starting products base_b(T_L) = prod_{i in T_H u R_b} u_i
//    over the subsets R_b of the lowest (up to) three high elements outside
//    T_H, and the 3^l entries B(T_L, S_L) level by level over |S_L \ T_L|, one
//    multiply each. The owners of T_L are chosen so that the warps get equal
//    shares.
//  * products (warp b takes the S_H = T_H u R_b u R' for all R' over the
//    remaining free high elements, depth first, so that each alpha vector is
//    its parent's times one u_i; the path stays in registers): for every S_L
//    the sum over its submasks T_L of alpha(T_L) B(T_L, S_L), one FMA per
//    (T, S) pair. The 3^l terms are laid out over 64 term streams, two per
//    lane, of at most ceil(3^l/64) terms each, by best fit (a set is cut
//    between streams only where it fits in none), with the B entries stored
//    stream-interleaved so that a lane reads its two as one 16-byte word, and
//    the terms inside each run ordered so that the alpha gathers of a
//    half-warp mostly hit distinct banks. A stream writes the sum of each run
//    of terms of one S_L to a result slot; the runs of a cut set are added
//    pairwise in rounds of one addition per lane (a fixed tree), and the warp
//    adds the 2^l sums into perm[S_H u S_L] in the output row by atomic
//    additions performed in L2 (fire and forget: no FP64 instruction and no
//    load latency on the SM). No two warps touch one S within a step and steps
//    are separated by CTA barriers, after which the earlier steps' additions
//    are visible, so every entry receives its terms in the same order on
//    every run: deterministic.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "apm_internal.cuh"

namespace apm {

constexpr int kPpmWarps = 8;
constexpr int kPpmMaxL = 7;
constexpr int kPpmMaxN = 16;
constexpr int kPpmVLanes = 64;      // term streams: two per lane
// row stride of the U and RL tables: one double more than the 128 columns, so
// that the 16 rows of one column, which a half-warp of the table phase writes
// or reads at once, fall on different banks
constexpr int kPpmLd = 129;
constexpr int kPpmBpSlots = 2240;   // stream-interleaved B table: 64 x 35 terms for l = 7
constexpr int kPpmResSlots = 236;   // 2^l sums + slots of the runs of cut sets (236 for l = 7)
constexpr int kPpmSchedInts = 60000;

// Schedules for l = 1..7, packed into one int array on the device.
struct PpmSched {
    int term;     // [maxlen][64] term words: T_L | 0x80 on the last term of a run | slot << 8; -1 past the end
    int first;    // [2^l] result slot that ends up holding the sum of S_L (its first run's)
    int rnd;      // [nrounds + 1] CSR offsets of the rounds of slot additions
    int pairs;    // slot additions (dst | src << 16): the runs of a cut set added pairwise, a tree
    int nrounds;
    int tl;       // [kPpmWarps + 1] CSR offsets of the T_L owned by each warp
    int tllist;   // [2^l] owned T_L, warp by warp
    int blvl;     // [kPpmWarps][l + 2] B entries of each warp, level by level
    int ent;      // [3^l][2] entries: (dst | src << 16), (e | T_L << 8); src 0xffff at level 0
    int len;      // [64] terms of each stream
    int maxlen;   // terms per stream (the first streams; the last one may have fewer)
    int nres;     // result slots used
};

__device__ __align__(16) int g_ppm_sched[kPpmSchedInts];
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

static int pdep_host(int k, int S) {  // k-th submask of S (increasing order)
    int r = 0;
    for (int m = S; m; m &= m - 1) {
        if (k & 1) r |= m & (-m);
        k >>= 1;
    }
    return r;
}

static void build_schedules(std::vector<int> &buf) {
    buf.clear();
    for (int l = 1; l <= kPpmMaxL; ++l) {
        PpmSched &s = h_sched[l];
        const int NL = 1 << l;
        int total = 1;
        for (int i = 0; i < l; ++i) total *= 3;
        const int cap = (total + kPpmVLanes - 1) / kPpmVLanes;
        // layout over 64 term streams (stream v = 2 lane + s) of at most cap
        // terms: sets S_L by decreasing size, each into the fullest stream it
        // still fits in whole (best fit); a set that fits nowhere fills the
        // emptiest stream and continues elsewhere (a cut set gets one result
        // slot per run). Streams are then ordered by decreasing length, so
        // that a lane's first stream is never the shorter one.
        std::vector<int> sets(NL);
        for (int S = 0; S < NL; ++S) sets[S] = S;
        for (int i = 1; i < NL; ++i)  // stable insertion sort by decreasing popcount
            for (int j = i; j > 0 && popc(sets[j]) > popc(sets[j - 1]); --j) std::swap(sets[j], sets[j - 1]);
        struct Run {
            int S, slot;
            std::vector<int> Ts;
        };
        std::vector<std::vector<Run>> runs(kPpmVLanes);
        std::vector<std::vector<int>> slots_of(NL);
        {
            std::vector<int> freec(kPpmVLanes, cap);
            int nres0 = NL;
            for (int S : sets) {
                const int terms = 1 << popc(S);
                int k = 0;
                std::vector<std::pair<int, int>> parts;  // (stream, count)
                while (k < terms) {
                    const int rem = terms - k;
                    int best = -1;
                    for (int v = 0; v < kPpmVLanes; ++v)
                        if (freec[v] >= rem && (best < 0 || freec[v] < freec[best])) best = v;
                    if (best < 0) {
                        best = 0;
                        for (int v = 1; v < kPpmVLanes; ++v)
                            if (freec[v] > freec[best]) best = v;
                    }
                    const int take = rem < freec[best] ? rem : freec[best];
                    parts.push_back({best, take});
                    freec[best] -= take;
                    k += take;
                }
                k = 0;
                for (const auto &pt : parts) {
                    Run r{S, parts.size() > 1 ? nres0++ : S, {}};
                    slots_of[S].push_back(r.slot);
                    for (int t = 0; t < pt.second; ++t, ++k) r.Ts.push_back(pdep_host(k, S));
                    runs[pt.first].push_back(r);
                }
            }
            s.nres = nres0;
            std::vector<int> len0(kPpmVLanes), order(kPpmVLanes);
            for (int v = 0; v < kPpmVLanes; ++v) {
                len0[v] = cap - freec[v];
                order[v] = v;
            }
            for (int a = 1; a < kPpmVLanes; ++a)  // stable sort by decreasing length
                for (int b2 = a; b2 > 0 && len0[order[b2]] > len0[order[b2 - 1]]; --b2)
                    std::swap(order[b2], order[b2 - 1]);
            std::vector<std::vector<Run>> sorted(kPpmVLanes);
            for (int v = 0; v < kPpmVLanes; ++v) sorted[v] = runs[order[v]];
            runs.swap(sorted);
        }
        // order of the terms inside each run (free: the run's sum is the same
        // up to rounding, and the order is fixed): position by position, the
        // streams read by one alpha gather of a half-warp (same s, 16 lanes)
        // pick, most constrained first, a T_L whose 8-byte bank of the alpha
        // vector is not yet taken by another T_L, so that the gathers are
        // (mostly) free of bank conflicts
        std::vector<int> term(static_cast<size_t>(cap) * kPpmVLanes, -1),
            pos_of(static_cast<size_t>(NL) * NL, -1);
        {
            std::vector<size_t> cur(kPpmVLanes, 0);
            for (int q = 0; q < cap; ++q)
                for (int grp = 0; grp < 4; ++grp) {
                    const int sgrp = grp & 1, hw = (grp >> 1) * 16;
                    std::vector<int> act;
                    for (int v = 2 * hw + sgrp; v < 2 * (hw + 16); v += 2) {
                        while (cur[v] < runs[v].size() && runs[v][cur[v]].Ts.empty()) ++cur[v];
                        if (cur[v] < runs[v].size()) act.push_back(v);
                    }
                    auto nbanks = [&](int v) {
                        int m = 0;
                        for (int T : runs[v][cur[v]].Ts) m |= 1 << (T & 15);
                        return popc(static_cast<unsigned>(m));
                    };
                    for (size_t i = 1; i < act.size(); ++i)  // stable sort by fewest banks
                        for (size_t j = i; j > 0 && nbanks(act[j]) < nbanks(act[j - 1]); --j)
                            std::swap(act[j], act[j - 1]);
                    int owner_T[16];
                    for (int b = 0; b < 16; ++b) owner_T[b] = -1;
                    for (int v : act) {
                        Run &r = runs[v][cur[v]];
                        size_t best = 0;
                        for (size_t i = 0; i < r.Ts.size(); ++i) {
                            const int b = r.Ts[i] & 15;
                            if (owner_T[b] < 0 || owner_T[b] == r.Ts[i]) {
                                best = i;
                                break;
                            }
                        }
                        const int T = r.Ts[best];
                        r.Ts.erase(r.Ts.begin() + static_cast<long>(best));
                        if (owner_T[T & 15] < 0) owner_T[T & 15] = T;
                        const bool last = r.Ts.empty();
                        term[static_cast<size_t>(q) * kPpmVLanes + v] = T | (last ? 0x80 : 0) | (r.slot << 8);
                        pos_of[static_cast<size_t>(r.S) * NL + pext_host(T, r.S)] = q * kPpmVLanes + v;
                    }
                }
        }
        // owners of the T_L for the tables: largest share (2^(l-|T_L|) B entries) first
        std::vector<int> tls(NL), owner(NL);
        for (int T = 0; T < NL; ++T) tls[T] = T;
        for (int i = 1; i < NL; ++i)
            for (int j = i; j > 0 && popc(tls[j]) < popc(tls[j - 1]); --j) std::swap(tls[j], tls[j - 1]);
        int wload[kPpmWarps] = {};
        for (int T : tls) {
            int best = 0;
            for (int w = 1; w < kPpmWarps; ++w)
                if (wload[w] < wload[best]) best = w;
            owner[T] = best;
            wload[best] += 1 << (l - popc(T));
        }
        std::vector<int> tl(kPpmWarps + 1), tllist;
        for (int w = 0; w < kPpmWarps; ++w) {
            tl[w] = static_cast<int>(tllist.size());
            for (int T = 0; T < NL; ++T)
                if (owner[T] == w) tllist.push_back(T);
        }
        tl[kPpmWarps] = static_cast<int>(tllist.size());
        // B entries, warp by warp, level by level over d = |S \ T|
        std::vector<int> blvl(static_cast<size_t>(kPpmWarps) * (l + 2)), ent;
        for (int w = 0; w < kPpmWarps; ++w) {
            for (int d = 0; d <= l; ++d) {
                blvl[static_cast<size_t>(w) * (l + 2) + d] = static_cast<int>(ent.size() / 2);
                for (int T = 0; T < NL; ++T) {
                    if (owner[T] != w) continue;
                    const int fr = (NL - 1) & ~T;
                    for (int R = fr;; R = (R - 1) & fr) {
                        if (popc(R) == d) {
                            const int S = T | R;
                            const int dst = pos_of[static_cast<size_t>(S) * NL + pext_host(T, S)];
                            int src = 0xffff, e = 0;
                            if (d > 0) {
                                e = 31 - __builtin_clz(static_cast<unsigned>(R));
                                const int Sp = S ^ (1 << e);
                                src = pos_of[static_cast<size_t>(Sp) * NL + pext_host(T, Sp)];
                            }
                            ent.push_back(dst | (src << 16));
                            ent.push_back(e | (T << 8));
                        }
                        if (R == 0) break;
                    }
                }
            }
            blvl[static_cast<size_t>(w) * (l + 2) + l + 1] = static_cast<int>(ent.size() / 2);
        }
        // the runs of every cut set are added pairwise (stride 1, 2, 4, ...) into the
        // slot of its first run; round r holds the additions of stride 2^r, at most
        // one per slot, so a warp does a round with one addition per lane
        std::vector<int> first(NL), rnd(1, 0), pairs;
        for (int S = 0; S < NL; ++S) first[S] = slots_of[S][0];
        for (int st = 1;; st *= 2) {
            bool any = false;
            for (int S = 0; S < NL; ++S) {
                const std::vector<int> &sl = slots_of[S];
                for (size_t i = 0; i + st < sl.size(); i += 2 * st) {
                    pairs.push_back(sl[i] | (sl[i + st] << 16));
                    any = true;
                }
            }
            if (!any) break;
            rnd.push_back(static_cast<int>(pairs.size()));
        }
        s.nrounds = static_cast<int>(rnd.size()) - 1;
        auto put = [&buf](const std::vector<int> &v) {
            const int at = static_cast<int>(buf.size());
            buf.insert(buf.end(), v.begin(), v.end());
            return at;
        };
        std::vector<int> len(kPpmVLanes, 0);
        for (int v = 0; v < kPpmVLanes; ++v)
            for (int q2 = 0; q2 < cap; ++q2)
                if (term[static_cast<size_t>(q2) * kPpmVLanes + v] >= 0) len[v] = q2 + 1;
        // the second stream of a lane runs as long as the first: pad it with
        // terms that end no run (T_L = 127, flag clear)
        for (int v = 1; v < kPpmVLanes; v += 2)
            for (int q2 = len[v]; q2 < len[v - 1]; ++q2) term[static_cast<size_t>(q2) * kPpmVLanes + v] = 0x7f;
        if (buf.size() & 1) buf.push_back(0);  // the term words are read in pairs (int2)
        s.term = put(term);
        s.len = put(len);
        s.first = put(first);
        s.rnd = put(rnd);
        s.pairs = put(pairs);
        s.tl = put(tl);
        s.tllist = put(tllist);
        s.blvl = put(blvl);
        if (buf.size() & 1) buf.push_back(0);  // the entries are read as int2 (8-byte aligned)
        s.ent = put(ent);
        s.maxlen = cap;
    }
}

// limits the kernel relies on: B table and result slots in shared memory, and
// at most 4 B entries per lane per level (the level-ahead prefetch)
static bool schedules_fit(const std::vector<int> &buf) {
    for (int l = 1; l <= kPpmMaxL; ++l) {
        const PpmSched &s = h_sched[l];
        if (s.maxlen * kPpmVLanes > kPpmBpSlots || s.nres > kPpmResSlots) return false;
        for (int w = 0; w < kPpmWarps; ++w)
            for (int d = 0; d <= l; ++d) {
                const int *lv = buf.data() + s.blvl + w * (l + 2);
                if (lv[d + 1] - lv[d] > 4 * 32) return false;
            }
        for (int r = 0; r < s.nrounds; ++r)  // one slot addition per lane and round
            if (buf[s.rnd + r + 1] - buf[s.rnd + r] > 32) return false;
    }
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

// The (T, S) terms of one lane: two independent streams (stream 2 lane + s),
// each a sequence of runs whose sums go to result slots. Both streams' FMAs
// are issued before anything reads their results (issue is in order and an
// FP64 result is hundreds of cycles away under load), so each warp keeps two
// FMAs in flight. A stream shorter than the lane's first one is padded with
// the word 0x7f (no run end): its tail terms only reach an accumulator that is
// never stored again. The next term words and B pair are fetched one step
// ahead; the pointers do not alias.
__device__ __forceinline__ void ppm_terms(const int2 *__restrict__ term2, const double *__restrict__ alpha,
                                          const double2 *__restrict__ Bp2, double *__restrict__ res, int len,
                                          int lane) {
    if (len == 0) return;
    double accA = 0.0, accB = 0.0;
    int2 wd = term2[lane];
    double2 bq = Bp2[lane];
    for (int q = 0; q < len; ++q) {
        const int qn = q + 1 < len ? q + 1 : q;
        const int2 wn = term2[qn * 32 + lane];
        const double2 bn = Bp2[qn * 32 + lane];
        const double nA = fma(alpha[wd.x & 0x7f], bq.x, accA);
        const double nB = fma(alpha[wd.y & 0x7f], bq.y, accB);
        if (wd.x & 0x80) res[wd.x >> 8] = nA;
        if (wd.y & 0x80) res[wd.y >> 8] = nB;
        accA = (wd.x & 0x80) ? 0.0 : nA;
        accB = (wd.y & 0x80) ? 0.0 : nB;
        wd = wn;
        bq = bn;
    }
}

// -x by the sign bit (no FP64 instruction)
__device__ __forceinline__ double neg_bits(double x) {
    return __longlong_as_double(__double_as_longlong(x) ^ static_cast<long long>(0x8000000000000000ull));
}

// prod over the set bits e of mask of U[(row0 + e) * kPpmLd + col] (1 for an empty
// mask): |mask| - 1 multiplies
__device__ __forceinline__ double set_prod(const double *U, int row0, int mask, int col) {
    if (mask == 0) return 1.0;
    double v = U[(row0 + __ffs(mask) - 1) * kPpmLd + col];
    for (int r = mask & (mask - 1); r; r &= r - 1) v *= U[(row0 + __ffs(r) - 1) * kPpmLd + col];
    return v;
}

struct PpmSmem {
    double U[kPpmMaxN * kPpmLd];   // [i][T_L], rows kPpmLd apart
    double RL[kPpmMaxN * kPpmLd];  // [i][T_L], rows kPpmLd apart
    double Bp[kPpmBpSlots];
    double alpha[kPpmWarps][128];  // base_w(T_L), then warp w's current alpha
    double res[kPpmWarps][kPpmResSlots];
    // high row sums RH_i(T_H) = sum_{j in T_H} A_i,l+j by popcount: row p holds
    // the latest T_H with p elements (a T_H's parent, T_H without its lowest
    // element, is the latest one with one element fewer)
    double rhs[kPpmMaxN - kPpmMaxL + 1][kPpmMaxN];
};
// three CTAs per SM: 228 KB of shared memory, 1 KB reserved per CTA
static_assert(3 * (sizeof(PpmSmem) + 1024) <= 228 * 1024, "three CTAs per SM");

__global__ void __launch_bounds__(kPpmWarps * 32, 3) ppm_kernel(const double *__restrict__ Ag, int n,
                                                                int64_t batch, double *perms, const PpmSched sc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PpmSmem &sm = *reinterpret_cast<PpmSmem *>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, T = blockDim.x;
    const int l = n < kPpmMaxL ? n : kPpmMaxL, h = n - l, NL = 1 << l;
    const int N = 1 << n;
    const int *term = g_ppm_sched + sc.term;
    const int *first = g_ppm_sched + sc.first;
    const int *rnd = g_ppm_sched + sc.rnd;
    const int *pairs = g_ppm_sched + sc.pairs;
    const int *tllist = g_ppm_sched + sc.tllist + g_ppm_sched[sc.tl + warp];
    const int ntl = g_ppm_sched[sc.tl + warp + 1] - g_ppm_sched[sc.tl + warp];
    const int *blvl = g_ppm_sched + sc.blvl + warp * (l + 2);
    const int2 *ent = reinterpret_cast<const int2 *>(g_ppm_sched + sc.ent);
    const int lenA = g_ppm_sched[sc.len + 2 * lane];  // the lane's first stream is the longer one
    const int2 *term2 = reinterpret_cast<const int2 *>(term);
    const double2 *Bp2 = reinterpret_cast<const double2 *>(sm.Bp);
    double *alpha = sm.alpha[warp];
    double *res = sm.res[warp];
    for (int64_t b = blockIdx.x; b < batch; b += gridDim.x) {
        double *perm = perms + b * N;
        const double *A = Ag + b * n * n;
        for (int t = tid; t < N; t += T) __stcg(perm + t, 0.0);
        if (tid < n) sm.rhs[0][tid] = 0.0;
        // low row sums r_i(T_L), T_L over elements 0..l-1
        for (int t = tid; t < NL * n; t += T) {
            const int i = t / NL, TL = t - i * NL;
            double s = 0.0;
            for (int j = 0; j < l; ++j)
                if ((TL >> j) & 1) s += __ldg(A + i * n + j);
            sm.RL[i * kPpmLd + TL] = s;
        }
        __syncthreads();
        for (int TH = 0; TH < (1 << h); ++TH) {
            const int freeH = ((1 << h) - 1) & ~TH;
            const int f = __popc(freeH), m = f < 3 ? f : 3;
            // the m lowest free high elements (their lattice gives the 2^m bases)
            int lowmask = 0;
            for (int k = 0, r = freeH; k < m; ++k, r &= r - 1) lowmask |= r & (-r);
            const int lm1 = lowmask & (lowmask - 1), lm2 = lm1 & (lm1 - 1);
            const int e0 = __ffs(lowmask) - 1, e1 = __ffs(lm1) - 1, e2 = __ffs(lm2) - 1;  // -1 where absent
            // ---- tables, each warp for its own T_L ----
            {
                // U[i][T_L]: lane = (T_L parity, row i)
                const int i = lane & 15;
                if (i < n) {
                    const double rhi = sm.rhs[__popc(TH)][i];
                    const bool high = i >= l;
                    const bool inTH = high && ((TH >> (i - l)) & 1);
                    for (int k = lane >> 4; k < ntl; k += 2) {
                        const int TL = tllist[k];
                        const bool inT = high ? inTH : ((TL >> i) & 1);
                        const double rr = rhi + sm.RL[i * kPpmLd + TL];
                        sm.U[i * kPpmLd + TL] = inT ? rr : neg_bits(rr);
                    }
                }
            }
            __syncwarp();
            for (int k = lane; k < ntl; k += 32) {
                const int TL = tllist[k];
                const double pt = set_prod(sm.U, l, TH, TL);
                double *base = &sm.alpha[0][TL];  // base[bb * 128] for the lattice element subsets bb
                base[0] = pt;
                if (m >= 1) {
                    const double u0 = sm.U[(l + e0) * kPpmLd + TL];
                    base[128] = pt * u0;
                    if (m >= 2) {
                        const double u1 = sm.U[(l + e1) * kPpmLd + TL];
                        const double b2 = pt * u1;
                        base[2 * 128] = b2;
                        base[3 * 128] = b2 * u0;
                        if (m >= 3) {
                            const double u2 = sm.U[(l + e2) * kPpmLd + TL];
                            const double b4 = pt * u2, b6 = b4 * u1;
                            base[4 * 128] = b4;
                            base[5 * 128] = b4 * u0;
                            base[6 * 128] = b6;
                            base[7 * 128] = b6 * u0;
                        }
                    }
                }
            }
            {
                // B entries level by level; this lane's entries of the next
                // level are fetched while the current one is computed
                int2 cur[4], nxt[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int e = blvl[0] + lane + 32 * k;
                    cur[k] = e < blvl[1] ? __ldcg(ent + e) : make_int2(0, 0);
                }
                for (int d = 0; d <= l; ++d) {
                    const int beg = blvl[d], end = blvl[d + 1], nend = d < l ? blvl[d + 2] : end;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int e = end + lane + 32 * k;
                        nxt[k] = e < nend ? __ldcg(ent + e) : make_int2(0, 0);
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (beg + lane + 32 * k < end) {
                            const int2 w = cur[k];
                            const int dst = w.x & 0xffff, src = (w.x >> 16) & 0xffff;
                            const int el = w.y & 0xff, TL = w.y >> 8;
                            sm.Bp[dst] = d == 0 ? set_prod(sm.U, 0, TL, TL) : sm.Bp[src] * sm.U[el * kPpmLd + TL];
                        }
                    }
                    __syncwarp();
#pragma unroll
                    for (int k = 0; k < 4; ++k) cur[k] = nxt[k];
                }
            }
            __syncthreads();
            // ---- products: warp w takes S_H = T_H u R_w u R' ----
            if (warp < (1 << m)) {
                const int Rw = pdep_dev(warp, lowmask);
                const int highmask = freeH & ~lowmask;
                const int fh = f - m;
                // path of alpha vectors over the inner (lowest four) remaining
                // free elements; a0 restarts for each outer block (n >= 15 only)
                // as the product over T_H, R_w and the block's outer elements
                double a0[4], a1[4], a2[4], a3[4], a4[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int TL = lane + 32 * k;
                    a0[k] = TL < NL ? alpha[TL] : 0.0;
                    a1[k] = a2[k] = a3[k] = a4[k] = 0.0;
                }
                for (int j = 0; j < (1 << fh); ++j) {
                    const int jj = j & 15, p = __popc(jj);
                    if (j > 0 && jj == 0) {
                        // new outer block: base times the outer elements of j
                        const int outer = pdep_dev(j, highmask) & ~pdep_dev(15, highmask);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int TL = lane + 32 * k;
                            if (TL < NL) a0[k] = set_prod(sm.U, l, TH | Rw | outer, TL);
                        }
                    }
                    if (p > 0) {
                        const int el = __ffs(pdep_dev(jj & (-jj), highmask)) - 1;
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int TL = lane + 32 * k;
                            if (TL < NL) {
                                const double u = sm.U[(l + el) * kPpmLd + TL];
                                switch (p) {
                                    case 1: a1[k] = a0[k] * u; break;
                                    case 2: a2[k] = a1[k] * u; break;
                                    case 3: a3[k] = a2[k] * u; break;
                                    default: a4[k] = a3[k] * u; break;
                                }
                            }
                        }
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int TL = lane + 32 * k;
                        if (TL < NL)
                            alpha[TL] = p == 0 ? a0[k] : p == 1 ? a1[k] : p == 2 ? a2[k] : p == 3 ? a3[k] : a4[k];
                    }
                    __syncwarp();
                    ppm_terms(term2, alpha, Bp2, res, lenA, lane);
                    __syncwarp();
                    const int SH = TH | Rw | pdep_dev(j, highmask);
                    for (int r = 0; r < sc.nrounds; ++r) {  // cut sets: their runs' sums, pairwise
                        const int i = rnd[r] + lane;
                        if (i < rnd[r + 1]) {
                            const int pw = pairs[i];
                            res[pw & 0xffff] += res[pw >> 16];
                        }
                        __syncwarp();
                    }
                    for (int S = lane; S < NL; S += 32) atomicAdd(perm + ((SH << l) | S), res[first[S]]);
                    __syncwarp();
                }
            }
            // row sums of the next high column subset (one add each, see rhs)
            if (warp == 0 && TH + 1 < (1 << h) && lane < n) {
                const int T2 = TH + 1, p2 = __popc(T2), e = __ffs(T2) - 1;
                sm.rhs[p2][lane] = sm.rhs[p2 - 1][lane] + __ldg(A + lane * n + l + e);
            }
            __syncthreads();  // tables and perm updates of this step done before the next
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
    if (g_sched_buf.size() > static_cast<size_t>(kPpmSchedInts) || !schedules_fit(g_sched_buf))
        return static_cast<int>(cudaErrorInvalidValue);
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
