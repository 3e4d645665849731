// Batched form of RandomSP: up to W = 64*K distinct sources ("lanes") share
// one persistent cooperative launch.  Per vertex the launch keeps K 64-bit
// words of visited bits and, for every level L, K words of frontier bits
// F_L(v) (bit j set iff v is at distance L from lane j's source).  A level is
// one pull pass over all vertices:
//     c = active & ~visited(v),  F_{L+1}(v) = OR_{u in in(v)} F_L(u) & c,
//     sigma_j(v) = sum over u in in(v) with bit j of F_L(u) & c of sigma_j(u)
// (the sigma recurrence of the oracle, summed in any order: the values are
// integers below 2^53, so every order gives the same exact result).  A lane
// retires once every target of its samples is discovered (its level is then
// complete) or its frontier is empty.  After the last level the same launch
// backtracks every sample of the batch (one warp per sample) exactly as the
// plain form does, reading the frontier history for the predecessor test.
//
// sigma is kept as exact integers: a dependent FP64 add costs ~64 cycles on
// GB300 while integer adds are cheap, and below 2^53 every conversion to FP64
// is exact, so the backtrack compares exactly the FP64 values a plain FP64
// implementation would.  Counts are stored in 32 bits (half the bytes per
// sector) until one reaches 2^32 (DEV_SIGMA_WIDE: the host reruns the phase
// with 64-bit storage), and in FP64 once one reaches 2^53
// (DEV_SIGMA_OVERFLOW), where counts beyond 2^53 round like FP64 sums.
//
// Layout in HBM (vertex-major so one warp reads a vertex's lanes coalesced):
//   visited  uint64 [n][K]
//   history  uint64 [Lcap+1][n][K]
//   sigma    uint64 or double [n][W]
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace percis {

namespace {

constexpr int kMsBlock = 256;
#ifndef PERCIS_BLOCK_DEG
#define PERCIS_BLOCK_DEG 256
#endif
constexpr int64_t kBlockDeg = PERCIS_BLOCK_DEG;  // in-degree above which a whole block counts one (vertex, word)

struct MsArgs {
    // batches of the persistent launch: a host plan, or W-lane batches over the
    // device-resident lane count *u_dev, or the single batch below
    const LaneBatch *plan;
    int32_t nplan;
    const long long *u_dev;
    // A launch covers the vertex range [vlo, vlo + n) of the loaded graph (the
    // whole graph, or the graphs of a multi-graph batch): rp / irp point at
    // entry vlo, column entries and sample vertices are global ids, and the
    // visited, frontier, count and queue arrays are indexed by id - vlo.
    int64_t n;
    int32_t vlo;
    const int64_t *irp;
    const int32_t *icol;
    uint64_t *vis;
    uint64_t *fh;
    void *sigma;
    MsCtl *ctl;
    int32_t Lcap;
    int32_t lane_base;
    int32_t nlanes;
    const int32_t *lane_src;
    const long long *lane_off;
    const int32_t *samp_t;
    const int32_t *samp_lane;
    const int32_t *sorted_samples;
    int32_t *found;
    int32_t *remaining;
    uint64_t seed;
    uint32_t tag;
    int32_t *kind;
    int32_t *ilen;
    long long *path_off;
    int32_t *arena;
    unsigned long long *arena_top;
    int64_t arena_cap;
    unsigned long long *cnt;
    int32_t full;
    uint64_t budget_ns;
    // push levels: out-adjacency, frontier queues, level stamps
    const int32_t *col;
    int32_t *fq0;
    int32_t *fq1;
    int32_t policy;                   // 0 = pull every level, 1 = push every level, 2 = by work estimate
    double push_alpha;                // policy 2: push while alpha * push work < pull work
    // instrumentation (INSTR variant only)
    const int64_t *rp;                // out-CSR offsets (out-degrees)
    unsigned long long *counters;     // 8 work counters (see percis_info.work)
    unsigned long long *levdeg;       // [W][Lcap+1] out-degree sums per lane and level
    // all-paths estimator: per-warp scratch (tau counts, claim stamps, two level lists)
    int32_t allpaths;
    int32_t ap_warps;
    int32_t ap_epoch;
    double *acc_ap;                   // per-vertex sum of sigma_sv tau_v / sigma_st
    unsigned long long *ap_tau;       // [ap_warps][n]
    int32_t *ap_stamp;                // [ap_warps][n]
    int32_t *ap_list;                 // [ap_warps][2n]
};

template <int K>
__device__ __forceinline__ void load_words(const uint64_t *p, uint64_t (&out)[K]) {
    if constexpr (K == 1) {
        out[0] = __ldcg(p);
    } else {
#pragma unroll
        for (int w = 0; w < K; w += 2) {
            const ulonglong2 q = __ldcg(reinterpret_cast<const ulonglong2 *>(p + w));
            out[w] = q.x;
            out[w + 1] = q.y;
        }
    }
}

template <class S>
__device__ __forceinline__ S warp_incl_scan(S v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const S o = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += o;
    }
    return v;
}

// Sum the counts of one 32-edge chunk's parents into the 64 lanes of word w:
// lane l's edge has parent u and frontier bits fw (already restricted to the
// lanes being counted).  Parents are taken in edge order, four per round so
// their loads overlap; acc0 / acc1 collect lanes l and l+32 of the word.
template <int SM, class ST, class S>
__device__ __forceinline__ void gather_chunk(const ST *sig, int W, int w, uint64_t fw, int32_t u, S &acc0, S &acc1,
                                             bool &ovf) {
    constexpr bool FPSIG = SM == 2;
    constexpr unsigned long long kLimit = SigmaMode<SM>::limit;
    const int lane = threadIdx.x & 31;
    unsigned nz = __ballot_sync(0xffffffffu, fw != 0ull);
    while (nz) {
        const int j0 = __ffs(nz) - 1;
        nz &= nz - 1;
        const bool h1 = nz != 0u;
        const int j1 = h1 ? __ffs(nz) - 1 : j0;
        if (h1) nz &= nz - 1;
        const bool h2 = nz != 0u;
        const int j2 = h2 ? __ffs(nz) - 1 : j0;
        if (h2) nz &= nz - 1;
        const bool h3 = nz != 0u;
        const int j3 = h3 ? __ffs(nz) - 1 : j0;
        if (h3) nz &= nz - 1;
        const uint64_t f0 = shfl64(fw, j0);
        const uint64_t f1 = h1 ? shfl64(fw, j1) : 0ull;
        const uint64_t f2 = h2 ? shfl64(fw, j2) : 0ull;
        const uint64_t f3 = h3 ? shfl64(fw, j3) : 0ull;
        const ST *r0 = sig + (int64_t)__shfl_sync(0xffffffffu, u, j0) * W + 64 * w;
        const ST *r1 = sig + (int64_t)__shfl_sync(0xffffffffu, u, j1) * W + 64 * w;
        const ST *r2 = sig + (int64_t)__shfl_sync(0xffffffffu, u, j2) * W + 64 * w;
        const ST *r3 = sig + (int64_t)__shfl_sync(0xffffffffu, u, j3) * W + 64 * w;
        S a0 = S(0), a1 = S(0), a2 = S(0), a3 = S(0), b0 = S(0), b1 = S(0), b2 = S(0), b3 = S(0);
        if ((f0 >> lane) & 1ull) a0 = __ldcg(r0 + lane);
        if ((f1 >> lane) & 1ull) a1 = __ldcg(r1 + lane);
        if ((f2 >> lane) & 1ull) a2 = __ldcg(r2 + lane);
        if ((f3 >> lane) & 1ull) a3 = __ldcg(r3 + lane);
        if ((f0 >> (lane + 32)) & 1ull) b0 = __ldcg(r0 + lane + 32);
        if ((f1 >> (lane + 32)) & 1ull) b1 = __ldcg(r1 + lane + 32);
        if ((f2 >> (lane + 32)) & 1ull) b2 = __ldcg(r2 + lane + 32);
        if ((f3 >> (lane + 32)) & 1ull) b3 = __ldcg(r3 + lane + 32);
        if (FPSIG) {
            // keep the in-adjacency order of the additions
            acc0 += a0; acc0 += a1; acc0 += a2; acc0 += a3;
            acc1 += b0; acc1 += b1; acc1 += b2; acc1 += b3;
        } else {
            acc0 += (a0 + a1) + (a2 + a3);
            acc1 += (b0 + b1) + (b2 + b3);
            // flag before four more addends could wrap 2^64
            ovf |= (acc0 >= kLimit) | (acc1 >= kLimit);
        }
    }
}

// One batch of lanes: levels, counts and the backtrack of its samples.  The
// batch covers lanes lane_base .. lane_base + nlanes - 1 and the vertex range
// [vlo, vlo + n); rp / irp point at entry vlo.  Returns false when the launch
// must stop (a bounded wait ran out, or the frontier history is too short).
template <int K, bool INSTR, int SM>
__device__ __forceinline__ bool ms_batch(const MsArgs &a, const int32_t lane_base, const int32_t nlanes,
                                         const int32_t vlo, const int64_t n, const int64_t *rp, const int64_t *irp,
                                         const int32_t ap_epoch) {
    constexpr int W = 64 * K;
    constexpr bool FPSIG = SM == 2;
    using S = typename SigmaMode<SM>::S;
    using ST = typename SigmaMode<SM>::ST;
    constexpr unsigned long long kLimit = SigmaMode<SM>::limit;
    ST *sig = static_cast<ST *>(a.sigma);
    bool ovf = false;
    unsigned long long n_sload = 0, n_swrite = 0, n_uv = 0, n_ue = 0;
    MsCtl *ctl = a.ctl;
    GridBarrier *bar = reinterpret_cast<GridBarrier *>(ctl);
    uint32_t *status = &ctl->status;
    const int lane = threadIdx.x & 31;
    const int warp_in_block = threadIdx.x >> 5;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t gwarp = tid >> 5;
    const int64_t nwarps = nthreads >> 5;
    const int64_t nk = n * K;
    const long long p0 = a.full ? 0 : a.lane_off[lane_base];
    const long long p1 = a.full ? 0 : a.lane_off[lane_base + nlanes];

    // ---- prologue: clear visited, frontiers 0 and 1, (push) sigma; reset lane state
    for (int64_t i = tid; i < nk; i += nthreads) {
        a.vis[i] = 0ull;
        a.fh[i] = 0ull;
        a.fh[nk + i] = 0ull;
    }
    for (long long p = p0 + tid; p < p1; p += nthreads) a.found[p] = -1;
    if (INSTR)
        for (int64_t i = tid; i < (int64_t)W * (a.Lcap + 1); i += nthreads) a.levdeg[i] = 0ull;
    if (blockIdx.x == 0) {
        for (int j = threadIdx.x; j < W; j += blockDim.x) a.remaining[j] = 0;
        if (threadIdx.x < K) {
            const int lo = threadIdx.x * 64;
            const int cntl = max(0, min(64, nlanes - lo));
            ctl->active[threadIdx.x] = cntl == 64 ? ~0ull : ((1ull << cntl) - 1ull);
            ctl->nonempty[0][threadIdx.x] = 0ull;
            ctl->nonempty[1][threadIdx.x] = 0ull;
        }
        if (threadIdx.x == 0) {
            ctl->ticket = 0;
            ctl->level = 0;
            ctl->qn[0] = nlanes;
            ctl->qn[1] = 0;
            ctl->qh[0] = 0;
            ctl->qh[1] = 0;
            ctl->push_next = a.policy != 0;
            ctl->t_start = globaltimer_ns();
        }
    }
    if (!grid_sync(bar, status, a.budget_ns)) return false;
    for (int64_t j = tid; j < nlanes; j += nthreads) {
        const int32_t v = a.lane_src[lane_base + j] - vlo;
        const uint64_t bit = 1ull << (j & 63);
        atomicOr((unsigned long long *)&a.vis[(int64_t)v * K + (j >> 6)], (unsigned long long)bit);
        atomicOr((unsigned long long *)&a.fh[(int64_t)v * K + (j >> 6)], (unsigned long long)bit);
        sig[(int64_t)v * W + j] = ST(1);
        a.fq0[j] = v;
        if (INSTR) a.levdeg[(int64_t)j * (a.Lcap + 1)] = (unsigned long long)(rp[v + 1] - rp[v]);
        if (!a.full) {
            const long long q0 = a.lane_off[lane_base + j], q1 = a.lane_off[lane_base + j + 1];
            a.remaining[j] = (int32_t)(q1 - q0);
        }
    }
    if (!grid_sync(bar, status, a.budget_ns)) return false;

    __shared__ unsigned long long s_nonempty[K];
    __shared__ unsigned long long s_act[K];
    __shared__ unsigned long long s_cont[K];
    __shared__ S s_red[kMsBlock / 32][64];  // per-warp partial sums of a block-wide gather
    int L = 0;
    for (;;) {
        bool any_act = false;
#pragma unroll
        for (int w = 0; w < K; ++w) any_act |= ld_relaxed_u64((const uint64_t *)&ctl->active[w]) != 0ull;
        if (!any_act) break;
        if (threadIdx.x < K) {
            s_nonempty[threadIdx.x] = 0ull;
            s_act[threadIdx.x] = ld_relaxed_u64((const uint64_t *)&ctl->active[threadIdx.x]);
        }
        __syncthreads();
        const uint64_t *fcur = a.fh + (int64_t)L * nk;
        uint64_t *fnext = a.fh + (int64_t)(L + 1) * nk;
        const int32_t *qcur = (L & 1) ? a.fq1 : a.fq0;
        int32_t *qnext = (L & 1) ? a.fq0 : a.fq1;
        int32_t *qn_next = &ctl->qn[(L + 1) & 1];
        int32_t *qh_next = &ctl->qh[(L + 1) & 1];
        const bool push = ld_relaxed_u32((const uint32_t *)&ctl->push_next) != 0u;

        // ---- phase A1: discover level L+1 (frontier bits only; counts follow in A2).
        // One warp per vertex with all K lane words at once: lane w < K holds
        // word w, edges are spread over the lanes and their K words are loaded
        // together.
        if (push) {
            const int64_t qn = (int64_t)ld_relaxed_u32((const uint32_t *)&ctl->qn[L & 1]);
            const int64_t qh = (int64_t)ld_relaxed_u32((const uint32_t *)&ctl->qh[L & 1]);
            // vertices of in-degree > 32 (the back of the queue) one block each,
            // its warps splitting the edges; then one warp per light vertex
            for (int64_t r = blockIdx.x; r < qh; r += gridDim.x) {
                const int32_t u = __ldcg(&qcur[n - 1 - r]);
                uint64_t fl = 0ull;
                if (lane < K) fl = __ldcg(&fcur[(int64_t)u * K + lane]) & s_act[lane];
                if (!__ballot_sync(0xffffffffu, fl != 0ull)) continue;
                uint64_t fu[K];
#pragma unroll
                for (int w = 0; w < K; ++w) fu[w] = shfl64(fl, w);
                const int64_t e0 = rp[u], e1 = rp[u + 1];
                for (int64_t e = e0 + warp_in_block * 32 + lane; e < e1; e += kMsBlock) {
                    const int32_t v = a.col[e] - vlo;
                    uint64_t vv[K];
                    load_words<K>(a.vis + (int64_t)v * K, vv);
#pragma unroll
                    for (int w = 0; w < K; ++w) {
                        const uint64_t m = fu[w] & ~vv[w];
                        if (m) atomicOr((unsigned long long *)&fnext[(int64_t)v * K + w], (unsigned long long)m);
                    }
                }
            }
            for (int64_t k = gwarp; k < qn; k += nwarps) {
                const int32_t u = __ldcg(&qcur[k]);
                uint64_t fl = 0ull;
                if (lane < K) fl = __ldcg(&fcur[(int64_t)u * K + lane]) & s_act[lane];
                if (!__ballot_sync(0xffffffffu, fl != 0ull)) continue;
                uint64_t fu[K];
#pragma unroll
                for (int w = 0; w < K; ++w) fu[w] = shfl64(fl, w);
                const int64_t e0 = rp[u], e1 = rp[u + 1];
                for (int64_t e = e0 + lane; e < e1; e += 32) {
                    const int32_t v = a.col[e] - vlo;
                    uint64_t vv[K];
                    load_words<K>(a.vis + (int64_t)v * K, vv);
#pragma unroll
                    for (int w = 0; w < K; ++w) {
                        const uint64_t m = fu[w] & ~vv[w];
                        // fire-and-forget: the new frontier is collected after the barrier
                        if (m) atomicOr((unsigned long long *)&fnext[(int64_t)v * K + w], (unsigned long long)m);
                    }
                }
            }
        } else {
            // every vertex with unvisited active lanes; the scan stops once each
            // such lane has found a parent
            for (int64_t v = gwarp; v < n; v += nwarps) {
                uint64_t cl = 0ull;
                if (lane < K) cl = s_act[lane] & ~__ldcg(&a.vis[v * K + lane]);
                if (!__ballot_sync(0xffffffffu, cl != 0ull)) continue;
                uint64_t nbl = 0ull;
                const int64_t e0 = irp[v], e1 = irp[v + 1];
                for (int64_t base = e0; base < e1; base += 32) {
                    const int64_t e = base + lane;
                    uint64_t f[K];
                    if (e < e1) {
                        load_words<K>(fcur + (int64_t)(a.icol[e] - vlo) * K, f);
                    } else {
#pragma unroll
                        for (int w = 0; w < K; ++w) f[w] = 0ull;
                    }
#pragma unroll
                    for (int w = 0; w < K; ++w) {
                        const uint64_t r = warp_or64(f[w]);
                        if (lane == w) nbl |= r & cl;
                    }
                    if (__all_sync(0xffffffffu, nbl == cl)) break;
                }
                if (lane < K && nbl) fnext[v * K + lane] = nbl;
                if (__ballot_sync(0xffffffffu, nbl != 0ull) && lane == 0) {
                    if (e1 - e0 > 32) qnext[n - 1 - atomicAdd(qh_next, 1)] = (int32_t)v;
                    else qnext[atomicAdd(qn_next, 1)] = (int32_t)v;
                }
            }
        }
        if (!grid_sync(bar, status, a.budget_ns)) return false;
        if (tid == 0 && L < 32) ctl->lvl_rec[L][4] = globaltimer_ns() - ctl->t_start;

        if (push) {
            // collect the vertices that gained frontier bits into the next queue
            // (warp-aggregated appends; each vertex is looked at by one thread)
            for (int64_t vb = gwarp * 32; vb < n; vb += nwarps * 32) {
                const int64_t v = vb + lane;
                bool any = false;
                if (v < n) {
                    if (K == 1) {
                        any = __ldcg(&fnext[v]) != 0ull;
                    } else {
                        uint64_t f[K];
                        load_words<K>(fnext + v * K, f);
#pragma unroll
                        for (int w = 0; w < K; ++w) any |= f[w] != 0ull;
                    }
                }
                const bool heavy = any && irp[v + 1] - irp[v] > 32;
                const unsigned am = __ballot_sync(0xffffffffu, any && !heavy);
                const unsigned hm = __ballot_sync(0xffffffffu, heavy);
                if (am) {
                    const int leader = __ffs(am) - 1;
                    int pos = 0;
                    if (lane == leader) pos = atomicAdd(qn_next, __popc(am));
                    pos = __shfl_sync(0xffffffffu, pos, leader);
                    if (any && !heavy) qnext[pos + __popc(am & ((1u << lane) - 1u))] = (int32_t)v;
                }
                if (hm) {
                    const int leader = __ffs(hm) - 1;
                    int pos = 0;
                    if (lane == leader) pos = atomicAdd(qh_next, __popc(hm));
                    pos = __shfl_sync(0xffffffffu, pos, leader);
                    if (heavy) qnext[n - 1 - (pos + __popc(hm & ((1u << lane) - 1u)))] = (int32_t)v;
                }
            }
        }
        // mark settled targets
        if (!a.full) {
            for (long long p = p0 + tid; p < p1; p += nthreads) {
                if (a.found[p] >= 0) continue;
                const int32_t j = a.samp_lane[p] - lane_base;
                const int32_t t = a.samp_t[p] - vlo;
                const int64_t q = (int64_t)t * K + (j >> 6);
                if (((__ldcg(&a.vis[q]) | __ldcg(&fnext[q])) >> (j & 63)) & 1ull) {
                    a.found[p] = L + 1;
                    atomicSub(&a.remaining[j], 1);
                }
            }
        }
        if (!grid_sync(bar, status, a.budget_ns)) return false;
        if (tid == 0 && L < 32) ctl->lvl_rec[L][5] = globaltimer_ns() - ctl->t_start;

        // ---- phase A2: counts of level L+1.  A lane whose last targets were
        // settled at this level retires after it, and of its level-(L+1)
        // vertices only those targets are ever read (by the backtrack), so its
        // counts are formed there alone.
        if (a.full) {
            if (threadIdx.x < K) s_cont[threadIdx.x] = s_act[threadIdx.x];
        } else {
            if (threadIdx.x < K) s_cont[threadIdx.x] = 0ull;
            __syncthreads();
            for (int j = threadIdx.x; j < W; j += blockDim.x) {
                const bool c = ((s_act[j >> 6] >> (j & 63)) & 1ull) && __ldcg(&a.remaining[j]) > 0;
                const unsigned bm = __ballot_sync(0xffffffffu, c);
                if (lane == 0 && bm) atomicOr(&s_cont[j >> 6], (unsigned long long)bm << (j & 32));
            }
        }
        __syncthreads();
        const int64_t qn1 = (int64_t)ld_relaxed_u32((const uint32_t *)qn_next);
        const int64_t qh1 = (int64_t)ld_relaxed_u32((const uint32_t *)qh_next);
        if (!FPSIG) {
            // in-degree > kBlockDeg: one block per (vertex, word), its warps
            // splitting the edges; the partial sums meet in shared memory
            // (integer sums, so the order does not matter)
            for (int64_t hi = blockIdx.x; hi < qh1 * K; hi += gridDim.x) {
                const int64_t h = hi / K;
                const int w = (int)(hi - h * K);
                const int32_t v = __ldcg(&qnext[n - 1 - h]);
                const int64_t e0 = irp[v], e1 = irp[v + 1];
                if (e1 - e0 <= kBlockDeg) continue;  // a warp item below; the same for the whole block
                const uint64_t nbw = __ldcg(&fnext[(int64_t)v * K + w]) & s_cont[w];
                if (nbw == 0ull) continue;
                S acc0 = S(0), acc1 = S(0);
                for (int64_t base = e0 + warp_in_block * 32; base < e1; base += kMsBlock) {
                    const int64_t e = base + lane;
                    int32_t u = 0;
                    uint64_t fw = 0ull;
                    if (e < e1) {
                        u = a.icol[e] - vlo;
                        fw = __ldcg(&fcur[(int64_t)u * K + w]) & nbw;
                    }
                    if (INSTR) n_sload += (unsigned long long)__popcll(fw);
                    gather_chunk<SM, ST, S>(sig, W, w, fw, u, acc0, acc1, ovf);
                }
                s_red[warp_in_block][lane] = acc0;
                s_red[warp_in_block][lane + 32] = acc1;
                __syncthreads();
                if (warp_in_block == 0) {
                    S t0 = S(0), t1 = S(0);
#pragma unroll
                    for (int q = 0; q < kMsBlock / 32; ++q) {
                        t0 += s_red[q][lane];
                        t1 += s_red[q][lane + 32];
                    }
                    ovf |= (t0 >= (S)kLimit) | (t1 >= (S)kLimit);
                    ST *drow = sig + (int64_t)v * W + 64 * w;
                    if ((nbw >> lane) & 1ull) drow[lane] = (ST)t0;
                    if ((nbw >> (lane + 32)) & 1ull) drow[lane + 32] = (ST)t1;
                    if (INSTR) n_swrite += lane == 0 ? (unsigned long long)__popcll(nbw) : 0ull;
                }
                __syncthreads();
            }
        }
        for (int64_t it = gwarp; it < qn1 + qh1 * K; it += nwarps) {
            if (it < qn1) {
                // in-degree <= 32: one warp per new vertex, its parents and all
                // their words loaded once; lane w < K holds the word's lanes to count
                const int32_t v = __ldcg(&qnext[it]);
                uint64_t nbl = 0ull;
                if (lane < K) nbl = __ldcg(&fnext[(int64_t)v * K + lane]) & s_cont[lane];
                const unsigned wm = __ballot_sync(0xffffffffu, nbl != 0ull);
                if (!wm) continue;
                const int64_t e0 = irp[v], e1 = irp[v + 1];
                ST *drow = sig + (int64_t)v * W;
                const int64_t e = e0 + lane;
                int32_t u = 0;
                uint64_t f[K];
                if (e < e1) {
                    u = a.icol[e] - vlo;
                    load_words<K>(fcur + (int64_t)u * K, f);
                } else {
#pragma unroll
                    for (int w = 0; w < K; ++w) f[w] = 0ull;
                }
#pragma unroll
                for (int w = 0; w < K; ++w) {
                    if (!((wm >> w) & 1u)) continue;
                    const uint64_t nbw = shfl64(nbl, w);
                    const uint64_t fw = f[w] & nbw;
                    if (INSTR) n_sload += (unsigned long long)__popcll(fw);
                    S acc0 = S(0), acc1 = S(0);
                    gather_chunk<SM, ST, S>(sig, W, w, fw, u, acc0, acc1, ovf);
                    if (FPSIG) ovf |= (acc0 >= (S)kLimit) | (acc1 >= (S)kLimit);
                    if ((nbw >> lane) & 1ull) drow[64 * w + lane] = (ST)acc0;
                    if ((nbw >> (lane + 32)) & 1ull) drow[64 * w + lane + 32] = (ST)acc1;
                    if (INSTR) n_swrite += lane == 0 ? (unsigned long long)__popcll(nbw) : 0ull;
                }
            } else {
                // in-degree in (32, kBlockDeg] (any, for FP64 counts, whose
                // additions keep the in-adjacency order): one warp per
                // (vertex, word) over 32-edge chunks
                const int64_t h = (it - qn1) / K;
                const int w = (int)(it - qn1 - h * K);
                const int32_t v = __ldcg(&qnext[n - 1 - h]);
                const int64_t e0 = irp[v], e1 = irp[v + 1];
                if (!FPSIG && e1 - e0 > kBlockDeg) continue;
                const uint64_t nbw = __ldcg(&fnext[(int64_t)v * K + w]) & s_cont[w];
                if (nbw == 0ull) continue;
                S acc0 = S(0), acc1 = S(0);
                for (int64_t base = e0; base < e1; base += 32) {
                    const int64_t e = base + lane;
                    int32_t u = 0;
                    uint64_t fw = 0ull;
                    if (e < e1) {
                        u = a.icol[e] - vlo;
                        fw = __ldcg(&fcur[(int64_t)u * K + w]) & nbw;
                    }
                    if (INSTR) n_sload += (unsigned long long)__popcll(fw);
                    gather_chunk<SM, ST, S>(sig, W, w, fw, u, acc0, acc1, ovf);
                }
                if (FPSIG) ovf |= (acc0 >= (S)kLimit) | (acc1 >= (S)kLimit);
                ST *drow = sig + (int64_t)v * W + 64 * w;
                if ((nbw >> lane) & 1ull) drow[lane] = (ST)acc0;
                if ((nbw >> (lane + 32)) & 1ull) drow[lane + 32] = (ST)acc1;
                if (INSTR) n_swrite += lane == 0 ? (unsigned long long)__popcll(nbw) : 0ull;
            }
        }
        if (!a.full) {
            // targets of the retiring lanes: one warp per sample settled at L+1
            for (long long p = p0 + gwarp; p < p1; p += nwarps) {
                if (__ldcg(&a.found[p]) != L + 1) continue;
                const int32_t j = a.samp_lane[p] - lane_base;
                const int w = j >> 6;
                const uint64_t bj = 1ull << (j & 63);
                if (s_cont[w] & bj) continue;
                const int32_t t = a.samp_t[p] - vlo;
                const int64_t e0 = irp[t], e1 = irp[t + 1];
                S acc = S(0);
                if (FPSIG) {
                    // in-adjacency order
                    if (lane == 0)
                        for (int64_t e = e0; e < e1; ++e) {
                            const int32_t u = a.icol[e] - vlo;
                            if (__ldcg(&fcur[(int64_t)u * K + w]) & bj) acc += (S)__ldcg(&sig[(int64_t)u * W + j]);
                        }
                } else {
                    for (int64_t e = e0 + lane; e < e1; e += 32) {
                        const int32_t u = a.icol[e] - vlo;
                        if (__ldcg(&fcur[(int64_t)u * K + w]) & bj) {
                            acc += (S)__ldcg(&sig[(int64_t)u * W + j]);
                            if (INSTR) ++n_sload;
                        }
                    }
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
                }
                if (lane == 0) {
                    ovf |= acc >= (S)kLimit;
                    sig[(int64_t)t * W + j] = (ST)acc;
                    if (INSTR) ++n_swrite;
                }
            }
        }

        // ---- phase B(1): settle the new frontier: visited bits, nonempty lanes,
        // next frontier's out-edges (no reader of these runs in this interval)
        {
            unsigned long long fe = 0ull;
            for (int64_t it = tid; it < (qn1 + qh1) * K; it += nthreads) {
                const int64_t k = it / K;
                const int w = (int)(it - k * K);
                const int32_t v = __ldcg(&qnext[k < qn1 ? k : n - 1 - (k - qn1)]);
                const uint64_t nb = __ldcg(&fnext[(int64_t)v * K + w]);
                if (!nb) continue;
                a.vis[(int64_t)v * K + w] = __ldcg(&a.vis[(int64_t)v * K + w]) | nb;
                atomicOr(&s_nonempty[w], (unsigned long long)nb);
                fe += (unsigned long long)(rp[v + 1] - rp[v]);
                if (INSTR && w == 0) {
                    n_uv += 1;
                    n_ue += (unsigned long long)(rp[v + 1] - rp[v]);
                }
                if (INSTR) {
                    const unsigned long long dg = (unsigned long long)(rp[v + 1] - rp[v]);
                    uint64_t m2 = nb;
                    while (m2) {
                        const int b = __ffsll((long long)m2) - 1;
                        m2 &= m2 - 1;
                        atomicAdd(&a.levdeg[(int64_t)(64 * w + b) * (a.Lcap + 1) + L + 1], dg);
                    }
                }
            }
            // frontier out-edges for the direction choice
            for (int off = 16; off > 0; off >>= 1) fe += __shfl_xor_sync(0xffffffffu, fe, off);
            if (lane == 0 && fe) atomicAdd(&ctl->fedges[(L + 1) & 1], fe);
            if (L + 2 <= a.Lcap) {
                uint64_t *f2 = a.fh + (int64_t)(L + 2) * nk;
                for (int64_t i = tid; i < nk; i += nthreads) f2[i] = 0ull;
            }
            if (a.policy == 2) {
                // pull work of the next level: in-edges of every (vertex, word) that
                // still has an unvisited active lane
                unsigned long long ue = 0ull;
                for (int64_t it = tid; it < nk; it += nthreads) {
                    const int64_t v = it / K;
                    const int w = (int)(it - v * K);
                    const uint64_t vw = __ldcg(&a.vis[it]) | __ldcg(&fnext[it]);
                    if (s_act[w] & ~vw) ue += (unsigned long long)(irp[v + 1] - irp[v]);
                }
                for (int off = 16; off > 0; off >>= 1) ue += __shfl_xor_sync(0xffffffffu, ue, off);
                if (lane == 0 && ue) atomicAdd(&ctl->uedges[(L + 1) & 1], ue);
            }
        }
        if (__any_sync(0xffffffffu, ovf) && lane == 0) atomicOr(status, SigmaMode<SM>::flag);
        ovf = false;
        __syncthreads();
        if (threadIdx.x < K && s_nonempty[threadIdx.x])
            atomicOr(&ctl->nonempty[L & 1][threadIdx.x], s_nonempty[threadIdx.x]);
        __syncthreads();
        __shared__ int s_last;
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            if (threadIdx.x < K) {
                const int w = threadIdx.x;
                uint64_t nact = s_act[w] & ld_relaxed_u64((const uint64_t *)&ctl->nonempty[L & 1][w]);
                if (!a.full) {
                    uint64_t m = nact;
                    while (m) {
                        const int b = __ffsll((long long)m) - 1;
                        m &= m - 1;
                        if (atomicAdd(&a.remaining[w * 64 + b], 0) <= 0) nact &= ~(1ull << b);
                    }
                }
                ctl->active[w] = nact;
                ctl->nonempty[L & 1][w] = 0ull;
            }
            if (threadIdx.x == 0) {
                ctl->ticket = 0;
                ctl->level = L + 1;
                if (L < 32) {
                    ctl->lvl_rec[L][0] = globaltimer_ns() - ctl->t_start;
                    ctl->lvl_rec[L][1] = (push ? 1ull : 0ull) | (ctl->uedges[L & 1] << 1);
                    ctl->lvl_rec[L][2] = (unsigned long long)(ctl->qn[L & 1] + ctl->qh[L & 1]);
                    ctl->lvl_rec[L][3] = ctl->fedges[L & 1];
                }
                ctl->qn[L & 1] = 0;  // the queue just consumed is refilled at level L+2
                ctl->qh[L & 1] = 0;
                const unsigned long long fe = ctl->fedges[(L + 1) & 1];
                const unsigned long long ue = ctl->uedges[(L + 1) & 1];
                ctl->fedges[L & 1] = 0ull;
                ctl->uedges[L & 1] = 0ull;
                ctl->push_next = a.policy == 1 || (a.policy == 2 && a.push_alpha * (double)fe < (double)ue);
            }
        }
        if (!grid_sync(bar, status, a.budget_ns)) return false;
        ++L;
        bool more = false;
#pragma unroll
        for (int w = 0; w < K; ++w) more |= ld_relaxed_u64((const uint64_t *)&ctl->active[w]) != 0ull;
        if (!more) break;
        if (L + 1 > a.Lcap) {
            if (tid == 0) atomicOr(status, DEV_NEED_LEVELS);
            return false;
        }
    }
    if (INSTR) {
        for (int off = 16; off > 0; off >>= 1) {
            n_sload += __shfl_xor_sync(0xffffffffu, n_sload, off);
            n_swrite += __shfl_xor_sync(0xffffffffu, n_swrite, off);
            n_uv += __shfl_xor_sync(0xffffffffu, n_uv, off);
            n_ue += __shfl_xor_sync(0xffffffffu, n_ue, off);
        }
        if (lane == 0) {
            atomicAdd(&a.counters[0], n_sload);
            atomicAdd(&a.counters[1], n_swrite);
            atomicAdd(&a.counters[2], n_uv);
            atomicAdd(&a.counters[3], n_ue);
        }
        if (tid == 0) atomicAdd(&a.counters[5], (unsigned long long)L);
    }
    if (a.full) return true;

    if (a.allpaths) {
        // ---- all-paths form (warp per sample): reverse sweep from t over the
        // shortest-path DAG of lane j; tau_v = number of shortest v-t paths
        // (exact integers), and every internal v receives
        // f(v) = sigma_sv tau_v / sigma_st.  Scratch is per warp; entries are
        // valid only where the claim stamp equals this sample's epoch.
        if (gwarp >= a.ap_warps) return true;
        S *tau = reinterpret_cast<S *>(a.ap_tau) + gwarp * n;  // integers, or FP64 beyond 2^53
        int32_t *stamp = a.ap_stamp + gwarp * n;
        int32_t *la = a.ap_list + gwarp * 2 * n;
        int32_t *lb = la + n;
        const unsigned lt = (1u << lane) - 1u;
        for (long long p = p0 + gwarp; p < p1; p += a.ap_warps) {
            const int32_t i = a.sorted_samples[p];
            const int32_t j = a.samp_lane[p] - lane_base;
            const int32_t t = a.samp_t[p] - vlo;
            const int32_t d = __ldcg(&a.found[p]);
            if (lane == 0) {
                if (d < 0) a.kind[i] = 2;
                a.ilen[i] = d < 0 ? 0 : d - 1;
                a.path_off[i] = 0;
            }
            if (d < 2) continue;
            const int32_t ep = ap_epoch + (int32_t)p + 1;  // sample positions are unique in a phase
            const int wj = j >> 6;
            const uint64_t bj = 1ull << (j & 63);
            const double sst = (double)(S)__ldcg(&sig[(int64_t)t * W + j]);
            if (lane == 0) {
                la[0] = t;
                tau[t] = S(1);
                stamp[t] = ep;
            }
            int na = 1;
            __syncwarp();
            for (int L = d - 1; L >= 1; --L) {
                const uint64_t *fL = a.fh + (int64_t)L * nk;
                int nb = 0;
                // claim the predecessors at level L (first claimer zeroes tau)
                for (int q = 0; q < na; ++q) {
                    const int32_t w = __ldcg(&la[q]);
                    const int64_t e0 = irp[w], e1 = irp[w + 1];
                    for (int64_t base = e0; base < e1; base += 32) {
                        const int64_t ee = base + lane;
                        bool mine = false;
                        int32_t pv = 0;
                        if (ee < e1) {
                            pv = a.icol[ee] - vlo;
                            if (__ldcg(&fL[(int64_t)pv * K + wj]) & bj) {
                                mine = atomicExch(&stamp[pv], ep) != ep;
                                if (mine) tau[pv] = S(0);
                            }
                        }
                        const unsigned m = __ballot_sync(0xffffffffu, mine);
                        if (mine) lb[nb + __popc(m & lt)] = pv;
                        nb += __popc(m);
                    }
                }
                __syncwarp();
                // tau_p += tau_w over the DAG edges into level L+1
                for (int q = 0; q < na; ++q) {
                    const int32_t w = __ldcg(&la[q]);
                    const S tw = __ldcg(&tau[w]);
                    const int64_t e0 = irp[w], e1 = irp[w + 1];
                    for (int64_t ee = e0 + lane; ee < e1; ee += 32) {
                        const int32_t pv = a.icol[ee] - vlo;
                        if (__ldcg(&fL[(int64_t)pv * K + wj]) & bj) atomicAdd(&tau[pv], tw);
                    }
                }
                __syncwarp();
                for (int q = lane; q < nb; q += 32) {
                    const int32_t v = __ldcg(&lb[q]);
                    const double f = (double)(S)__ldcg(&sig[(int64_t)v * W + j]) * (double)__ldcg(&tau[v]) / sst;
                    atomicAdd(&a.acc_ap[v + vlo], f);
                }
                __syncwarp();
                int32_t *tmp = la;
                la = lb;
                lb = tmp;
                na = nb;
            }
        }
        return true;
    }

    // ---- backtrack every sample of the batch (warp per sample)
    for (long long p = p0 + gwarp; p < p1; p += nwarps) {
        const int32_t i = a.sorted_samples[p];
        const int32_t j = a.samp_lane[p] - lane_base;
        const int32_t t = a.samp_t[p] - vlo;
        const int32_t s = a.lane_src[lane_base + j] - vlo;
        const int32_t d = __ldcg(&a.found[p]);
        if (INSTR) {
            // edges a top-down truncated BFS from s scans before settling t
            const int32_t lmax = d < 0 ? a.Lcap : d - 1;
            unsigned long long e = 0;
            for (int32_t Lq = lane; Lq <= lmax; Lq += 32) e += a.levdeg[(int64_t)j * (a.Lcap + 1) + Lq];
            for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
            if (lane == 0) {
                atomicAdd(&a.counters[4], e);
                atomicAdd(&a.counters[6], 1ull);
            }
        }
        if (d < 0) {
            if (lane == 0) {
                a.kind[i] = 2;
                a.ilen[i] = 0;
                a.path_off[i] = 0;
            }
            continue;
        }
        const int32_t len = d - 1;
        unsigned long long off = 0;
        if (lane == 0) {
            off = atomicAdd(a.arena_top, (unsigned long long)len);
            a.ilen[i] = len;
            a.path_off[i] = (long long)off;
            if ((int64_t)(off + len) > a.arena_cap) atomicOr(status, DEV_ARENA_OVERFLOW);
        }
        off = __shfl_sync(0xffffffffu, off, 0);
        const bool store = (int64_t)(off + len) <= a.arena_cap;
        const int wj = j >> 6;
        const uint64_t bj = 1ull << (j & 63);
        int32_t w = t;
        int32_t lw = d;
        uint32_t step = 0;
        int32_t k = 0;
        while (w != s) {
            const double target = __dmul_rn(uniform_at(a.seed, (uint64_t)i, a.tag, step),
                                            (double)(S)__ldcg(&sig[(int64_t)w * W + j]));
            const uint64_t *fprev = a.fh + (int64_t)(lw - 1) * nk;
            const int64_t e0 = irp[w], e1 = irp[w + 1];
            S carry = S(0);
            int32_t pick = -1;
            for (int64_t base = e0; base < e1 && pick < 0; base += 32) {
                const int64_t e = base + lane;
                int32_t pv = -1;
                S val = S(0);
                if (e < e1) {
                    pv = a.icol[e] - vlo;
                    if (__ldcg(&fprev[(int64_t)pv * K + wj]) & bj) val = (S)__ldcg(&sig[(int64_t)pv * W + j]);
                }
                // running sums are exact (integers; FP64 sums of integers below 2^53)
                const S cum = carry + warp_incl_scan<S>(val);
                const unsigned hit = __ballot_sync(0xffffffffu, val > S(0) && (double)cum >= target);
                if (hit) pick = __shfl_sync(0xffffffffu, pv, __ffs(hit) - 1);
                carry = __shfl_sync(0xffffffffu, cum, 31);
            }
            if (pick < 0) {
                if (lane == 0) atomicOr(status, DEV_BAD_PATH);
                break;
            }
            if (pick != s) {
                if (lane == 0) {
                    if (store) a.arena[off + k] = pick + vlo;
                    atomicAdd(&a.cnt[pick + vlo], 1ULL);
                }
                ++k;
            }
            w = pick;
            --lw;
            ++step;
        }
    }
    return true;
}

// The persistent launch: every batch of a phase in turn, separated by grid
// barriers.  Batches come from a host plan (many graphs), from the lane count
// the grouping left in device memory (W lanes each, so a phase needs no host
// round trip), or are the single batch given in the arguments.
template <int K, bool INSTR, int SM>
__global__ void __launch_bounds__(kMsBlock, 4) k_msbfs(MsArgs a) {
    constexpr int W = 64 * K;
    MsCtl *ctl = a.ctl;
    GridBarrier *bar = reinterpret_cast<GridBarrier *>(ctl);
    uint32_t *status = &ctl->status;
    int64_t B = 1;
    long long U = 0;
    if (a.plan) {
        B = a.nplan;
    } else if (a.u_dev) {
        U = *a.u_dev;
        B = (U + W - 1) / W;
    }
    for (int64_t b = 0; b < B; ++b) {
        int32_t lane_base = a.lane_base, nlanes = a.nlanes, vlo = a.vlo;
        int64_t n = a.n;
        if (a.plan) {
            lane_base = a.plan[b].lane_base;
            nlanes = a.plan[b].nlanes;
            vlo = a.plan[b].vlo;
            n = a.plan[b].nr;
        } else if (a.u_dev) {
            lane_base = (int32_t)(b * W);
            nlanes = (int32_t)min((long long)W, U - b * W);
        }
        // the previous batch's backtrack reads what this batch's prologue clears
        if (b > 0 && !grid_sync(bar, status, a.budget_ns)) return;
        if (!ms_batch<K, INSTR, SM>(a, lane_base, nlanes, vlo, n, a.rp + vlo, a.irp + vlo, a.ap_epoch)) return;
    }
}

// dist/sigma of every lane after a full traversal, source-major output.
template <int K, int SM>
__global__ void k_ms_extract(const uint64_t *fh, const void *sigma_v, int64_t n, int32_t levels, int32_t nsrc,
                             int32_t *dist, double *sig) {
    constexpr int W = 64 * K;
    using ST = typename SigmaMode<SM>::ST;
    const ST *sigma = static_cast<const ST *>(sigma_v);
    const int64_t total = n * (int64_t)nsrc;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
        const int64_t j = q / n, v = q % n;
        int32_t d = -1;
        for (int32_t L = 0; L <= levels; ++L) {
            if ((fh[(int64_t)L * n * K + v * K + (j >> 6)] >> (j & 63)) & 1ull) {
                d = L;
                break;
            }
        }
        if (dist) dist[q] = d;
        if (sig) sig[q] = d >= 0 ? (double)sigma[v * W + j] : 0.0;
    }
}

struct GridCache {
    int grid[2][3][4] = {};
};
GridCache g_ms_grid;

template <int K, bool INSTR, int SM>
int ms_grid(percis_ctx *ctx) {
    const int idx = K == 1 ? 0 : K == 2 ? 1 : K == 4 ? 2 : 3;
    int &slot = g_ms_grid.grid[INSTR ? 1 : 0][SM][idx];
    if (slot == 0) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_msbfs<K, INSTR, SM>, kMsBlock, 0);
        slot = std::max(1, per_sm) * ctx->num_sms;
    }
    return slot;
}

template <int K, bool INSTR, int SM>
percis_status launch_ms(percis_ctx *ctx, MsArgs &a) {
    void *args[] = {&a};
    const int grid = ms_grid<K, INSTR, SM>(ctx);
    PERCIS_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)k_msbfs<K, INSTR, SM>, dim3(grid), dim3(kMsBlock),
                                                 args, 0, ctx->stream));
    ctx->launches++;
    return PERCIS_OK;
}

template <int SM>
percis_status launch_ms_k2(percis_ctx *ctx, int K, MsArgs &a) {
    const bool instr = a.counters != nullptr;
    switch (K) {
        case 1: return instr ? launch_ms<1, true, SM>(ctx, a) : launch_ms<1, false, SM>(ctx, a);
        case 2: return instr ? launch_ms<2, true, SM>(ctx, a) : launch_ms<2, false, SM>(ctx, a);
        case 4: return instr ? launch_ms<4, true, SM>(ctx, a) : launch_ms<4, false, SM>(ctx, a);
        default: return instr ? launch_ms<8, true, SM>(ctx, a) : launch_ms<8, false, SM>(ctx, a);
    }
}

int ms_grid_for(percis_ctx *ctx, int K) {
    switch (K) {
        case 1: return ms_grid<1, false, 0>(ctx);
        case 2: return ms_grid<2, false, 0>(ctx);
        case 4: return ms_grid<4, false, 0>(ctx);
        default: return ms_grid<8, false, 0>(ctx);
    }
}

percis_status launch_ms_k(percis_ctx *ctx, int K, MsArgs &a) {
    switch (ctx->sigma_mode) {
        case 0: return launch_ms_k2<0>(ctx, K, a);
        case 1: return launch_ms_k2<1>(ctx, K, a);
        default: return launch_ms_k2<2>(ctx, K, a);
    }
}

percis_status ensure_ms(percis_ctx *ctx, int W, int Lcap, int64_t nr) {
    const int64_t n = nr;  // vertices of the largest launch range
    const int K = W / 64;
    PERCIS_TRY(ensure(ctx, ctx->fq0, sizeof(int32_t) * n, "frontier queue"));
    PERCIS_TRY(ensure(ctx, ctx->fq1, sizeof(int32_t) * n, "frontier queue"));
    PERCIS_TRY(ensure(ctx, ctx->vis, sizeof(uint64_t) * n * K, "visited bits"));
    PERCIS_TRY(ensure(ctx, ctx->fhist, sizeof(uint64_t) * n * K * (int64_t)(Lcap + 1), "frontier history"));
    PERCIS_TRY(ensure(ctx, ctx->sigmaW, sizeof(double) * n * W, "lane sigma"));
    PERCIS_TRY(ensure(ctx, ctx->remaining, sizeof(int32_t) * 512, "lane remaining"));
    PERCIS_TRY(ensure(ctx, ctx->ms_ctl, sizeof(MsCtl), "ms ctl"));
    return PERCIS_OK;
}

void fill_common(percis_ctx *ctx, MsArgs &a, int Lcap) {
    a.n = ctx->n;
    a.irp = ctx->directed ? ctx->irp.as<int64_t>() : ctx->rp.as<int64_t>();
    a.icol = ctx->directed ? ctx->icol.as<int32_t>() : ctx->col.as<int32_t>();
    a.vis = ctx->vis.as<uint64_t>();
    a.fh = ctx->fhist.as<uint64_t>();
    a.sigma = ctx->sigmaW.p;
    a.ctl = ctx->ms_ctl.as<MsCtl>();
    a.Lcap = Lcap;
    a.budget_ns = (uint64_t)(ctx->opt.timeout_s * 1e9);
    a.rp = ctx->rp.as<int64_t>();
    a.col = ctx->col.as<int32_t>();
    a.counters = nullptr;
    a.levdeg = nullptr;
    a.fq0 = ctx->fq0.as<int32_t>();
    a.fq1 = ctx->fq1.as<int32_t>();
    a.policy = ctx->opt.direction;
    a.push_alpha = ctx->opt.push_alpha > 0.0 ? ctx->opt.push_alpha : 0.5;
}

}  // namespace

int choose_lanes(percis_ctx *ctx, int64_t n_sources) {
    int W = ctx->opt.lanes;
    if (W != 64 && W != 128 && W != 256 && W != 512) {
        W = 512;
        while (W > 64 && (int64_t)W / 2 >= n_sources) W /= 2;
        // keep the lane sigma array within a modest share of device memory
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess) {
            const double nv = (double)(ctx->multi ? multi_range(ctx) : ctx->n);
            while (W > 64 && nv * W * 8.0 > 0.25 * (double)total_b) W /= 2;
        }
    }
    return W;
}

percis_status batched_phase(percis_ctx *ctx, uint64_t seed, uint32_t tag_path, int64_t count, int64_t n_sources,
                            int64_t *batches) {
    const int W = choose_lanes(ctx, n_sources);
    const int K = W / 64;
    int Lcap = std::max(ctx->levels_alloc, 32);
    // many graphs: a host plan of lane batches over vertex ranges; one graph:
    // W-lane batches over the lane count the grouping left on the device
    std::vector<LaneBatch> plan;
    int64_t nr_max = ctx->n;
    if (ctx->multi) {
        PERCIS_TRY(multi_plan_batches(ctx, n_sources, W, &plan));
        nr_max = 1;
        for (const LaneBatch &lb : plan) nr_max = std::max(nr_max, lb.nr);
    }
    if (!ctx->directed && ctx->vertex_diam > 0) {
        // no undirected shortest path has more than D + 1 edges: enough levels
        // up front (within a 16 GiB frontier history), so deep graphs need no
        // re-runs with a longer history
        const int64_t lmem = (16ll << 30) / std::max<int64_t>(1, nr_max * K * 8) - 1;
        Lcap = (int)std::max<int64_t>(Lcap, std::min<int64_t>(ctx->vertex_diam + 3, std::min<int64_t>(lmem, 1 << 20)));
    }
    PERCIS_TRY(ensure_ms(ctx, W, Lcap, nr_max));
    ctx->levels_alloc = Lcap;
    ctx->lanes_alloc = W;
    PERCIS_TRY(ensure(ctx, ctx->found, sizeof(int32_t) * (count + 1), "found"));
    PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->ms_ctl.p, 0, sizeof(MsCtl), ctx->stream));
    const int64_t B = ctx->multi ? (int64_t)plan.size() : (n_sources + W - 1) / W;
    *batches = B;
    MsArgs a{};
    fill_common(ctx, a, Lcap);
    a.lane_src = ctx->lane_src.as<int32_t>();
    a.lane_off = ctx->lane_off.as<long long>();
    a.samp_t = ctx->samp_t.as<int32_t>();
    a.samp_lane = ctx->samp_lane.as<int32_t>();
    a.sorted_samples = ctx->sorted_samples.as<int32_t>();
    a.found = ctx->found.as<int32_t>();
    a.remaining = ctx->remaining.as<int32_t>();
    a.seed = seed;
    a.tag = tag_path;
    a.kind = ctx->kind.as<int32_t>();
    a.ilen = ctx->ilen.as<int32_t>();
    a.path_off = ctx->path_off.as<long long>();
    a.arena = ctx->arena.as<int32_t>();
    a.arena_top = ctx->arena_top.as<unsigned long long>();
    a.arena_cap = ctx->arena_cap;
    a.cnt = ctx->cnt.as<unsigned long long>();
    a.full = 0;
    if (ctx->opt.instrument) {
        PERCIS_TRY(ensure(ctx, ctx->levdeg, sizeof(unsigned long long) * W * (size_t)(Lcap + 1), "level degrees"));
        a.counters = ctx->counters.as<unsigned long long>();
        a.levdeg = ctx->levdeg.as<unsigned long long>();
    }
    a.allpaths = ctx->opt.estimator == 1;
    if (a.allpaths) {
        // per-warp scratch of 20 n bytes, within a 8 GiB budget
        const int64_t n = nr_max;
        const int64_t per_warp = 20 * n;
        const int64_t warps = (int64_t)ms_grid_for(ctx, K) * (kMsBlock / 32);
        const int64_t ap_warps = std::max<int64_t>(1, std::min<int64_t>(warps, (8ll << 30) / per_warp));
        if (ctx->ap_warps != ap_warps || ctx->ap_n != n) {
            PERCIS_TRY(ensure(ctx, ctx->ap_tau, sizeof(unsigned long long) * n * ap_warps, "all-paths tau"));
            PERCIS_TRY(ensure(ctx, ctx->ap_stamp, sizeof(int32_t) * n * ap_warps, "all-paths stamps"));
            PERCIS_TRY(ensure(ctx, ctx->ap_list, sizeof(int32_t) * 2 * n * ap_warps, "all-paths lists"));
            PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->ap_stamp.p, 0, sizeof(int32_t) * n * ap_warps, ctx->stream));
            ctx->ap_warps = ap_warps;
            ctx->ap_n = n;
            ctx->ap_epoch = 0;
        }
        if (ctx->ap_epoch > (1 << 30)) {
            PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->ap_stamp.p, 0, sizeof(int32_t) * n * ap_warps, ctx->stream));
            ctx->ap_epoch = 0;
        }
        a.ap_warps = (int32_t)ap_warps;
        a.acc_ap = ctx->acc_ap.as<double>();
        a.ap_tau = ctx->ap_tau.as<unsigned long long>();
        a.ap_stamp = ctx->ap_stamp.as<int32_t>();
        a.ap_list = ctx->ap_list.as<int32_t>();
    }
    if (ctx->multi) {
        PERCIS_TRY(ensure(ctx, ctx->plan_dev, sizeof(LaneBatch) * std::max<size_t>(plan.size(), 1), "batch plan"));
        PERCIS_CUDA(ctx, cudaMemcpyAsync(ctx->plan_dev.p, plan.data(), sizeof(LaneBatch) * plan.size(),
                                         cudaMemcpyHostToDevice, ctx->stream));
        a.plan = ctx->plan_dev.as<LaneBatch>();
        a.nplan = (int32_t)plan.size();
    } else {
        a.u_dev = ctx->lane_of_v.as<long long>() + ctx->n;  // number of lanes
    }
    if (a.allpaths) {
        a.ap_epoch = ctx->ap_epoch;
        ctx->ap_epoch += (int32_t)std::min<int64_t>(count, 1 << 30) + 1;
    }
    // every batch of the phase in one persistent launch
    cudaEvent_t e0 = next_event(ctx), e1 = next_event(ctx);
    if (e0) cudaEventRecord(e0, ctx->stream);
    PERCIS_TRY(launch_ms_k(ctx, K, a));
    if (e1) cudaEventRecord(e1, ctx->stream);
    return PERCIS_OK;
}

// Full traversal from nsrc <= 512 sources (inspection and exact centrality).
percis_status msbfs_full(percis_ctx *ctx, int32_t nsrc, const int32_t *sources, int32_t *dist, double *sigma) {
    ctx->sigma_mode = 0;
    int W = 64;
    while (W < nsrc) W *= 2;
    const int K = W / 64;
    int Lcap = std::max(ctx->levels_alloc, 32);
    for (int attempt = 0; attempt < 12; ++attempt) {
        PERCIS_TRY(ensure_ms(ctx, W, Lcap, ctx->n));
        ctx->levels_alloc = Lcap;
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->ms_ctl.p, 0, sizeof(MsCtl), ctx->stream));
        MsArgs a{};
        fill_common(ctx, a, Lcap);
        a.lane_src = sources;
        a.lane_base = 0;
        a.nlanes = nsrc;
        a.remaining = ctx->remaining.as<int32_t>();
        a.full = 1;
        PERCIS_TRY(launch_ms_k(ctx, K, a));
        MsCtl hc;
        PERCIS_CUDA(ctx, cudaMemcpyAsync(&hc, ctx->ms_ctl.p, sizeof(hc), cudaMemcpyDeviceToHost, ctx->stream));
        PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (hc.status & DEV_TIMEOUT) return set_err(ctx, PERCIS_E_TIMEOUT, "batched BFS timed out");
        if (hc.status & DEV_NEED_LEVELS) {
            Lcap *= 2;
            continue;
        }
        if ((hc.status & DEV_SIGMA_WIDE) && ctx->sigma_mode == 0) {
            ctx->sigma_mode = 1;  // counts reached 2^32: redo with 64-bit storage
            continue;
        }
        if ((hc.status & DEV_SIGMA_OVERFLOW) && ctx->sigma_mode == 1) {
            ctx->sigma_mode = 2;  // counts reached 2^53: redo with FP64 sigma
            continue;
        }
        const int levels = hc.level;
        if (!dist && !sigma) return PERCIS_OK;
        const int grid = grid_for(ctx, ctx->n * nsrc, 256);
        const void *sg = ctx->sigmaW.p;
        const uint64_t *fhp = ctx->fhist.as<uint64_t>();
        const int64_t nn = ctx->n;
#define PERCIS_EXTRACT(KK, SMM) \
    k_ms_extract<KK, SMM><<<grid, 256, 0, ctx->stream>>>(fhp, sg, nn, levels, nsrc, dist, sigma)
#define PERCIS_EXTRACT_K(SMM)            \
    switch (K) {                         \
        case 1: PERCIS_EXTRACT(1, SMM); break; \
        case 2: PERCIS_EXTRACT(2, SMM); break; \
        case 4: PERCIS_EXTRACT(4, SMM); break; \
        default: PERCIS_EXTRACT(8, SMM); break; \
    }
        if (ctx->sigma_mode == 0) {
            PERCIS_EXTRACT_K(0);
        } else if (ctx->sigma_mode == 1) {
            PERCIS_EXTRACT_K(1);
        } else {
            PERCIS_EXTRACT_K(2);
        }
#undef PERCIS_EXTRACT_K
#undef PERCIS_EXTRACT
        PERCIS_CHECK_LAUNCH(ctx, "ms extract");
        return PERCIS_OK;
    }
    return set_err(ctx, PERCIS_E_TOO_LARGE, "frontier history exceeded the level cap");
}

}  // namespace percis
