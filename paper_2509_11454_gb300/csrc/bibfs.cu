// RandomSP by a balanced bidirectional BFS (Section III-B), one block per
// sample.  The paper names the traversal but not its details; the reading
// (the same one the oracle follows):
//   * forward side from s over out-edges, backward side from t over in-edges,
//     each with its own levels and exact integer path counts;
//   * while both frontiers are non-empty, the side whose frontier has the
//     smaller sum of degrees (in its direction; forward on a tie) expands one
//     level;
//   * the first new level that holds vertices the other side has reached ends
//     the search: those vertices all sit at the other side's last level b, so
//     d(s,t) = a + b and sigma_st = sum over them of sigma_s(v) sigma_t(v);
//   * the meeting vertex is the first, in vertex-id order, whose running sum of
//     sigma_s sigma_t reaches u_0 sigma_st; both sides are then backtracked
//     from it (towards s over in-edges, towards t over out-edges), each step
//     taking the first candidate whose running count reaches u sigma(w).
// Samples are independent, so blocks take them from a shared counter and
// never wait on one another.  Each block owns a slot of scratch arrays
// (level + epoch word, count and queue per vertex and side); a vertex belongs
// to the current sample only while its word carries the sample's epoch, so
// nothing is ever cleared: a claim swaps a side's {level word, count} pair in
// one 16-byte compare-and-swap, setting the count to the claiming parent's,
// and the other parents of the level add theirs, all in one pass over the
// level's edges.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace percis {

namespace {

#ifndef PERCIS_BI_BLOCK
#define PERCIS_BI_BLOCK 256
#endif
constexpr int kBiBlock = PERCIS_BI_BLOCK;
#ifndef PERCIS_MEET_CAP
#define PERCIS_MEET_CAP 256
#endif
constexpr int kMeetCap = PERCIS_MEET_CAP;  // meeting-layer members kept in shared memory
constexpr int kFlat = 512;  // frontiers up to this size have their edges spread over the block
#ifndef PERCIS_BI_MINB
#define PERCIS_BI_MINB 6
#endif

struct BiArgs {
    int64_t n;
    const int64_t *rp, *irp;
    const int32_t *col, *icol;
    int64_t count;
    const int32_t *pair_s, *pair_t;
    int32_t *kind, *ilen;
    long long *path_off;
    int32_t *arena;
    unsigned long long *arena_top;
    int64_t arena_cap;
    unsigned long long *cnt;
    uint64_t seed;
    uint32_t tag;
    uint32_t epoch_base;
    unsigned long long *vs;     // [slots][n][4]: per vertex and side {level word (epoch << 32 |
                                // level), path count}, side 0 first: one 32-byte sector holds
                                // everything a visit touches
    int32_t *queue;             // [slots][2][n]: visited vertices of each side in level order
    int32_t slots;
    unsigned long long *next;   // next sample to take
    uint32_t *status;
    // many graphs: records are indexed within the sample's graph (vertex - its
    // first id), so a slot holds nslot records (the largest graph)
    const int32_t *gid;         // graph of every vertex, or null for one graph
    const int64_t *vbase;       // first vertex id of every graph
    int64_t nslot;
    unsigned long long *work;   // optional work counters: [0] edges scanned, [1] count additions,
                                // [2] vertices reached (both sides), [3] samples traversed
};

// one field of the per-vertex records, indexed by vertex
struct Strided {
    unsigned long long *p;
    __device__ __forceinline__ unsigned long long &operator[](int64_t v) const { return p[4 * v]; }
};

// the path-count fields, as exact integers or (past 2^53) as FP64
template <class C>
struct CountView {
    unsigned long long *p;
    __device__ __forceinline__ C &operator[](int64_t v) const { return *reinterpret_cast<C *>(p + 4 * v); }
};

__device__ __forceinline__ unsigned long long pack(uint32_t ep, uint32_t lev) {
    return ((unsigned long long)ep << 32) | lev;
}

template <class C>
__device__ __forceinline__ unsigned long long count_bits(C c) {
    if constexpr (std::is_floating_point<C>::value) return (unsigned long long)__double_as_longlong(c);
    else return c;
}
template <class C>
__device__ __forceinline__ C count_of(unsigned long long b) {
    if constexpr (std::is_floating_point<C>::value) return __longlong_as_double((long long)b);
    else return b;
}

// one side's {level word, count} of a vertex: 16 aligned bytes, read in one request
__device__ __forceinline__ void ld_pair(const unsigned long long *p, unsigned long long &w, unsigned long long &c) {
    asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(w), "=l"(c) : "l"(p) : "memory");
}

// 16-byte compare-and-swap of {level word, count}: the previous pair
__device__ __forceinline__ void cas_pair(unsigned long long *p, unsigned long long cw, unsigned long long cc,
                                         unsigned long long nw, unsigned long long nc, unsigned long long &ow,
                                         unsigned long long &oc) {
    asm volatile(
        "{\n\t.reg .b128 d, c, s;\n\t"
        "mov.b128 c, {%2, %3};\n\t"
        "mov.b128 s, {%4, %5};\n\t"
        "atom.global.cas.b128 d, [%6], c, s;\n\t"
        "mov.b128 {%0, %1}, d;\n\t}"
        : "=l"(ow), "=l"(oc)
        : "l"(cw), "l"(cc), "l"(nw), "l"(nc), "l"(p)
        : "memory");
}

template <class T>
__device__ __forceinline__ T block_sum(T v, T *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T t = T(0);
    for (int q = 0; q < kBiBlock / 32; ++q) t += red[q];
    return t;
}

// C = unsigned long long: exact counts (flagged at 2^53, products checked);
// C = double: FP64 counts, the rerun of a phase whose counts passed 2^53.
template <class C>
__global__ void __launch_bounds__(kBiBlock, PERCIS_BI_MINB) k_bibfs(BiArgs a) {
    constexpr bool FP = std::is_floating_point<C>::value;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nw = kBiBlock / 32;
    const int64_t n = a.n;
    const size_t slot = blockIdx.x;
    // side 0 = forward from s over out-edges, side 1 = backward from t over in-edges
    unsigned long long *const vslot = a.vs + slot * (size_t)a.nslot * 4;
    int32_t *const queue0 = a.queue + (slot * 2) * a.nslot, *const queue1 = queue0 + a.nslot;

    __shared__ long long s_i;
    // claims of a level go to counter set it % 3; thread 0 clears set (it + 1) % 3
    // at the start of level it, two barriers after its last readers
    __shared__ int s_new[3], s_meet;
    __shared__ unsigned long long s_newcost[3];
    __shared__ int s_nm;
    __shared__ int32_t s_mv[kMeetCap];
    __shared__ C s_mw[kMeetCap];
    __shared__ C s_redc[nw];
    __shared__ int32_t s_best[nw];
    __shared__ int64_t s_fe[kFlat];  // first edge of each frontier vertex
    __shared__ C s_fs[kFlat];
    __shared__ int32_t s_pre[kFlat + 1];
    __shared__ unsigned long long s_work[4];
    if (threadIdx.x < 4) s_work[threadIdx.x] = 0ull;
    unsigned long long n_add = 0ull;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_i = (long long)atomicAdd(a.next, 1ull);
        __syncthreads();
        const long long i = s_i;
        if (i >= a.count) break;
        if (a.kind[i] != 0) {  // zero weight: no path (block-uniform)
            if (threadIdx.x == 0) {
                a.ilen[i] = 0;
                a.path_off[i] = 0;
            }
            continue;
        }
        const int32_t s = a.pair_s[i], t = a.pair_t[i];
        const uint32_t ep = a.epoch_base + (uint32_t)i + 1u;
        // record of vertex v at vrec[4 (v - base)]: the sample's graph starts at base
        const int64_t base = a.gid ? a.vbase[a.gid[s]] : 0;
        unsigned long long *const vrec = vslot - 4 * base;
        // record: {level word, count} of side 0, then of side 1
        const Strided info0{vrec}, info1{vrec + 2};
        const CountView<C> sig0{vrec + 1}, sig1{vrec + 3};
        if (threadIdx.x == 0) {
            info0[s] = pack(ep, 0);
            sig0[s] = C(1);
            queue0[0] = s;
            info1[t] = pack(ep, 0);
            sig1[t] = C(1);
            queue1[0] = t;
            s_new[0] = 0;
            s_newcost[0] = 0ull;
            s_meet = 0;
        }
        __syncthreads();
        // level state of both sides, the same in every thread
        long long qlo[2] = {0, 0}, qhi[2] = {1, 1};
        uint32_t lev[2] = {0u, 0u};
        unsigned long long cost[2] = {(unsigned long long)(a.rp[s + 1] - a.rp[s]),
                                      (unsigned long long)(a.irp[t + 1] - a.irp[t])};
        int x = 0;
        bool met = s != t;
        if (met) {
            met = false;
            for (int it = 0;; ++it) {
                if (qhi[0] == qlo[0] || qhi[1] == qlo[1]) break;  // a side ran dry: t unreachable
                x = cost[0] <= cost[1] ? 0 : 1;
                const long long lo = x ? qlo[1] : qlo[0], hi = x ? qhi[1] : qhi[0];
                const uint32_t nl = (x ? lev[1] : lev[0]) + 1;
                const int cs = it % 3;
                if (threadIdx.x == 0) {
                    s_new[(it + 1) % 3] = 0;
                    s_newcost[(it + 1) % 3] = 0ull;
                }
                const unsigned long long want = pack(ep, nl);
                unsigned long long ne = 0ull;
                // level nl: claim unreached neighbours and add the counts over
                // every edge into the level in one pass
                const Strided infx = x ? info1 : info0;
                const CountView<C> sigx = x ? sig1 : sig0;
                const Strided infy = x ? info0 : info1;
                int32_t *qx = x ? queue1 : queue0;
                const int64_t *px = x ? a.irp : a.rp;
                const int32_t *ax = x ? a.icol : a.col;
                const long long f = hi - lo;
                // one edge: claim the neighbour if unreached, add the parent's count if
                // it lies on the new level.  A claim swaps the whole {level word,
                // count} pair, so it also sets the count to the claiming parent's and
                // counts never need clearing: a count is read only where its level
                // word carries the sample's epoch.
                auto visit = [&](const int32_t v, const C su) {
                    unsigned long long *const pr = &infx[v];
                    // what a claim needs (degree, the other side's level word) is read
                    // alongside the pair, off the claim's dependent chain
                    const uint32_t dg = (uint32_t)(px[v + 1] - px[v]);  // < 2^31
                    const unsigned long long oy = __ldcg(&infy[v]);
                    unsigned long long ow, oc;
                    ld_pair(pr, ow, oc);
                    bool at = ow == want, won = false;
                    if ((uint32_t)(ow >> 32) != ep) {
                        unsigned long long pw, pc;
                        cas_pair(pr, ow, oc, want, count_bits(su), pw, pc);
                        if (pw == ow && pc == oc) {
                            won = true;
                            // the lanes that claimed together reserve their queue slots and
                            // add their degrees with one shared atomic each (a 64-bit shared
                            // add would be a contended compare-and-swap loop per lane)
                            const unsigned grp = __activemask();
                            const int lead = __ffs(grp) - 1;
                            const uint32_t dlo = __reduce_add_sync(grp, dg & 0xffffu);
                            const uint32_t dhi = __reduce_add_sync(grp, dg >> 16);
                            int q0 = 0;
                            if (lane == lead) {
                                q0 = atomicAdd(&s_new[cs], __popc(grp));
                                atomicAdd(&s_newcost[cs], ((unsigned long long)dhi << 16) + dlo);
                            }
                            q0 = __shfl_sync(grp, q0, lead);
                            qx[hi + q0 + __popc(grp & ((1u << lane) - 1u))] = v;
                            if ((uint32_t)(oy >> 32) == ep) s_meet = 1;
                        } else {
                            at = pw == want;  // claimed in this level by another thread
                        }
                    }
                    if (a.work && (at || won)) ++n_add;
                    if (at) {
                        const C o = atomicAdd(&sigx[v], su);
                        if ((double)(o + su) >= kTwo53) atomicOr(a.status, DEV_SIGMA_OVERFLOW);
                    }
                };
                // (the flat form keeps the level's edge offsets in 32 bits)
                if (f <= kFlat && (x ? cost[1] : cost[0]) < (1ull << 31)) {
                    // the level's edges spread evenly over the block (a hub's
                    // adjacency is not left to one warp): warp 0 loads the frontier and
                    // writes its degree prefix sums to shared memory, each edge then
                    // finds its vertex by bisection
                    if (warp == 0) {
                        constexpr int per = kFlat / 32;
                        int32_t loc[per];
                        int32_t tot = 0;
#pragma unroll
                        for (int r = 0; r < per; ++r) {
                            const long long k = (long long)lane * per + r;
                            int32_t dg = 0;
                            if (k < f) {
                                const int32_t u = qx[lo + k];
                                const int64_t e0 = px[u];
                                s_fe[k] = e0;
                                s_fs[k] = __ldcg(&sigx[u]);
                                dg = (int32_t)(px[u + 1] - e0);
                            }
                            loc[r] = tot;
                            tot += dg;
                        }
                        int32_t incl = tot;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const int32_t t2 = __shfl_up_sync(0xffffffffu, incl, o);
                            if (lane >= o) incl += t2;
                        }
                        const int32_t first = incl - tot;
#pragma unroll
                        for (int r = 0; r < per; ++r) {
                            const long long k = (long long)lane * per + r;
                            if (k < f) s_pre[k] = first + loc[r];
                        }
                        if (lane == 31) s_pre[f] = incl;
                    }
                    __syncthreads();
                    const int32_t E = s_pre[f];
                    ne = threadIdx.x == 0 ? (unsigned long long)E : 0ull;
                    for (int32_t j = threadIdx.x; j < E; j += kBiBlock) {
                        int32_t klo = 0, khi = (int32_t)f - 1;  // last k with s_pre[k] <= j
                        while (klo < khi) {
                            const int32_t mid = (klo + khi + 1) >> 1;
                            if (s_pre[mid] <= j) klo = mid;
                            else khi = mid - 1;
                        }
                        visit(ax[s_fe[klo] + (j - s_pre[klo])], s_fs[klo]);
                    }
                } else {
                    for (long long q = lo + warp; q < hi; q += nw) {
                        const int32_t u = qx[q];
                        const C su = __ldcg(&sigx[u]);
                        const int64_t e0 = px[u], e1 = px[u + 1];
                        if (lane == 0) ne += (unsigned long long)(e1 - e0);
                        for (int64_t e = e0 + lane; e < e1; e += 32) visit(ax[e], su);
                    }
                }
                if (a.work && ne) atomicAdd(&s_work[0], ne);
                __syncthreads();
                const long long nh = hi + s_new[cs];
                const unsigned long long nc = s_newcost[cs];
                if (x) {
                    qlo[1] = hi;
                    qhi[1] = nh;
                    lev[1] = nl;
                    cost[1] = nc;
                } else {
                    qlo[0] = hi;
                    qhi[0] = nh;
                    lev[0] = nl;
                    cost[0] = nc;
                }
                if (s_meet) {
                    met = true;
                    break;
                }
            }
        }
        if (!met) {
            if (threadIdx.x == 0) {
                a.kind[i] = 2;
                a.ilen[i] = 0;
                a.path_off[i] = 0;
            }
        } else {
            // meeting layer: level s_lev[x] of side x reached by the other side
            const Strided infy = x ? info0 : info1;
            const int32_t *qx = x ? queue1 : queue0;
            const long long mlo = x ? qlo[1] : qlo[0], mhi = x ? qhi[1] : qhi[0];
            // the layer's members with their weights sigma_s sigma_t, kept in
            // shared memory when they fit
            if (threadIdx.x == 0) s_nm = 0;
            __syncthreads();
            C part = C(0);
            for (long long q = mlo + threadIdx.x; q < mhi; q += kBiBlock) {
                const int32_t v = qx[q];
                if ((uint32_t)(__ldcg(&infy[v]) >> 32) == ep) {
                    const C a0 = __ldcg(&sig0[v]), a1 = __ldcg(&sig1[v]);
                    const C p = a0 * a1;
                    if ((double)a0 * (double)a1 >= kTwo53) atomicOr(a.status, DEV_SIGMA_OVERFLOW);
                    part += p;
                    const int slot_m = atomicAdd(&s_nm, 1);
                    if (slot_m < kMeetCap) {
                        s_mv[slot_m] = v;
                        s_mw[slot_m] = p;
                    }
                }
            }
            const C sst = block_sum(part, s_redc);
            if (threadIdx.x == 0 && (double)sst >= kTwo53) atomicOr(a.status, DEV_SIGMA_OVERFLOW);
            const double target = __dmul_rn(uniform_at(a.seed, (uint64_t)i, a.tag, 0), (double)sst);
            const int nm = s_nm;
            if (a.work && threadIdx.x == 0 && nm > kMeetCap) s_work[3] += 1ull << 32;  // large layers (high word)
            int32_t vm;
            if (nm <= kMeetCap) {
                // member j qualifies when the weights of the members with ids <= its
                // own reach the target; the meeting vertex is the smallest such id
                int32_t best = 0x7fffffff;
                for (int j = threadIdx.x; j < nm; j += kBiBlock) {
                    const int32_t vj = s_mv[j];
                    C pre = C(0);
                    for (int k2 = 0; k2 < nm; ++k2)
                        if (s_mv[k2] <= vj) pre += s_mw[k2];
                    if ((double)pre >= target) best = min(best, vj);
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, off));
                __syncthreads();
                if (lane == 0) s_best[warp] = best;
                __syncthreads();
                vm = s_best[0];
                for (int q = 1; q < nw; ++q) vm = min(vm, s_best[q]);
            } else {
                // a large layer: the first vertex id T whose layer prefix sum
                // reaches the target, by bisection over the ids
                int32_t blo = 0, bhi = (int32_t)(n - 1);
                while (blo < bhi) {
                    const int32_t mid = blo + (bhi - blo) / 2;
                    C pm = C(0);
                    for (long long q = mlo + threadIdx.x; q < mhi; q += kBiBlock) {
                        const int32_t v = qx[q];
                        if (v <= mid && (uint32_t)(__ldcg(&infy[v]) >> 32) == ep)
                            pm += __ldcg(&sig0[v]) * __ldcg(&sig1[v]);
                    }
                    const C sm = block_sum(pm, s_redc);
                    if ((double)sm >= target) bhi = mid;
                    else blo = mid + 1;
                }
                vm = blo;
            }
            if (warp == 0) {
                const uint32_t la = (uint32_t)(__ldcg(&info0[vm]) & 0xffffffffu);
                const uint32_t lb = (uint32_t)(__ldcg(&info1[vm]) & 0xffffffffu);
                const int32_t len = (int32_t)(la + lb) - 1;
                unsigned long long off = 0ull;
                if (lane == 0) {
                    off = atomicAdd(a.arena_top, (unsigned long long)len);
                    if ((int64_t)(off + len) > a.arena_cap) atomicOr(a.status, DEV_ARENA_OVERFLOW);
                    a.ilen[i] = len;
                    a.path_off[i] = (long long)off;
                }
                off = __shfl_sync(0xffffffffu, off, 0);
                const bool store = (int64_t)(off + len) <= a.arena_cap;
                int32_t k = 0;
                if (vm != s && vm != t) {
                    if (lane == 0) {
                        if (store) a.arena[off] = vm;
                        atomicAdd(&a.cnt[vm], 1ull);
                    }
                    k = 1;
                }
                uint32_t step = 1;
                for (int z = 0; z < 2; ++z) {
                    // towards s: predecessors over in-edges; towards t: successors over out-edges
                    const int64_t *bp = z == 0 ? a.irp : a.rp;
                    const int32_t *bc = z == 0 ? a.icol : a.col;
                    const Strided infz = z == 0 ? info0 : info1;
                    const CountView<C> sigz = z == 0 ? sig0 : sig1;
                    const int32_t endz = z == 0 ? s : t;
                    int32_t w = vm;
                    while (w != endz) {
                        const uint32_t lw = (uint32_t)(__ldcg(&infz[w]) & 0xffffffffu);
                        const unsigned long long prev = pack(ep, lw - 1);
                        const double tg = __dmul_rn(uniform_at(a.seed, (uint64_t)i, a.tag, step),
                                                    (double)__ldcg(&sigz[w]));
                        const int64_t e0 = bp[w], e1 = bp[w + 1];
                        C carry = C(0);
                        int32_t pick = -1, last = -1;
                        for (int64_t base = e0; base < e1 && pick < 0; base += 32) {
                            const int64_t e = base + lane;
                            int32_t pv = -1;
                            C val = C(0);
                            if (e < e1) {
                                pv = bc[e];
                                unsigned long long lw2, lc2;
                                ld_pair(&infz[pv], lw2, lc2);
                                if (lw2 == prev) val = count_of<C>(lc2);
                            }
                            C cum = val;
#pragma unroll
                            for (int o = 1; o < 32; o <<= 1) {
                                const C t2 = __shfl_up_sync(0xffffffffu, cum, o);
                                if (lane >= o) cum += t2;
                            }
                            cum += carry;
                            const unsigned hit = __ballot_sync(0xffffffffu, val > C(0) && (double)cum >= tg);
                            if (hit) pick = __shfl_sync(0xffffffffu, pv, __ffs(hit) - 1);
                            const unsigned cand = __ballot_sync(0xffffffffu, val > C(0));
                            if (cand) last = __shfl_sync(0xffffffffu, pv, 31 - __clz(cand));
                            carry = __shfl_sync(0xffffffffu, cum, 31);
                        }
                        // FP64 counts past 2^53 may round the running sum just below u sigma(w):
                        // the last candidate then takes the remainder
                        if (pick < 0 && FP) pick = last;
                        if (pick < 0) {
                            if (lane == 0) atomicOr(a.status, DEV_BAD_PATH);
                            break;
                        }
                        if (pick != endz) {
                            if (lane == 0) {
                                if (store && k < len) a.arena[off + k] = pick;
                                atomicAdd(&a.cnt[pick], 1ull);
                            }
                            ++k;
                        }
                        w = pick;
                        ++step;
                    }
                }
            }
        }
        __syncthreads();
        if (a.work && threadIdx.x == 0) {
            s_work[2] += (unsigned long long)(qhi[0] + qhi[1]);
            s_work[3] += 1ull;
        }
    }
    if (a.work) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) n_add += __shfl_xor_sync(0xffffffffu, n_add, off);
        if (lane == 0 && n_add) atomicAdd(&s_work[1], n_add);
    }
    __syncthreads();
    if (a.work && threadIdx.x < 4 && s_work[threadIdx.x]) atomicAdd(&a.work[threadIdx.x], s_work[threadIdx.x]);
}

}  // namespace

// All samples of a phase (pairs, kinds already drawn): kinds of unreachable
// targets, |I|, paths and counts, as the batched form leaves them.
percis_status bidir_phase(percis_ctx *ctx, uint64_t seed, uint32_t tag_path, int64_t count) {
    const int64_t n = ctx->n;
    const int32_t *gid = nullptr;
    const int64_t *vbase = nullptr;
    int64_t nslot = n;
    if (ctx->multi) multi_graph_view(ctx, &gid, &vbase, &nslot);
    const size_t per_slot = (size_t)nslot * (sizeof(unsigned long long) * 4 + sizeof(int32_t) * 2);
    static int per_sm = 0;
    if (!per_sm) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bibfs<unsigned long long>, kBiBlock, 0) !=
                cudaSuccess ||
            per_sm < 1)
            per_sm = 1;
    }
    // at most 16 GiB of scratch
    int64_t slots = std::min<int64_t>((int64_t)per_sm * ctx->num_sms, std::max<int64_t>(1, (16ll << 30) / per_slot));
    slots = std::min<int64_t>(slots, std::max<int64_t>(count, 1));
    if (ctx->bi_slots < slots || ctx->bi_n != nslot) {
        PERCIS_TRY(ensure(ctx, ctx->bi_info, sizeof(unsigned long long) * 4 * nslot * slots, "bidirectional records"));
        PERCIS_TRY(ensure(ctx, ctx->bi_queue, sizeof(int32_t) * 2 * nslot * slots, "bidirectional queues"));
        // level words of no sample (epoch 0)
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->bi_info.p, 0, sizeof(unsigned long long) * 4 * nslot * slots, ctx->stream));
        ctx->bi_slots = slots;
        ctx->bi_n = nslot;
        ctx->bi_epoch = 0;
    }
    if ((uint64_t)ctx->bi_epoch + (uint64_t)count + 2 > 0xffffffffull) {
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->bi_info.p, 0, sizeof(unsigned long long) * 4 * nslot * ctx->bi_slots,
                                         ctx->stream));
        ctx->bi_epoch = 0;
    }
    PERCIS_TRY(ensure(ctx, ctx->ms_ctl, sizeof(MsCtl), "ms ctl"));
    // the status word may be freshly allocated: it must start at zero
    PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->ms_ctl.p, 0, sizeof(MsCtl), ctx->stream));
    PERCIS_TRY(ensure(ctx, ctx->red, 64, "sample counter"));
    PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->red.p, 0, sizeof(unsigned long long), ctx->stream));
    BiArgs a{};
    a.n = n;
    a.gid = gid;
    a.vbase = vbase;
    a.nslot = nslot;
    a.rp = ctx->rp.as<int64_t>();
    a.col = ctx->col.as<int32_t>();
    a.irp = ctx->directed ? ctx->irp.as<int64_t>() : ctx->rp.as<int64_t>();
    a.icol = ctx->directed ? ctx->icol.as<int32_t>() : ctx->col.as<int32_t>();
    a.count = count;
    a.pair_s = ctx->pair_s.as<int32_t>();
    a.pair_t = ctx->pair_t.as<int32_t>();
    a.kind = ctx->kind.as<int32_t>();
    a.ilen = ctx->ilen.as<int32_t>();
    a.path_off = ctx->path_off.as<long long>();
    a.arena = ctx->arena.as<int32_t>();
    a.arena_top = ctx->arena_top.as<unsigned long long>();
    a.arena_cap = ctx->arena_cap;
    a.cnt = ctx->cnt.as<unsigned long long>();
    a.seed = seed;
    a.tag = tag_path;
    a.epoch_base = (uint32_t)ctx->bi_epoch;
    ctx->bi_epoch += count + 1;
    a.vs = ctx->bi_info.as<unsigned long long>();
    a.queue = ctx->bi_queue.as<int32_t>();
    a.slots = (int32_t)ctx->bi_slots;
    a.next = ctx->red.as<unsigned long long>();
    a.status = &ctx->ms_ctl.as<MsCtl>()->status;
    a.work = ctx->opt.instrument ? ctx->counters.as<unsigned long long>() : nullptr;
    if (ctx->sigma_mode == 2) k_bibfs<double><<<(int)ctx->bi_slots, kBiBlock, 0, ctx->stream>>>(a);
    else k_bibfs<unsigned long long><<<(int)ctx->bi_slots, kBiBlock, 0, ctx->stream>>>(a);
    PERCIS_CHECK_LAUNCH(ctx, "bidirectional sigma-BFS");
    return PERCIS_OK;
}

}  // namespace percis
