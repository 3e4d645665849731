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
// never wait on one another.
//
// Scratch.  Each block owns a slot; a sample's state is one 32-byte entry per
// vertex it reached: per side a word {level, sample epoch} and a path count.
// A vertex belongs to the current sample only while a word carries the
// sample's epoch, so nothing is ever cleared: a claim swaps a side's {word,
// count} pair in one 16-byte compare-and-swap, setting the count to the
// claiming parent's, and the other parents of the level add theirs, all in
// one pass over the level's edges.  Two stores of the entries:
//   * hashed (every sample first): an open-addressing table per slot keyed by
//     vertex id (the words carry the vertex too), linear probing.  A sample
//     starts in a small table that stays in L2 across the samples of the slot
//     (2,048 entries = 64 KB by default) and, between levels, moves to a table
//     four times larger whenever the coming level could fill more than half of
//     it (the entries are re-inserted by walking both sides' queues).  Work and
//     memory follow the vertices a sample touches, not n.
//   * direct (samples that would overfill the largest table or pass 4,095
//     levels): entry v for vertex v, O(n) per slot, so few slots.  The hashed
//     pass hands such samples over untouched (it writes nothing outside its
//     slot before the sides meet).
// A sample's pairs, paths and counts do not depend on which store ran it.
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
constexpr int kMeetBuckets = 1024;          // id buckets per round of the large-layer search
constexpr int kBackWarp = 256;              // candidate lists up to this length: one warp per backtrack step
constexpr int kLvCap = 64;                  // levels per side whose queue ranges are kept (reverse backtrack)
constexpr int kFlat = 512;  // frontier vertices per chunk whose edges are spread over the block
#ifndef PERCIS_EDGE_BATCH
#define PERCIS_EDGE_BATCH 2
#endif
constexpr int kEdgeBatch = PERCIS_EDGE_BATCH;  // edges a thread has in flight (their loads issued together)
#ifndef PERCIS_HEAVY_EDGE_BATCH
#define PERCIS_HEAVY_EDGE_BATCH 2
#endif
constexpr int kHeavyEdgeBatch = PERCIS_HEAVY_EDGE_BATCH;  // the same in the heavy pass
#ifndef PERCIS_BI_MINB
#define PERCIS_BI_MINB 4
#endif
constexpr unsigned long long kHubDegree = 16384;  // graphs with a vertex of this degree get a heavy pass by default
// Meeting-scan filters and thresholds (build-time tuning constants, like the
// ones above: a variant build defines them).  Heavy pass: a 2^20-bit filter of
// the other side's vertices (128 KB; 2^19 measured the same).
#ifndef PERCIS_HEAVY_BLOOM_LOG
#define PERCIS_HEAVY_BLOOM_LOG 20
#endif
constexpr int kHeavyBloomLog = PERCIS_HEAVY_BLOOM_LOG;
constexpr int kBloomWords = 1 << (kHeavyBloomLog - 5);
#ifndef PERCIS_FIRST_BLOOM
#define PERCIS_FIRST_BLOOM 0
#endif
#ifndef PERCIS_MEET_HITS_FIRST
#define PERCIS_MEET_HITS_FIRST 3.0
#endif
// first pass: none by default (a 2^17-bit filter, 16 KB beside four blocks per SM,
// measured neutral on R-MAT 22 and Barabasi-Albert graphs)
constexpr int kBloomWordsFirst = PERCIS_FIRST_BLOOM ? (1 << 12) : 0;
// expected meeting hits above which a level is scanned for its meeting layer
// first: in the first pass, and in the heavy pass (whose filter makes a scan
// that finds no member cheap)
constexpr double kMeetOnlyHits = PERCIS_MEET_HITS_FIRST;
#ifndef PERCIS_MEET_HITS_BLOOM
#define PERCIS_MEET_HITS_BLOOM 0.02
#endif
constexpr double kMeetOnlyHitsBloom = PERCIS_MEET_HITS_BLOOM;
#ifndef PERCIS_MEET_BATCH
#define PERCIS_MEET_BATCH 8
#endif
constexpr int kMeetBatch = PERCIS_MEET_BATCH;  // columns a thread loads together in a filtered meeting scan
// first pass: samples taken in the queue's last kTailRounds rounds (one round =
// a sample per block) hand levels above kTailEdges to the heavy pass, so that
// no block of the pass ends long after the others (0: off; on R-MAT 22, two
// rounds at 2,048 edges cut the first passes by 0.17 ms a step, one or four
// rounds and 4,096 edges less)
#ifndef PERCIS_TAIL_ROUNDS
#define PERCIS_TAIL_ROUNDS 2
#endif
#ifndef PERCIS_TAIL_EDGES
#define PERCIS_TAIL_EDGES 2048
#endif
constexpr int kTailRounds = PERCIS_TAIL_ROUNDS;
constexpr unsigned long long kTailEdges = PERCIS_TAIL_EDGES;
constexpr unsigned long long kLazyDegEdges = 2048;  // levels of this many edges load degrees after
constexpr uint32_t kHashLevels = 4095;            // levels a hashed word holds (12 bits)
constexpr uint32_t kHashEpochs = (1u << 20) - 1;  // epochs a hashed word holds (20 bits)
constexpr int kMaxHLog = 20;                      // largest table: at most 2^20 entries
constexpr int kMinHLog = 10;                      // smallest table (new entries stop at 3/4 minus a block)
constexpr int kDefaultHLog = 18;                  // default: one table of at most 262,144 entries per block

struct BiArgs {
    int64_t n;
    const int64_t *rp, *irp;
    const int32_t *col, *icol;
    int64_t count;               // samples of the phase, or of the list
    const unsigned int *count_dev;  // when set: the list's length, read on the device
    const int32_t *list;         // sample indices to run (null: 0 .. count-1)
    const int32_t *pair_s, *pair_t;
    int32_t *kind, *ilen;
    long long *path_off;
    int32_t *arena;
    unsigned long long *arena_top;
    int64_t arena_cap;
    unsigned long long *cnt;
    uint64_t seed;
    uint32_t tag;
    unsigned long long *ent;     // entries: [slots][region][4] {word 0, count 0, word 1, count 1}
    int2 *queue;                 // [slots][3][qcap]: {vertex, entry} of each side in level order, then
                                 // the meeting layer's members (claims of vertices the other side holds)
    int64_t region;              // entries per slot
    int64_t qcap;                // queue entries per side and slot
    unsigned long long *next;    // next sample to take
    uint32_t *status;
    unsigned long long *work;    // optional work counters: [0] edges scanned, [1] count additions,
                                 // [2] vertices reached (both sides), [3] samples traversed (+ 2^32 per
                                 // meeting layer above the shared capacity), [4] samples handed to the
                                 // direct store, [5] table moves
    // direct store
    uint32_t epoch_base;         // epoch of sample i: epoch_base + i + 1 (32 bits)
    const int32_t *gid;          // many graphs: graph of every vertex (entries indexed within the
    const int64_t *vbase;        //   sample's graph: vertex - first id), or null for one graph
    // hashed store
    int32_t h0_log, hmax_log;    // first and largest table: 2^h0_log, 2^hmax_log entries (step x4)
    uint32_t *slot_epoch;        // per slot: last epoch used (20 bits; persists across launches)
    int32_t *deferred;           // samples handed to the heavy pass
    unsigned long long *defer_cost;  // edges of the level each was handed over at
    unsigned int *n_deferred;
    int32_t sorted;              // every adjacency list strictly increasing (reverse backtrack allowed)
    unsigned long long heavy_edges;  // a level scanning more edges than this hands the sample over (0: never)
    const unsigned long long *max_degree;  // largest out- or in-degree of the graph (device word)
    int32_t heavy_auto;          // heavy_edges applies only where max_degree >= kHubDegree
    unsigned long long *trace;   // optional, per sample: {start ns, end ns, edges scanned,
                                 // levels | store << 32 | slot << 33 | heavy pass << 63, end of the
                                 // levels ns, end of the meeting vertex's choice ns, and where a
                                 // backtrack found no candidate: kind | side << 4 | step << 8 |
                                 // list length << 32, vertex << 32 | its level}
};

// ------------------------------------------------------------------ words
// direct:  word = epoch (32) << 32 | level (32)
// hashed:  word = vertex (32) << 32 | epoch (20) << 12 | level (12)
template <bool HASH>
struct Word;
template <>
struct Word<false> {
    static __device__ __forceinline__ unsigned long long make(int32_t, uint32_t ep, uint32_t lev) {
        return ((unsigned long long)ep << 32) | lev;
    }
    static __device__ __forceinline__ bool current(unsigned long long w, uint32_t ep) {
        return (uint32_t)(w >> 32) == ep;
    }
    static __device__ __forceinline__ uint32_t level(unsigned long long w) { return (uint32_t)w; }
};
template <>
struct Word<true> {
    static __device__ __forceinline__ unsigned long long make(int32_t v, uint32_t ep, uint32_t lev) {
        return ((unsigned long long)(uint32_t)v << 32) | ((unsigned long long)ep << 12) | lev;
    }
    static __device__ __forceinline__ bool current(unsigned long long w, uint32_t ep) {
        return (uint32_t)((w >> 12) & 0xfffffu) == ep;
    }
    static __device__ __forceinline__ uint32_t level(unsigned long long w) { return (uint32_t)(w & 0xfffu); }
    static __device__ __forceinline__ int32_t vertex(unsigned long long w) { return (int32_t)(w >> 32); }
};

// home entry of vertex v in a table of 2^lg entries (Fibonacci hashing)
__device__ __forceinline__ uint32_t hash_home(int32_t v, int lg) {
    return ((uint32_t)v * 0x9E3779B1u) >> (32 - lg);
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

// one side's {word, count} of an entry: 16 aligned bytes, read in one request
__device__ __forceinline__ void ld_pair(const unsigned long long *p, unsigned long long &w, unsigned long long &c) {
    asm volatile("ld.global.cg.v2.u64 {%0, %1}, [%2];" : "=l"(w), "=l"(c) : "l"(p) : "memory");
}

__device__ __forceinline__ void st_pair(unsigned long long *p, unsigned long long w, unsigned long long c) {
    asm volatile("st.global.cg.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(w), "l"(c) : "memory");
}

// 16-byte compare-and-swap of {word, count}: the previous pair
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

template <int BT, class T>
__device__ __forceinline__ T block_sum(T v, T *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    T t = T(0);
    for (int q = 0; q < BT / 32; ++q) t += red[q];
    return t;
}

// Entry of vertex v in a hashed table (tab, 2^lg entries), or -1 when no word
// of the current sample carries v.  An entry holds one vertex: its words of
// the current epoch (one or both sides) all name it.
__device__ __forceinline__ int64_t hash_find(const unsigned long long *tab, int lg, int32_t v, uint32_t ep) {
    using W = Word<true>;
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t p = hash_home(v, lg);
    for (uint32_t k = 0; k <= mask; ++k, p = (p + 1) & mask) {
        const unsigned long long w0 = __ldcg(&tab[4ull * p]), w1 = __ldcg(&tab[4ull * p + 2]);
        const bool c0 = W::current(w0, ep), c1 = W::current(w1, ep);
        if (!c0 && !c1) return -1;
        if (W::vertex(c0 ? w0 : w1) == v) return p;
    }
    return -1;
}

// C = unsigned long long: exact counts (flagged at 2^53, products checked);
// C = double: FP64 counts, the rerun of a phase whose counts passed 2^53.
template <class C, bool HASH, int BT>
__global__ void __launch_bounds__(BT, BT == kBiBlock ? PERCIS_BI_MINB : 1024 / BT) k_bibfs(BiArgs a) {
    using W = Word<HASH>;
    // The heavy pass scans a meeting level against a Bloom filter of the other
    // side's vertices in shared memory (two hashes of the vertex id): a vertex
    // whose bits are not both set is not in the meeting layer, and its entry is
    // never loaded.  (The first pass has no room for it.)
    constexpr bool BLOOM = BT != kBiBlock || kBloomWordsFirst > 0;
    constexpr int NBW = BT == kBiBlock ? kBloomWordsFirst : kBloomWords;  // filter words
    constexpr int NBB = BT == kBiBlock ? 17 : kHeavyBloomLog;              // filter bits (log2)
    extern __shared__ uint32_t s_bloom[];  // NBW words
    auto bloom_bits = [](int32_t v, uint32_t &h1, uint32_t &h2) {
        const unsigned long long m = (unsigned long long)(uint32_t)v * 0x9E3779B97F4A7C15ull;
        h1 = (uint32_t)(m >> (64 - NBB));
        h2 = (uint32_t)(m >> 24) & ((1u << NBB) - 1u);
    };
    constexpr bool FP = std::is_floating_point<C>::value;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int nw = BT / 32;
    const int64_t n = a.n;
    const size_t slot = blockIdx.x;
    unsigned long long *const sent = a.ent + slot * (size_t)a.region * 4;
    int2 *const queue0 = a.queue + (slot * 3) * (size_t)a.qcap, *const queue1 = queue0 + a.qcap;
    int2 *const memb = queue1 + a.qcap;

    __shared__ long long s_i;
    __shared__ int s_tail;
    // claims of a level go to counter set it % 3; thread 0 clears set (it + 1) % 3
    // at the start of level it, two barriers after its last readers
    __shared__ int s_new[3], s_meet, s_full;
    __shared__ C s_bkt[kMeetBuckets];
    __shared__ int s_sel;
    __shared__ C s_base;
    __shared__ unsigned long long s_off;  // the sample's path slot in the arena
    __shared__ int32_t s_pick;            // a backtrack step's choice
    __shared__ long long s_pickp;
    __shared__ int s_tstar, s_tlast;      // segment of a long candidate list holding the choice
    __shared__ C s_tpre;
    __shared__ int32_t s_lv[2][kLvCap + 2];  // queue range of level L of a side: [s_lv[L], s_lv[L+1])
    __shared__ int32_t s_mj[kMeetCap];       // a reverse backtrack candidate's place in the list
    __shared__ int s_nc;
    __shared__ unsigned long long s_newcost[3];
    __shared__ int32_t s_mv[kMeetCap];
    __shared__ int32_t s_mp[kMeetCap];
    __shared__ C s_mw[kMeetCap];
    __shared__ C s_redc[nw];
    __shared__ unsigned long long s_best[nw];
    __shared__ int64_t s_fe[kFlat];  // first edge of each frontier vertex of a chunk
    __shared__ C s_fs[kFlat];        // its path count
    __shared__ int64_t s_pre[kFlat + 1];  // prefix sums of the chunk's degrees
    __shared__ unsigned long long s_work[6];
    __shared__ long long s_wsum[nw];    // per-warp degree sums of a chunk
    __shared__ double s_wcnt[nw];       // per-warp sums of a chunk's path counts
    if (threadIdx.x < 6) s_work[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) s_tlast = -1;
    unsigned long long n_add = 0ull;
    uint32_t ep_slot = HASH ? a.slot_epoch[slot] : 0u;
    const long long count = a.count_dev ? (long long)__ldcg(a.count_dev) : a.count;
    // default rule: a heavy pass only where hubs can make a single level huge
    const unsigned long long heavy_lim =
        (a.heavy_auto && a.max_degree && __ldg(a.max_degree) < kHubDegree) ? 0ull : a.heavy_edges;

    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const long long k = (long long)atomicAdd(a.next, 1ull);
            s_i = k < count ? (a.list ? (long long)a.list[k] : k) : -1ll;
            s_tail = kTailRounds > 0 && k >= count - (long long)kTailRounds * gridDim.x;
        }
        __syncthreads();
        const long long i = s_i;
        // (block-uniform) the level size above which this sample is handed over
        const unsigned long long lim =
            (heavy_lim && s_tail && kTailEdges < heavy_lim) ? kTailEdges : heavy_lim;
        if (i < 0) break;
        const unsigned long long t_start = a.trace && threadIdx.x == 0 ? globaltimer_ns() : 0ull;
        unsigned long long t_levels = 0ull, t_meet = 0ull;
        unsigned long long smp_edges = 0ull;  // (thread 0)
        int smp_levels = 0;
        if (a.kind[i] != 0) {  // zero weight: no path (block-uniform)
            if (threadIdx.x == 0) {
                a.ilen[i] = 0;
                a.path_off[i] = 0;
            }
            continue;
        }
        const int32_t s = a.pair_s[i], t = a.pair_t[i];
        uint32_t ep;
        if constexpr (HASH) {
            if (ep_slot >= kHashEpochs) {
                // the slot's epochs are used up: clear every word of its tables (once per
                // 2^20 - 1 samples of the slot), then start again at 1
                for (int64_t e = threadIdx.x; e < a.region; e += BT) {
                    sent[4 * e] = 0ull;
                    sent[4 * e + 2] = 0ull;
                }
                __threadfence();
                __syncthreads();
                ep_slot = 0u;
            }
            ep = ++ep_slot;
        } else {
            ep = a.epoch_base + (uint32_t)i + 1u;
        }
        // the table in use: hashed, 2^lg entries at tab (offset toff in the slot);
        // direct, entry v - base of the sample's graph at tab + 4 v
        int lg = a.h0_log;
        int64_t toff = 0;
        unsigned long long *tab = sent;
        if constexpr (!HASH) {
            if (a.gid) tab = sent - 4 * a.vbase[a.gid[s]];
        }
        int64_t ps, pt;
        if constexpr (HASH) {
            // s and t are the sample's first entries: s at its home, t at its own
            // (the next entry, as linear probing gives, when the homes collide)
            ps = hash_home(s, lg);
            pt = hash_home(t, lg);
            if (pt == ps) pt = (pt + 1) & ((1 << lg) - 1);
        } else {
            ps = s;
            pt = t;
        }
        if (threadIdx.x == 0) {
            st_pair(&tab[4 * ps], W::make(s, ep, 0), count_bits(C(1)));
            st_pair(&tab[4 * pt + 2], W::make(t, ep, 0), count_bits(C(1)));
            queue0[0] = make_int2(s, (int)ps);
            queue1[0] = make_int2(t, (int)pt);
            s_new[0] = 0;
            s_newcost[0] = 0ull;
            s_meet = 0;
            s_full = 0;
            s_lv[0][0] = s_lv[1][0] = 0;
            s_lv[0][1] = s_lv[1][1] = 1;
        }
        __syncthreads();
        // level state of both sides, the same in every thread
        long long qlo[2] = {0, 0}, qhi[2] = {1, 1};
        uint32_t lev[2] = {0u, 0u};
        unsigned long long cost[2] = {(unsigned long long)(a.rp[s + 1] - a.rp[s]),
                                      (unsigned long long)(a.irp[t + 1] - a.irp[t])};
        int x = 0;
        bool met = s != t, handed = false;
        // expected hits that try a level for its meeting layer first (lower where the
        // filter makes a scan that finds no member cheap)
        double meet_hits = BT != kBiBlock ? kMeetOnlyHitsBloom : kMeetOnlyHits;
        int bloom_side = -1;                // the filter holds side bloom_side's first bloom_n vertices
        long long bloom_n = 0;
        if (met) {
            met = false;
            for (int it = 0;; ++it) {
                if (qhi[0] == qlo[0] || qhi[1] == qlo[1]) break;  // a side ran dry: t unreachable
                x = cost[0] <= cost[1] ? 0 : 1;
                const long long lo = x ? qlo[1] : qlo[0], hi = x ? qhi[1] : qhi[0];
                const uint32_t nl = (x ? lev[1] : lev[0]) + 1;
                if (lim && (x ? cost[1] : cost[0]) > lim) {
                    handed = true;  // a heavy level: the pass with larger blocks takes the sample
                    break;
                }
                if constexpr (HASH) {
                    if (nl > kHashLevels) {  // past the words' 12 bits: the direct store takes it
                        handed = true;
                        break;
                    }
                    // the coming level adds at most cost[x] entries: keep the table at most
                    // half full (the largest table is the limit; claims past 3/4 of it hand
                    // the sample over)
                    const unsigned long long need =
                        2ull * ((unsigned long long)(qhi[0] + qhi[1]) + (x ? cost[1] : cost[0])) + 2ull * BT;
                    int nlg = lg;
                    int64_t noff = toff;
                    while (nlg + 2 <= a.hmax_log && (1ull << nlg) < need) {
                        noff += 1ll << nlg;
                        nlg += 2;
                    }
                    if (nlg != lg) {
                        // move to the table of 2^nlg entries: re-insert every entry by
                        // walking the queues.  Side 0's queue first, claiming side-0 pairs
                        // only (and copying a side-1 pair of the same vertex with it); then,
                        // after a barrier, side 1's queue, whose vertices are either found
                        // (reached by side 0 too) or claim side-1 pairs.  Within each walk
                        // every claim is on the same pair of words, so two vertices never
                        // share an entry.
                        unsigned long long *ntab = sent + 4 * noff;
                        const uint32_t nmask = (1u << nlg) - 1u;
                        for (int z = 0; z < 2; ++z) {
                            int2 *qz = z ? queue1 : queue0;
                            const long long qn = z ? qhi[1] : qhi[0];
                            const int zs = z ? 2 : 0;
                            for (long long k = threadIdx.x; k < qn; k += BT) {
                                const int2 qe = qz[k];
                                unsigned long long o0, oc0, o1, oc1;
                                ld_pair(&tab[4ull * qe.y], o0, oc0);
                                ld_pair(&tab[4ull * qe.y + 2], o1, oc1);
                                const bool cur0 = W::current(o0, ep), cur1 = W::current(o1, ep);
                                uint32_t p = hash_home(qe.x, nlg);
                                for (uint32_t probes = 0; probes <= nmask;) {
                                    unsigned long long w0, c0, w1, c1;
                                    ld_pair(&ntab[4ull * p], w0, c0);
                                    ld_pair(&ntab[4ull * p + 2], w1, c1);
                                    const bool n0 = W::current(w0, ep), n1 = W::current(w1, ep);
                                    if (n0 || n1) {
                                        if (Word<true>::vertex(n0 ? w0 : w1) == qe.x) break;  // inserted
                                        p = (p + 1) & nmask;  // another vertex's entry
                                        ++probes;
                                        continue;
                                    }
                                    // an empty entry: claim it with this walk's pair (side 1 walk:
                                    // only vertices side 0 never reached get here)
                                    unsigned long long pw, pc;
                                    const unsigned long long ew = z ? w1 : w0, ec = z ? c1 : c0;
                                    cas_pair(&ntab[4ull * p + zs], ew, ec, z ? o1 : o0, z ? oc1 : oc0, pw, pc);
                                    if (pw == ew && pc == ec) {
                                        if (z == 0 && cur1) st_pair(&ntab[4ull * p + 2], o1, oc1);
                                        break;
                                    }
                                    // claimed meanwhile: look at the same entry again
                                }
                                (void)cur0;
                                qz[k].y = (int)p;
                            }
                            __syncthreads();
                        }
                        if (a.work && threadIdx.x == 0) s_work[5] += 1ull;
                        __syncthreads();
                        lg = nlg;
                        toff = noff;
                        tab = ntab;
                    }
                }
                const int cs = it % 3;
                // a large level's claims leave the degrees to a pass after it (lazy_deg)
                const bool lazy_deg = (x ? cost[1] : cost[0]) >= kLazyDegEdges;
                if (threadIdx.x == 0) {
                    s_new[(it + 1) % 3] = 0;
                    s_newcost[(it + 1) % 3] = 0ull;
                }
                const int64_t hmask = HASH ? (1ll << lg) - 1 : 0;
                // new entries stop short of 3/4 of the table (each thread has at most one
                // claim in flight past the check)
                const long long cap_new = HASH ? ((3ll << lg) >> 2) - BT : 0ll;
                const long long known = qhi[0] + qhi[1];
                unsigned long long ne = 0ull;
                // level nl: claim unreached neighbours and add the counts over
                // every edge into the level in one pass
                const int xs = x ? 2 : 0, ys = x ? 0 : 2;  // word offsets of the two sides in an entry
                int2 *qx = x ? queue1 : queue0;
                const int64_t *px = x ? a.irp : a.rp;
                const int32_t *ax = x ? a.icol : a.col;
                // one edge: claim the neighbour if unreached, add the parent's count if
                // it lies on the new level.  A claim swaps the whole {word, count} pair,
                // so it also sets the count to the claiming parent's and counts never
                // need clearing: a count is read only where its word carries the epoch.
                // one edge into v: what the claim or the count addition needs is loaded
                // first (prefetch), for several edges at once, then resolved
                struct Pre {
                    int32_t v;
                    int64_t p;
                    unsigned long long ow, oc, oy;
                };
                auto prefetch = [&](const int32_t v) -> Pre {
                    Pre r;
                    r.v = v;
                    r.p = HASH ? (int64_t)hash_home(v, lg) : (int64_t)v;
                    ld_pair(&tab[4 * r.p + xs], r.ow, r.oc);
                    r.oy = __ldcg(&tab[4 * r.p + ys]);
                    return r;
                };
                // claim v if unreached, add the parent's count if it lies on the new
                // level.  A claim swaps the whole {word, count} pair, so it also sets the
                // count to the claiming parent's and counts never need clearing: a count
                // is read only where its word carries the sample's epoch.
                auto resolve = [&](Pre &r, const C su, const bool checked, const bool meet_only) {
                    if (HASH && s_full) return;  // the sample goes to the direct store
                    const int32_t v = r.v;
                    const unsigned long long want = W::make(v, ep, nl);
                    int64_t p = r.p;
                    unsigned long long ow = r.ow, oc = r.oc, oy = r.oy;
                    bool at = false, won = false, meet = false;
                    for (int64_t probes = 0;;) {
                        const bool yc = W::current(oy, ep);
                        bool again = false;
                        if constexpr (HASH) {
                            const bool xc = W::current(ow, ep);
                            if ((xc || yc) && Word<true>::vertex(xc ? ow : oy) != v) {
                                p = (p + 1) & hmask;  // another vertex's entry
                                if (++probes > hmask) {
                                    s_full = 1;
                                    break;
                                }
                                again = true;
                            } else if (!xc && !yc && !meet_only && known + s_new[cs] >= cap_new) {  // would overfill
                                s_full = 1;
                                break;
                            }
                        }
                        if (!again) {
                            if (W::current(ow, ep)) {
                                at = ow == want;
                                break;
                            }
                            if (meet_only && !yc) break;  // not in the meeting layer: left to a full pass
                            unsigned long long pw, pc;
                            cas_pair(&tab[4 * p + xs], ow, oc, want, count_bits(su), pw, pc);
                            if (pw == ow && pc == oc) {
                                won = true;
                                meet = yc;
                                break;
                            }
                        }
                        // another entry, or this one claimed meanwhile: (re)read it
                        ld_pair(&tab[4 * p + xs], ow, oc);
                        oy = __ldcg(&tab[4 * p + ys]);
                    }
                    if (won) {
                        // the lanes that claimed together reserve their queue slots and
                        // add their degrees with one shared atomic each (a 64-bit shared
                        // add would be a contended compare-and-swap loop per lane); the
                        // degree is loaded by the claim's winner alone, and in a large
                        // level not at all (lazy_deg)
                        const uint32_t dg = lazy_deg ? 0u : (uint32_t)(px[v + 1] - px[v]);  // < 2^31
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
                        qx[hi + q0 + __popc(grp & ((1u << lane) - 1u))] = make_int2(v, (int)p);
                        if (meet) {  // a member of the meeting layer: listed for the meeting step
                            const unsigned mg = __activemask();
                            const int ml = __ffs(mg) - 1;
                            int m0 = 0;
                            if (lane == ml) m0 = atomicAdd(&s_meet, __popc(mg));
                            m0 = __shfl_sync(mg, m0, ml);
                            memb[m0 + __popc(mg & ((1u << lane) - 1u))] = make_int2(v, (int)p);
                        }
                    }
                    if (a.work && (at || won)) ++n_add;
                    if (at) {
                        C *cp = reinterpret_cast<C *>(&tab[4 * p + xs + 1]);
                        if (checked) {  // counts may pass 2^53: find the addition that does
                            const C o = atomicAdd(cp, su);
                            if ((double)(o + su) >= kTwo53) atomicOr(a.status, DEV_SIGMA_OVERFLOW);
                        } else {
                            atomicAdd(cp, su);  // (no result waited for)
                        }
                    }
                };
                constexpr int EB = BT == kBiBlock ? kEdgeBatch : kHeavyEdgeBatch;
                // A level likely to meet the other side (the edges it scans times the
                // vertices the other side holds reach kMeetOnlyHits n) is first scanned for
                // the meeting layer alone: only vertices the other side holds are claimed,
                // which is all a level that meets needs (nothing reads its other
                // vertices).  If it holds none the level is scanned again in full.
                bool meet_only = a.gid == nullptr &&
                                 (double)(x ? cost[1] : cost[0]) * (double)(x ? qhi[0] : qhi[1]) >=
                                     meet_hits * (double)a.n;
                if (BLOOM && meet_only) {
                    // the other side's vertices into the filter (it only grows: a side's
                    // queue lists every vertex it reached, in order)
                    const int y = 1 - x;
                    const long long ny = y ? qhi[1] : qhi[0];
                    if (bloom_side != y || bloom_n != ny) {
                        const long long from = bloom_side == y ? bloom_n : 0;
                        if (from == 0) {
                            for (int w = threadIdx.x; w < NBW; w += BT) s_bloom[w] = 0u;
                            __syncthreads();
                        }
                        const int2 *qy = y ? queue1 : queue0;
                        for (long long q = from + threadIdx.x; q < ny; q += BT) {
                            uint32_t h1, h2;
                            bloom_bits(qy[q].x, h1, h2);
                            atomicOr(&s_bloom[h1 >> 5], 1u << (h1 & 31));
                            atomicOr(&s_bloom[h2 >> 5], 1u << (h2 & 31));
                        }
                        __syncthreads();
                        bloom_side = y;
                        bloom_n = ny;
                    }
                }
                for (;;) {
                    // every count of the new level is at most the sum of the frontier's
                    // counts loaded so far (fcnt, FP64): below 2^52 no count can reach 2^53,
                    // so the count additions need not wait for their results
                    double fcnt = 0.0;
                    // the level's edges spread evenly over the block, kFlat frontier vertices
                    // at a time (a hub's adjacency is not left to one warp): the block loads
                    // the chunk, a few vertices per thread with their loads in flight
                    // together, and writes its degree prefix sums to shared memory; each
                    // edge then finds its vertex by bisection
                    for (long long c0 = lo; c0 < hi; c0 += kFlat) {
                        const int fc = (int)(hi - c0 < kFlat ? hi - c0 : kFlat);
                        {
                            constexpr int per = kFlat >= BT ? kFlat / BT : 1;
                            int64_t loc[per];
                            int64_t tot = 0;
                            double csum = 0.0;  // the chunk's path counts
    #pragma unroll
                            for (int r = 0; r < per; ++r) {
                                const int k = (int)threadIdx.x * per + r;
                                int64_t dg = 0;
                                if (k < fc) {
                                    const int2 qe = qx[c0 + k];
                                    const int64_t e0 = px[qe.x];
                                    s_fe[k] = e0;
                                    const C fs = count_of<C>(__ldcg(&tab[4ll * qe.y + xs + 1]));
                                    s_fs[k] = fs;
                                    csum += (double)fs;
                                    dg = px[qe.x + 1] - e0;
                                }
                                loc[r] = tot;
                                tot += dg;
                            }
                            int64_t incl = tot;
    #pragma unroll
                            for (int o = 1; o < 32; o <<= 1) {
                                const int64_t t2 = __shfl_up_sync(0xffffffffu, incl, o);
                                if (lane >= o) incl += t2;
                            }
                            if (lane == 31) s_wsum[warp] = incl;
    #pragma unroll
                            for (int o = 16; o > 0; o >>= 1) csum += __shfl_xor_sync(0xffffffffu, csum, o);
                            if (lane == 0) s_wcnt[warp] = csum;
                            __syncthreads();
                            int64_t first = incl - tot;
                            for (int q = 0; q < warp; ++q) first += s_wsum[q];
                            for (int q = 0; q < nw; ++q) fcnt += s_wcnt[q];
    #pragma unroll
                            for (int r = 0; r < per; ++r) {
                                const int k = (int)threadIdx.x * per + r;
                                if (k < fc) s_pre[k] = first + loc[r];
                            }
                            if (threadIdx.x == BT - 1) s_pre[fc] = first + tot;  // (vertices past fc add 0)
                        }
                        __syncthreads();
                        const int64_t E = s_pre[fc];
                        if (threadIdx.x == 0) ne += (unsigned long long)E;
                        auto vertex_of = [&](int64_t j) -> int {  // last k with s_pre[k] <= j
                            int klo = 0, khi = fc - 1;
                            while (klo < khi) {
                                const int mid = (klo + khi + 1) >> 1;
                                if (s_pre[mid] <= j) klo = mid;
                                else khi = mid - 1;
                            }
                            return klo;
                        };
                        if (BLOOM && meet_only) {
                            // a meeting scan with the filter: each thread takes a contiguous
                            // range of the chunk's edges (one bisection), loads eight columns
                            // at a time and tests them; only the members are claimed
                            const int64_t per_t = (E + BT - 1) / BT;
                            int64_t jb = (int64_t)threadIdx.x * per_t;
                            const int64_t je = jb + per_t < E ? jb + per_t : E;
                            int k = jb < je ? vertex_of(jb) : 0;
                            for (; jb < je; jb += kMeetBatch) {
                                int kk[kMeetBatch];
                                int32_t vv[kMeetBatch];
    #pragma unroll
                                for (int b = 0; b < kMeetBatch; ++b) {
                                    const int64_t e = jb + b;
                                    vv[b] = -1;
                                    kk[b] = k;
                                    if (e < je) {
                                        while (s_pre[k + 1] <= e) ++k;  // (s_pre[fc] = E > e)
                                        kk[b] = k;
                                        vv[b] = ax[s_fe[k] + (e - s_pre[k])];
                                    }
                                }
    #pragma unroll
                                for (int b = 0; b < kMeetBatch; ++b) {
                                    if (vv[b] < 0) continue;
                                    uint32_t h1, h2;
                                    bloom_bits(vv[b], h1, h2);
                                    if (!((s_bloom[h1 >> 5] >> (h1 & 31)) & (s_bloom[h2 >> 5] >> (h2 & 31)) & 1u))
                                        vv[b] = -1;  // not a member of the other side
                                }
    #pragma unroll
                                for (int b = 0; b < kMeetBatch; ++b) {
                                    if (vv[b] < 0) continue;
                                    Pre pr = prefetch(vv[b]);
                                    resolve(pr, s_fs[kk[b]], fcnt >= 0x1p52, true);
                                }
                            }
                        } else {
                            for (int64_t j = threadIdx.x; j < E; j += (int64_t)EB * BT) {
                                Pre pr[EB];
                                int kk[EB];
                                int32_t vv[EB];
    #pragma unroll
                                for (int b = 0; b < EB; ++b) {
                                    const int64_t jb = j + (int64_t)b * BT;
                                    kk[b] = jb < E ? vertex_of(jb) : 0;
                                    vv[b] = jb < E ? ax[s_fe[kk[b]] + (jb - s_pre[kk[b]])] : -1;
                                }
    #pragma unroll
                                for (int b = 0; b < EB; ++b)
                                    if (vv[b] >= 0) pr[b] = prefetch(vv[b]);
    #pragma unroll
                                for (int b = 0; b < EB; ++b)
                                    if (vv[b] >= 0) resolve(pr[b], s_fs[kk[b]], fcnt >= 0x1p52, meet_only);
                            }
                        }
                        if (c0 + kFlat < hi) __syncthreads();  // the chunk's shared arrays are reused
                    }
                    if (!meet_only) break;
                    __syncthreads();
                    if (s_meet || (HASH && s_full)) break;  // (the same in every thread after the barrier)
                    meet_only = false;  // no member: the level in full (nothing was claimed)
                    meet_hits *= 8.0;   // (targets are not uniform: on grids the balls meet late)
                    __syncthreads();    // the chunk's shared arrays are reloaded
                }
                if (a.work && ne) atomicAdd(&s_work[0], ne);
                smp_edges += ne;
                ++smp_levels;
                __syncthreads();
                if (HASH && s_full) {  // (the same in every thread after the barrier)
                    handed = true;
                    break;
                }
                const long long nh = hi + s_new[cs];
                unsigned long long nc = s_newcost[cs];
                if (lazy_deg && !s_meet) {
                    // the new level's degrees, which the claims of this large level did not
                    // load: most such levels end the search, and then nothing reads them
                    long long part = 0;
                    for (long long q = hi + threadIdx.x; q < nh; q += BT) {
                        const int32_t v = qx[q].x;
                        part += px[v + 1] - px[v];
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                    if (lane == 0) s_wsum[warp] = part;
                    __syncthreads();
                    long long tot = 0;
                    for (int q = 0; q < nw; ++q) tot += s_wsum[q];
                    nc = (unsigned long long)tot;
                    __syncthreads();  // s_wsum is reused by the next level's chunks
                }
                if (threadIdx.x == 0 && nl + 1 <= (uint32_t)kLvCap) s_lv[x][nl + 1] = (int32_t)nh;
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
        if (a.trace && threadIdx.x == 0) t_levels = globaltimer_ns();
        if (handed) {
            // nothing of the sample was written outside the slot: the heavy pass runs it
            if (threadIdx.x == 0) {
                const unsigned int d = atomicAdd(a.n_deferred, 1u);
                a.deferred[d] = (int32_t)i;
                a.defer_cost[d] = x ? cost[1] : cost[0];
                if (a.work) s_work[4] += 1ull;
            }
            continue;
        }

        if (!met) {
            if (threadIdx.x == 0) {
                a.kind[i] = 2;
                a.ilen[i] = 0;
                a.path_off[i] = 0;
            }
        } else {
            // meeting layer: the members of the last level of side x (vertices the
            // other side holds), listed as they were claimed; weights sigma_s sigma_t,
            // kept in shared memory when they fit
            const int nm = s_meet;
            auto weight = [&](const int2 qe) -> C {
                return count_of<C>(__ldcg(&tab[4ll * qe.y + 1])) * count_of<C>(__ldcg(&tab[4ll * qe.y + 3]));
            };
            C part = C(0);
            for (int m = threadIdx.x; m < nm; m += BT) {
                const int2 qe = memb[m];
                const C a0 = count_of<C>(__ldcg(&tab[4ll * qe.y + 1]));
                const C a1 = count_of<C>(__ldcg(&tab[4ll * qe.y + 3]));
                const C p = a0 * a1;
                if ((double)a0 * (double)a1 >= kTwo53) atomicOr(a.status, DEV_SIGMA_OVERFLOW);
                part += p;
                if (m < kMeetCap) {
                    s_mv[m] = qe.x;
                    s_mp[m] = qe.y;
                    s_mw[m] = p;
                }
            }
            const C sst = block_sum<BT>(part, s_redc);
            if (threadIdx.x == 0 && (double)sst >= kTwo53) atomicOr(a.status, DEV_SIGMA_OVERFLOW);
            const double target = __dmul_rn(uniform_at(a.seed, (uint64_t)i, a.tag, 0), (double)sst);
            if (a.work && threadIdx.x == 0 && nm > kMeetCap) s_work[3] += 1ull << 32;  // large layers (high word)
            int32_t vm;
            int64_t pm;
            if (nm <= kMeetCap) {
                // member j qualifies when the weights of the members with ids <= its
                // own reach the target; the meeting vertex is the smallest such id
                unsigned long long best = ~0ull;  // vertex << 32 | entry
                for (int j = threadIdx.x; j < nm; j += BT) {
                    const int32_t vj = s_mv[j];
                    C pre = C(0);
                    for (int k2 = 0; k2 < nm; ++k2)
                        if (s_mv[k2] <= vj) pre += s_mw[k2];
                    if ((double)pre >= target)
                        best = min(best, ((unsigned long long)(uint32_t)vj << 32) | (uint32_t)s_mp[j]);
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, off));
                __syncthreads();
                if (lane == 0) s_best[warp] = best;
                __syncthreads();
                unsigned long long bk = s_best[0];
                for (int q = 1; q < nw; ++q) bk = min(bk, s_best[q]);
                if (bk == ~0ull) {  // (FP64 counts) no member reaches the target: the last one takes it
                    unsigned long long lk = 0ull;
                    for (int j = 0; j < nm; ++j)
                        lk = max(lk, ((unsigned long long)(uint32_t)s_mv[j] << 32) | (uint32_t)s_mp[j]);
                    bk = lk;
                }
                vm = (int32_t)(bk >> 32);
                pm = (int64_t)(uint32_t)bk;
            } else {
                // a large layer: the first id whose prefix sum (members in id order)
                // reaches the target, narrowed in rounds of kMeetBuckets id buckets: the
                // members' weights are summed per bucket in shared memory, the first
                // bucket whose running total reaches the target holds the answer, and
                // the next round splits that bucket (exact integer sums, so the same id
                // as a sequential scan; three rounds for 2^30 ids)
                int64_t lo_id = 0, span = n;
                C base = C(0);  // weight of the members below lo_id
                while (span > 1) {
                    const int64_t wb = (span + kMeetBuckets - 1) / kMeetBuckets;
                    for (int b = threadIdx.x; b < kMeetBuckets; b += BT) s_bkt[b] = C(0);
                    __syncthreads();
                    for (int m = threadIdx.x; m < nm; m += BT) {
                        const int2 qe = memb[m];
                        if (qe.x >= lo_id && qe.x < lo_id + span) atomicAdd(&s_bkt[(qe.x - lo_id) / wb], weight(qe));
                    }
                    __syncthreads();
                    if (warp == 0) {
                        constexpr int per = kMeetBuckets / 32;
                        C lsum = C(0);
                        for (int j = 0; j < per; ++j) lsum += s_bkt[lane * per + j];
                        C incl = lsum;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const C t2 = __shfl_up_sync(0xffffffffu, incl, o);
                            if (lane >= o) incl += t2;
                        }
                        const unsigned hit = __ballot_sync(0xffffffffu, (double)(base + incl) >= target);
                        const unsigned nz = __ballot_sync(0xffffffffu, lsum > C(0));
                        // FP64 counts past 2^53 may leave every total just below the target:
                        // the last bucket with weight then takes the remainder
                        const int L0 = hit ? __ffs(hit) - 1 : (nz ? 31 - __clz(nz) : 0);
                        if (lane == L0) {  // the bucket within this lane's range, and the total below it
                            C run = base + (incl - lsum), below = run;
                            int bsel = 0;
                            for (int j = 0; j < per; ++j) {
                                const C bw = s_bkt[L0 * per + j];
                                if (bw == C(0)) continue;
                                bsel = j;
                                below = run;
                                run += bw;
                                if (hit && (double)run >= target) break;
                            }
                            s_sel = L0 * per + bsel;
                            s_base = below;
                        }
                    }
                    __syncthreads();
                    const int64_t nlo = lo_id + (int64_t)s_sel * wb;
                    span = min(wb, lo_id + span - nlo);
                    lo_id = nlo;
                    base = s_base;
                    __syncthreads();
                }
                vm = (int32_t)lo_id;
                if constexpr (HASH) pm = hash_find(tab, lg, vm, ep);
                else pm = vm;
            }
            if (a.trace && threadIdx.x == 0) t_meet = globaltimer_ns();
            // the path: the meeting vertex, then the s side backtracked from it, then
            // the t side.  A backtrack step scans the candidates (in-neighbours towards
            // s, out-neighbours towards t) in adjacency order for the first one one level
            // closer whose running count reaches u sigma(w): one warp for short lists; the
            // whole block for long ones (hubs), in two passes -- every thread sums a
            // contiguous segment, a block scan of the sums finds the segment where the
            // running count reaches the target, one warp scans that segment.
            {
                const uint32_t la = W::level(__ldcg(&tab[4 * pm]));
                const uint32_t lb = W::level(__ldcg(&tab[4 * pm + 2]));
                const int32_t len = (int32_t)(la + lb) - 1;
                if (threadIdx.x == 0) {
                    const unsigned long long o = atomicAdd(a.arena_top, (unsigned long long)len);
                    if ((int64_t)(o + len) > a.arena_cap) atomicOr(a.status, DEV_ARENA_OVERFLOW);
                    a.ilen[i] = len;
                    a.path_off[i] = (long long)o;
                    s_off = o;
                    if (vm != s && vm != t) {
                        if ((int64_t)(o + len) <= a.arena_cap) a.arena[o] = vm;
                        atomicAdd(&a.cnt[vm], 1ull);
                    }
                }
                __syncthreads();
                const unsigned long long off = s_off;
                const bool store = (int64_t)(off + len) <= a.arena_cap;
                int32_t k = (vm != s && vm != t) ? 1 : 0;
                uint32_t step = 1;
                for (int z = 0; z < 2; ++z) {
                    // towards s: predecessors over in-edges; towards t: successors over out-edges
                    const int64_t *bp = z == 0 ? a.irp : a.rp;
                    const int32_t *bc = z == 0 ? a.icol : a.col;
                    const int zs = z ? 2 : 0;
                    const int32_t endz = z == 0 ? s : t;
                    int32_t w = vm;
                    int64_t pw = pm;
                    bool bad = false;
                    while (w != endz) {  // (the same in every thread)
                        const uint32_t lw = W::level(__ldcg(&tab[4 * pw + zs]));
                        const double tg = __dmul_rn(uniform_at(a.seed, (uint64_t)i, a.tag, step),
                                                    (double)count_of<C>(__ldcg(&tab[4 * pw + zs + 1])));
                        const int64_t e0 = bp[w], e1 = bp[w + 1];
                        // the count of candidate e if it lies one level closer, else 0
                        auto cand = [&](int64_t e, int32_t &pv, int64_t &pp) -> C {
                            pv = bc[e];
                            if constexpr (HASH) pp = hash_find(tab, lg, pv, ep);
                            else pp = pv;
                            if (pp < 0) return C(0);
                            unsigned long long lw2, lc2;
                            ld_pair(&tab[4 * pp + zs], lw2, lc2);
                            return (W::current(lw2, ep) && W::level(lw2) + 1 == lw) ? count_of<C>(lc2) : C(0);
                        };
                        // one warp scans [b0, b1) from running count c0: first lane whose running
                        // count reaches tg, else (FP64 counts) the last candidate
                        auto warp_scan = [&](int64_t b0, int64_t b1, C c0) {
                            C carry = c0;
                            int32_t pick = -1, last = -1;
                            int64_t pickp = -1, lastp = -1;
                            for (int64_t eb = b0; eb < b1 && pick < 0; eb += 32) {
                                const int64_t e = eb + lane;
                                int32_t pv = -1;
                                int64_t pp = -1;
                                const C val = e < b1 ? cand(e, pv, pp) : C(0);
                                C cum = val;
#pragma unroll
                                for (int o = 1; o < 32; o <<= 1) {
                                    const C t2 = __shfl_up_sync(0xffffffffu, cum, o);
                                    if (lane >= o) cum += t2;
                                }
                                cum += carry;
                                const unsigned hit = __ballot_sync(0xffffffffu, val > C(0) && (double)cum >= tg);
                                if (hit) {
                                    pick = __shfl_sync(0xffffffffu, pv, __ffs(hit) - 1);
                                    pickp = __shfl_sync(0xffffffffu, pp, __ffs(hit) - 1);
                                }
                                const unsigned cm = __ballot_sync(0xffffffffu, val > C(0));
                                if (cm) {
                                    last = __shfl_sync(0xffffffffu, pv, 31 - __clz(cm));
                                    lastp = __shfl_sync(0xffffffffu, pp, 31 - __clz(cm));
                                }
                                carry = __shfl_sync(0xffffffffu, cum, 31);
                            }
                            // FP64 counts past 2^53 may round the running sum just below u sigma(w):
                            // the last candidate then takes the remainder
                            if (pick < 0 && FP) {
                                pick = last;
                                pickp = lastp;
                            }
                            if (lane == 0) {
                                s_pick = pick;
                                s_pickp = pickp;
                            }
                        };
                        // the previous level of side z, when its queue range is kept
                        const uint32_t Lp = lw - 1;
                        const long long lq0 = Lp + 1 <= (uint32_t)kLvCap ? s_lv[z][Lp] : 0;
                        const long long lq1 = Lp + 1 <= (uint32_t)kLvCap ? s_lv[z][Lp + 1] : 0;
                        if (e1 - e0 <= kBackWarp) {
                            if (warp == 0) warp_scan(e0, e1, C(0));
                        } else if (a.sorted && Lp + 1 <= (uint32_t)kLvCap && lq1 - lq0 <= kMeetCap) {
                            // a long list and a small previous level: the candidates are that
                            // level's vertices found in w's (sorted) list by bisection, their
                            // places in it give the scan order; the choice is the first, in
                            // that order, whose running count reaches the target
                            const int2 *qz = z ? queue1 : queue0;
                            if (threadIdx.x == 0) s_nc = 0;
                            __syncthreads();
                            for (long long q = lq0 + threadIdx.x; q < lq1; q += BT) {
                                const int2 qe = qz[q];
                                int64_t blo = e0, bhi = e1;
                                while (blo < bhi) {
                                    const int64_t mid = blo + ((bhi - blo) >> 1);
                                    if (bc[mid] < qe.x) blo = mid + 1;
                                    else bhi = mid;
                                }
                                if (blo < e1 && bc[blo] == qe.x) {
                                    const int c = atomicAdd(&s_nc, 1);
                                    s_mv[c] = qe.x;
                                    s_mp[c] = qe.y;
                                    s_mw[c] = count_of<C>(__ldcg(&tab[4ll * qe.y + zs + 1]));
                                    s_mj[c] = (int32_t)(blo - e0);
                                }
                            }
                            __syncthreads();
                            const int nc = s_nc;
                            unsigned long long best = ~0ull, lastc = 0ull;  // place << 32 | candidate
                            for (int c = threadIdx.x; c < nc; c += BT) {
                                const int32_t jc = s_mj[c];
                                C pre = C(0);
                                for (int c2 = 0; c2 < nc; ++c2)
                                    if (s_mj[c2] <= jc) pre += s_mw[c2];
                                const unsigned long long key = ((unsigned long long)(uint32_t)jc << 32) | (uint32_t)c;
                                if (s_mw[c] > C(0)) {
                                    if ((double)pre >= tg) best = min(best, key);
                                    lastc = max(lastc, key + 1ull);
                                }
                            }
#pragma unroll
                            for (int o = 16; o > 0; o >>= 1) {
                                best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
                                lastc = max(lastc, __shfl_xor_sync(0xffffffffu, lastc, o));
                            }
                            if (lane == 0) {
                                s_best[warp] = best;
                                s_redc[warp] = C(0);
                            }
                            __syncthreads();
                            unsigned long long bk = s_best[0];
                            for (int q = 1; q < nw; ++q) bk = min(bk, s_best[q]);
                            __syncthreads();
                            if (lane == 0) s_best[warp] = lastc;
                            __syncthreads();
                            if (threadIdx.x == 0) {
                                // FP64 counts past 2^53 may round the running sum just below u
                                // sigma(w): the last candidate then takes the remainder
                                if (bk == ~0ull && FP) {
                                    unsigned long long lk = 0ull;
                                    for (int q = 0; q < nw; ++q) lk = max(lk, s_best[q]);
                                    bk = lk ? lk - 1ull : ~0ull;
                                }
                                const int c = bk == ~0ull ? -1 : (int)(uint32_t)bk;
                                s_pick = c < 0 ? -1 : s_mv[c];
                                s_pickp = c < 0 ? -1 : s_mp[c];
                            }
                        } else {
                            const int64_t seg = (e1 - e0 + BT - 1) / BT;
                            const int64_t sb = min(e1, e0 + (int64_t)threadIdx.x * seg), se = min(e1, sb + seg);
                            C my = C(0);
                            int64_t e = sb;
                            for (; e + 4 <= se; e += 4) {  // four candidates in flight
                                int32_t pv[4];
                                int64_t pp[4];
                                C v[4];
#pragma unroll
                                for (int u = 0; u < 4; ++u) v[u] = cand(e + u, pv[u], pp[u]);
                                my += (v[0] + v[1]) + (v[2] + v[3]);
                            }
                            for (; e < se; ++e) {
                                int32_t pv;
                                int64_t pp;
                                my += cand(e, pv, pp);
                            }
                            // exclusive block scan of the segment sums
                            C inc = my;
#pragma unroll
                            for (int o = 1; o < 32; o <<= 1) {
                                const C t2 = __shfl_up_sync(0xffffffffu, inc, o);
                                if (lane >= o) inc += t2;
                            }
                            if (threadIdx.x == 0) s_tstar = 0x7fffffff;
                            if (lane == 31) s_redc[warp] = inc;
                            __syncthreads();
                            C pre = inc - my;
                            for (int q = 0; q < warp; ++q) pre += s_redc[q];
                            const bool reach = my > C(0) && (double)(pre + my) >= tg;
                            const unsigned rb = __ballot_sync(0xffffffffu, reach);
                            if (rb && lane == __ffs(rb) - 1) atomicMin(&s_tstar, (int)threadIdx.x);
                            __syncthreads();
                            int ts = s_tstar;
                            if (ts == 0x7fffffff) {  // FP64 counts: the last segment with a candidate
                                const unsigned nzb = __ballot_sync(0xffffffffu, my > C(0));
                                if (nzb && lane == 31 - __clz(nzb)) atomicMax(&s_tlast, (int)threadIdx.x);
                                __syncthreads();
                                ts = s_tlast;
                            }
                            if ((int)threadIdx.x == ts) s_tpre = pre;
                            __syncthreads();
                            if (warp == 0) {
                                if (ts >= 0 && ts < BT) {  // (no segment with a candidate: no choice)
                                    const int64_t tb = min(e1, e0 + (int64_t)ts * seg);
                                    warp_scan(tb, min(e1, tb + seg), s_tpre);
                                } else if (lane == 0) {
                                    s_pick = -1;
                                    s_pickp = -1;
                                }
                            }
                            if (threadIdx.x == 0) s_tlast = -1;
                        }
                        __syncthreads();
                        const int32_t pick = s_pick;
                        const int64_t pickp = s_pickp;
                        __syncthreads();  // s_pick is written again by the next step
                        if (pick < 0) {
                            if (threadIdx.x == 0) {
                                atomicOr(a.status, DEV_BAD_PATH);
                                if (a.trace) {  // where the path ended without a candidate
                                    a.trace[8 * i + 6] = (e1 - e0 <= BT ? 1ull : 2ull) | ((unsigned long long)z << 4) |
                                                         ((unsigned long long)step << 8) |
                                                         ((unsigned long long)(e1 - e0) << 32);
                                    a.trace[8 * i + 7] = ((unsigned long long)(uint32_t)w << 32) | lw;
                                }
                            }
                            bad = true;
                            break;
                        }
                        if (pick != endz) {
                            if (threadIdx.x == 0) {
                                if (store && k < len) a.arena[off + k] = pick;
                                atomicAdd(&a.cnt[pick], 1ull);
                            }
                            ++k;
                        }
                        w = pick;
                        pw = pickp;
                        ++step;
                    }
                    if (bad) break;
                }
            }
        }
        __syncthreads();
        if (a.work && threadIdx.x == 0) {
            s_work[2] += (unsigned long long)(qhi[0] + qhi[1]);
            s_work[3] += 1ull;
        }
        if (a.trace && threadIdx.x == 0) {
            unsigned long long *tr = a.trace + 8 * i;
            tr[0] = t_start;
            tr[1] = globaltimer_ns();
            tr[2] = smp_edges;
            tr[3] = (unsigned long long)smp_levels | ((unsigned long long)(HASH ? 0 : 1) << 32) |
                    ((unsigned long long)slot << 33) | ((unsigned long long)(BT != kBiBlock) << 63);
            tr[4] = t_levels;
            tr[5] = t_meet ? t_meet : t_levels;
        }
    }
    if (HASH && threadIdx.x == 0) a.slot_epoch[slot] = ep_slot;
    if (a.work) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) n_add += __shfl_xor_sync(0xffffffffu, n_add, off);
        if (lane == 0 && n_add) atomicAdd(&s_work[1], n_add);
    }
    __syncthreads();
    if (a.work && threadIdx.x < 6 && s_work[threadIdx.x]) atomicAdd(&a.work[threadIdx.x], s_work[threadIdx.x]);
}

constexpr int kHeavySort = 4096;  // heavy samples ordered by cost when there are at most this many

// The handed-over samples in decreasing cost, ties by sample number: one block,
// a bitonic sort of (~cost, sample) keys in shared memory.
__global__ void __launch_bounds__(1024) k_order_heavy(int32_t *defer, const unsigned long long *cost,
                                                      const unsigned int *n_def) {
    __shared__ unsigned long long s_k[kHeavySort];
    const int nd = (int)*n_def;
    if (nd <= 1 || nd > kHeavySort) return;  // (more: taken in the order they came)
    int P = 1;
    while (P < nd) P <<= 1;
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
        if (j < nd) {
            const unsigned long long c = cost[j] < 0xffffffffull ? cost[j] : 0xffffffffull;
            s_k[j] = ((0xffffffffull - c) << 32) | (uint32_t)defer[j];
        } else {
            s_k[j] = ~0ull;
        }
    }
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int t = threadIdx.x; t < P; t += blockDim.x) {
                const int u = t ^ j;
                if (u > t) {
                    const unsigned long long A = s_k[t], B = s_k[u];
                    if ((A > B) == ((t & k) == 0)) {
                        s_k[t] = B;
                        s_k[u] = A;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int j = threadIdx.x; j < nd; j += blockDim.x) defer[j] = (int32_t)(uint32_t)s_k[j];
}

#ifndef PERCIS_HEAVY_BLOCK
#define PERCIS_HEAVY_BLOCK 1024
#endif
constexpr int kHeavyBlock = PERCIS_HEAVY_BLOCK;  // threads per sample in the heavy pass
constexpr unsigned long long kDefaultHeavyEdges = 16384;  // a level scanning more edges is heavy
constexpr int64_t kDefaultScratchGiB = 48;  // direct store: one heavy-pass block per SM up to n = 6M

template <bool HASH, int BT>
int blocks_per_sm(int *cache) {
    if (!*cache) {
        int per_sm = 0;
        const int dyn = (int)(sizeof(uint32_t) * (BT == kBiBlock ? kBloomWordsFirst : kBloomWords));
        if (dyn > 48 * 1024)
            cudaFuncSetAttribute(k_bibfs<unsigned long long, HASH, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 dyn);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bibfs<unsigned long long, HASH, BT>, BT, dyn) !=
                cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        *cache = per_sm;
    }
    return *cache;
}

template <bool HASH, int BT>
void launch(percis_ctx *ctx, int grid, const BiArgs &a) {
    // the heavy pass's Bloom filter (dynamic shared memory)
    const int dyn = (int)(sizeof(uint32_t) * (BT == kBiBlock ? kBloomWordsFirst : kBloomWords));
    if (dyn > 48 * 1024) {
        cudaFuncSetAttribute(k_bibfs<double, HASH, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
        cudaFuncSetAttribute(k_bibfs<unsigned long long, HASH, BT>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
    }
    if (ctx->sigma_mode == 2) k_bibfs<double, HASH, BT><<<grid, BT, dyn, ctx->stream>>>(a);
    else k_bibfs<unsigned long long, HASH, BT><<<grid, BT, dyn, ctx->stream>>>(a);
}

BiArgs common_args(percis_ctx *ctx, uint64_t seed, uint32_t tag_path) {
    BiArgs a{};
    a.n = ctx->n;
    a.rp = ctx->rp.as<int64_t>();
    a.col = ctx->col.as<int32_t>();
    a.irp = ctx->directed ? ctx->irp.as<int64_t>() : ctx->rp.as<int64_t>();
    a.icol = ctx->directed ? ctx->icol.as<int32_t>() : ctx->col.as<int32_t>();
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
    a.status = &ctx->ms_ctl.as<MsCtl>()->status;
    a.work = ctx->opt.instrument ? ctx->counters.as<unsigned long long>() : nullptr;
    a.trace = ctx->opt.instrument >= 2 ? ctx->bi_trace.as<unsigned long long>() : nullptr;
    a.sorted = ctx->rows_sorted ? 1 : 0;
    a.max_degree = ctx->graph_info.as<unsigned long long>();
    return a;
}

// The direct store over `count` samples (all of the phase, or the list), BT
// threads per sample; samples with a level above heavy_edges are listed in
// defer (heavy_edges = 0: none).
template <int BT>
percis_status direct_pass(percis_ctx *ctx, uint64_t seed, uint32_t tag_path, int64_t count, const int32_t *list,
                          unsigned long long heavy_edges, int32_t heavy_auto, int32_t *defer,
                          unsigned long long *defer_cost, unsigned int *n_def, const unsigned int *count_dev = nullptr) {
    const int32_t *gid = nullptr;
    const int64_t *vbase = nullptr;
    int64_t nslot = ctx->n;
    if (ctx->multi) multi_graph_view(ctx, &gid, &vbase, &nslot);
    const size_t per_slot = (size_t)nslot * (sizeof(unsigned long long) * 4 + sizeof(int2) * 3);
    int per_sm = blocks_per_sm<false, BT>(BT == kBiBlock ? &ctx->bi_per_sm : &ctx->bi_heavy_per_sm);
    if (BT == kBiBlock && ctx->opt.bi_blocks_per_sm > 0) per_sm = std::min(per_sm, ctx->opt.bi_blocks_per_sm);
    const int64_t budget = (int64_t)(ctx->opt.bi_scratch_gib > 0 ? ctx->opt.bi_scratch_gib : kDefaultScratchGiB) << 30;
    int64_t slots = std::min<int64_t>((int64_t)per_sm * ctx->num_sms, std::max<int64_t>(1, budget / (int64_t)per_slot));
    slots = std::min<int64_t>(slots, std::max<int64_t>(count, 1));  // (count: at most that many with count_dev)
    if (ctx->bi_slots < slots || ctx->bi_n != nslot) {
        PERCIS_TRY(ensure(ctx, ctx->bi_info, sizeof(unsigned long long) * 4 * nslot * slots, "bidirectional records"));
        PERCIS_TRY(ensure(ctx, ctx->bi_queue, sizeof(int2) * 3 * nslot * slots, "bidirectional queues"));
        // level words of no sample (epoch 0)
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->bi_info.p, 0, sizeof(unsigned long long) * 4 * nslot * slots, ctx->stream));
        ctx->bi_slots = slots;
        ctx->bi_n = nslot;
        ctx->bi_epoch = 0;
    }
    const int64_t span = ctx->phase_span;  // epochs are indexed by sample number
    if ((uint64_t)ctx->bi_epoch + (uint64_t)span + 2 > 0xffffffffull) {
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->bi_info.p, 0, sizeof(unsigned long long) * 4 * nslot * ctx->bi_slots,
                                         ctx->stream));
        ctx->bi_epoch = 0;
    }
    PERCIS_TRY(ensure(ctx, ctx->red, 64, "sample counter"));
    PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->red.p, 0, sizeof(unsigned long long), ctx->stream));
    BiArgs a = common_args(ctx, seed, tag_path);
    a.count = count;
    a.count_dev = count_dev;
    a.list = list;
    a.gid = gid;
    a.vbase = vbase;
    a.epoch_base = (uint32_t)ctx->bi_epoch;
    ctx->bi_epoch += span + 1;
    a.ent = ctx->bi_info.as<unsigned long long>();
    a.queue = ctx->bi_queue.as<int2>();
    a.region = nslot;
    a.qcap = nslot;
    a.next = ctx->red.as<unsigned long long>();
    a.heavy_edges = heavy_edges;
    a.heavy_auto = heavy_auto;
    a.deferred = defer;
    a.defer_cost = defer_cost;
    a.n_deferred = n_def;
    launch<false, BT>(ctx, (int)slots, a);
    PERCIS_CHECK_LAUNCH(ctx, BT == kBiBlock ? "bidirectional sigma-BFS (direct)" : "bidirectional sigma-BFS (heavy)");
    return PERCIS_OK;
}

}  // namespace

// All samples of a phase (pairs, kinds already drawn): kinds of unreachable
// targets, |I|, paths and counts, as the batched form leaves them.  Every
// sample runs first with 256 threads (the direct store, or hashed tables);
// samples with a heavy level, or that outgrow their table, are handed over
// untouched and run afterwards with 1,024 threads in the direct store.
percis_status bidir_phase(percis_ctx *ctx, uint64_t seed, uint32_t tag_path, int64_t count) {
    PERCIS_TRY(ensure(ctx, ctx->ms_ctl, sizeof(MsCtl), "ms ctl"));
    // the status word may be freshly allocated: it must start at zero
    PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->ms_ctl.p, 0, sizeof(MsCtl), ctx->stream));
    ctx->phase_span = count;
    if (ctx->opt.instrument >= 2) {
        PERCIS_TRY(ensure(ctx, ctx->bi_trace, sizeof(unsigned long long) * 8 * std::max<int64_t>(count, 1),
                          "sample trace"));
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->bi_trace.p, 0, sizeof(unsigned long long) * 8 * count, ctx->stream));
        ctx->bi_trace_n = count;
    }
    // default: a heavy pass only where hubs can make a single level huge (a vertex of
    // degree >= kHubDegree, decided on the device from the graph's largest degree);
    // without hubs a handed-over sample runs no faster there
    const unsigned long long heavy =
        ctx->opt.bi_heavy_edges == 0 ? kDefaultHeavyEdges
                                     : (ctx->opt.bi_heavy_edges < 0 ? 0ull : (unsigned long long)ctx->opt.bi_heavy_edges);
    const int32_t heavy_auto = ctx->opt.bi_heavy_edges == 0 ? 1 : 0;
    if (heavy_auto && ctx->max_degree_host < 0) {
        // the graph's largest degree, once per graph (the in-degree is computed with
        // the in-adjacency, which this phase waits for anyway)
        unsigned long long md = 0ull;
        PERCIS_CUDA(ctx, cudaMemcpyAsync(&md, ctx->graph_info.p, sizeof(md), cudaMemcpyDeviceToHost, ctx->stream));
        PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        ctx->max_degree_host = (int64_t)md;
    }
    const bool heavy_on = heavy != 0ull && (!heavy_auto || ctx->max_degree_host >= (int64_t)kHubDegree);
    const int64_t cd = std::max<int64_t>(count, 1);
    PERCIS_TRY(ensure(ctx, ctx->bi_defer, (sizeof(unsigned long long) + sizeof(int32_t)) * cd + 64,
                      "handed-over samples"));
    unsigned long long *defer_cost = ctx->bi_defer.as<unsigned long long>();
    int32_t *defer = reinterpret_cast<int32_t *>(defer_cost + cd);
    unsigned int *n_def = reinterpret_cast<unsigned int *>(defer + cd);
    PERCIS_CUDA(ctx, cudaMemsetAsync(n_def, 0, sizeof(unsigned int), ctx->stream));
    int64_t nslot = ctx->n;
    if (ctx->multi) {
        const int32_t *gid;
        const int64_t *vbase;
        multi_graph_view(ctx, &gid, &vbase, &nslot);
    }
    // default: the direct store when its entries for every resident block fit the
    // scratch budget (it is the faster store per sample), else hashed tables, whose
    // memory follows the vertices a sample reaches rather than n
    bool direct = ctx->opt.bi_table_log < 0;
    if (ctx->opt.bi_table_log == 0) {
        const int64_t per_slot = nslot * (int64_t)(sizeof(unsigned long long) * 4 + sizeof(int2) * 3);
        const int64_t budget = (int64_t)(ctx->opt.bi_scratch_gib > 0 ? ctx->opt.bi_scratch_gib : kDefaultScratchGiB) << 30;
        const int64_t full = (int64_t)blocks_per_sm<false, kBiBlock>(&ctx->bi_per_sm) * ctx->num_sms;
        direct = full * per_slot <= budget;
    }
    if (direct) {
        PERCIS_TRY(
            direct_pass<kBiBlock>(ctx, seed, tag_path, count, nullptr, heavy, heavy_auto, defer, defer_cost, n_def));
    } else {
        // default: one table per block that holds the (largest) graph's vertices half
        // full, at most 2^18 entries; else 2^h0 growing 4x up to 2^hmax
        int h0, cap;
        if (ctx->opt.bi_table_log == 0) {
            h0 = kMinHLog;
            while (h0 < kDefaultHLog && (1ll << h0) < 2 * nslot + 4 * kBiBlock) ++h0;
            cap = h0;
        } else {
            h0 = std::min(std::max(ctx->opt.bi_table_log, kMinHLog), kMaxHLog);
            cap = ctx->opt.bi_table_max_log > 0 ? std::min(ctx->opt.bi_table_max_log, kMaxHLog) : kMaxHLog;
        }
        int hmax = h0;
        while (hmax + 2 <= cap && (1ll << hmax) < 2 * nslot + 4 * kBiBlock) hmax += 2;
        int64_t region = 0;
        for (int l = h0; l <= hmax; l += 2) region += 1ll << l;
        const int64_t qcap = 1ll << hmax;
        int per_sm = blocks_per_sm<true, kBiBlock>(&ctx->bi_hash_per_sm);
        if (ctx->opt.bi_blocks_per_sm > 0) per_sm = std::min(per_sm, ctx->opt.bi_blocks_per_sm);
        const int64_t slots = (int64_t)per_sm * ctx->num_sms;
        const size_t ent_bytes = sizeof(unsigned long long) * 4 * (size_t)region * slots;
        const size_t q_bytes = sizeof(int2) * 3 * (size_t)qcap * slots;
        if (ctx->bi_hregion != region || ctx->bi_hslots != slots || ctx->bi_h0 != h0) {
            PERCIS_TRY(ensure(ctx, ctx->bi_hent, ent_bytes, "hashed entries"));
            PERCIS_TRY(ensure(ctx, ctx->bi_hq, q_bytes, "hashed queues"));
            PERCIS_TRY(ensure(ctx, ctx->bi_hep, sizeof(uint32_t) * slots, "slot epochs"));
            // words of no sample (epoch 0) and epochs from 1
            PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->bi_hent.p, 0, ent_bytes, ctx->stream));
            PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->bi_hep.p, 0, sizeof(uint32_t) * slots, ctx->stream));
            ctx->bi_hregion = region;
            ctx->bi_hslots = slots;
            ctx->bi_h0 = h0;
        }
        PERCIS_TRY(ensure(ctx, ctx->red, 64, "sample counter"));
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->red.p, 0, sizeof(unsigned long long), ctx->stream));
        BiArgs a = common_args(ctx, seed, tag_path);
        a.count = count;
        a.list = nullptr;
        a.ent = ctx->bi_hent.as<unsigned long long>();
        a.queue = ctx->bi_hq.as<int2>();
        a.region = region;
        a.qcap = qcap;
        a.next = ctx->red.as<unsigned long long>();
        a.h0_log = h0;
        a.hmax_log = hmax;
        a.slot_epoch = ctx->bi_hep.as<uint32_t>();
        a.deferred = defer;
        a.defer_cost = defer_cost;
        a.n_deferred = n_def;
        a.heavy_edges = heavy;
        a.heavy_auto = heavy_auto;
        launch<true, kBiBlock>(ctx, (int)std::min<int64_t>(slots, std::max<int64_t>(count, 1)), a);
        PERCIS_CHECK_LAUNCH(ctx, "bidirectional sigma-BFS (hashed)");
    }
    // The heavy pass.  Where heavy levels hand samples over, it is launched at once
    // with one block per SM, its sample count read on the device (no host round
    // trip; blocks without a sample return).  Otherwise only a hashed first pass
    // can hand samples over (a full table, a side past 4,095 levels): rare, so the
    // count is read first and the direct store sized for it.
    ctx->bi_launches = 1;
    if (heavy_on) {
        k_order_heavy<<<1, 1024, 0, ctx->stream>>>(defer, defer_cost, n_def);  // largest first
        PERCIS_CHECK_LAUNCH(ctx, "heavy-pass order");
        PERCIS_TRY(direct_pass<kHeavyBlock>(ctx, seed, tag_path, count, defer, 0ull, 0, nullptr, nullptr, nullptr,
                                            n_def));
        ctx->bi_launches = 2;
    } else if (!direct) {
        unsigned int nd = 0;
        PERCIS_CUDA(ctx, cudaMemcpyAsync(&nd, n_def, sizeof(nd), cudaMemcpyDeviceToHost, ctx->stream));
        PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (nd > 0) {
            k_order_heavy<<<1, 1024, 0, ctx->stream>>>(defer, defer_cost, n_def);
            PERCIS_CHECK_LAUNCH(ctx, "heavy-pass order");
            PERCIS_TRY(
                direct_pass<kHeavyBlock>(ctx, seed, tag_path, (int64_t)nd, defer, 0ull, 0, nullptr, nullptr, nullptr));
            ctx->bi_launches = 2;
        }
    }
    return PERCIS_OK;
}

}  // namespace percis
