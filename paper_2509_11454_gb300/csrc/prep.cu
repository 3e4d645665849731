// Preprocessing kernels: CSR validation and transpose, the stable sort of
// the percolation states, Algorithm 2's tables, C_v, lambda_v and d^.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace percis {

namespace {

// ------------------------------------------------------------- validation

// Validation, and whether every row is strictly increasing, in two kernels so
// that the in-adjacency can be built while the columns are checked: the rows
// (row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz; desc[1] counts the rows
// whose first column is <= the previous row's last; the largest row length into
// *maxdeg), then the columns (in [0, n); desc[0] counts the positions e >= 1
// with col[e] <= col[e-1]).  The rows are strictly sorted when the counts agree.
// Counts are summed per warp: one atomic per warp and loop.
__global__ void k_check_rows(const int64_t *rp, const int32_t *col, int64_t n, int64_t nnz, uint32_t *status,
                             unsigned long long *desc, unsigned long long *maxdeg) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    unsigned long long d1 = 0, m = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t r0 = rp[v], r1 = rp[v + 1];
        if (r0 > r1 || r0 < 0 || r1 > nnz) {
            atomicOr(status, 1u);
        } else {
            m = max(m, (unsigned long long)(r1 - r0));
            if (r0 > 0 && r0 < r1 && col[r0] <= col[r0 - 1]) ++d1;
        }
        if (v == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicOr(status, 1u);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        d1 += __shfl_xor_sync(0xffffffffu, d1, off);
        m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    }
    if (lane == 0) {
        if (d1) atomicAdd(&desc[1], d1);
        if (m) atomicMax(maxdeg, m);
    }
}

__global__ void k_check_cols(const int32_t *col, int64_t n, int64_t nnz, uint32_t *status, unsigned long long *desc) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    unsigned long long d0 = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const int32_t c = col[e];
        if (c < 0 || (int64_t)c >= n) atomicOr(status, 1u);
        if (e > 0 && c <= col[e - 1]) ++d0;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) d0 += __shfl_xor_sync(0xffffffffu, d0, off);
    if (lane == 0 && d0) atomicAdd(&desc[0], d0);
}

// Largest row length of a CSR (out- or in-degree) into *out.
__global__ void k_max_degree(const int64_t *rp, int64_t n, unsigned long long *out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long m = 0ull;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        m = max(m, (unsigned long long)(rp[v + 1] - rp[v]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

__global__ void k_check_states(const double *x, int64_t n, uint32_t *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const double a = x[v];
        if (!(a >= 0.0 && a <= 1.0)) atomicOr(status, DEV_BAD_STATE);
    }
}

// ---------------------------------------------------------- state keys

__global__ void k_state_keys(const double *x, int64_t n, uint64_t *keys, int32_t *vals) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const double a = x[v] + 0.0;  // -0.0 -> +0.0
        // x >= 0: larger value <-> larger bit pattern; complement sorts descending
        keys[v] = ~(uint64_t)__double_as_longlong(a);
        vals[v] = (int32_t)v;
    }
}

__global__ void k_gather_sorted(const double *x, const int32_t *perm, int64_t n, double *xs) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) xs[i] = x[perm[i]] + 0.0;
}

// ------------------------------------------------------- Algorithm 2 scan
// The recurrences of Algorithm 2 (w_i = w_{i+1} + x_i, c_i = max(0, (n-i+1) x_i - w_i),
// r_i = r_{i+1} + c_i for i = n down to 1, and c = r_1) are chains of FP64 roundings
// whose results the sampler compares exactly, so w and r must equal the sequential
// evaluation bit for bit.  A dependent chain of FP64 adds is slow on this GPU (its
// FP64 pipe is narrow), so the two running sums are evaluated in parallel, exactly:
//  - every term is >= 0, so a running sum s never decreases and stays in one binade
//    for long stretches.  Inside a binade the doubles are the integer multiples of
//    u = ulp(s) (the subnormals and the lowest normal binade share u = 2^-1074), so
//    fl(s + a) = u * RNE(s/u + a/u) while the result stays below the binade's top:
//    an integer addition.
//  - a/u rounds to q or q + 1 from its own bits alone, except at an exact halfway
//    point, where ties-to-even picks by the parity of s/u before the term.  Each term
//    is therefore a map (parity in) -> (parity out, integer added); these maps compose
//    associatively, so one scan over them gives every running sum of a window of
//    terms at once: each block scans its chunk of 4,096 terms, the blocks' runs are
//    composed after a grid barrier, so a window spans every block of the launch.
//  - the first term whose sum reaches the top of the binade (a grid-wide minimum)
//    is added with one hardware FP64 add, and the next window starts after it in
//    the new binade (a non-decreasing sum enters each binade once).
// Both evaluations give the correctly rounded sum of the same operands in the same
// order (IEEE 754 round to nearest, ties to even) at every step, hence equal results.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;  // terms per thread and chunk
constexpr int kScanChunk = kScanThreads * kScanPer;
constexpr int kMaxTableBlocks = 1024;
constexpr unsigned long long kTwo53u = 1ull << 53;
constexpr long long kNoTerm = 0x7fffffffffffffffll;

// map of a run of terms: for parity p of s/u before the run, d0 / d1 is the integer
// added and bit p of par the parity after it
struct ParityMap {
    unsigned long long d0, d1;
    unsigned par;
};

__device__ __forceinline__ ParityMap pm_identity() { return ParityMap{0ull, 0ull, 2u}; }

// the run f followed by the run g
__device__ __forceinline__ ParityMap pm_then(const ParityMap &f, const ParityMap &g) {
    const unsigned f0 = f.par & 1u, f1 = (f.par >> 1) & 1u;
    ParityMap h;
    h.d0 = f.d0 + (f0 ? g.d1 : g.d0);
    h.d1 = f.d1 + (f1 ? g.d1 : g.d0);
    h.par = ((g.par >> f0) & 1u) | (((g.par >> f1) & 1u) << 1);
    return h;
}

__device__ __forceinline__ ParityMap pm_shfl_up(const ParityMap &m, int off) {
    ParityMap o;
    o.d0 = __shfl_up_sync(0xffffffffu, m.d0, off);
    o.d1 = __shfl_up_sync(0xffffffffu, m.d1, off);
    o.par = __shfl_up_sync(0xffffffffu, m.par, off);
    return o;
}

// one term a >= 0 against a running sum whose binade has exponent field e (>= 1):
// q = a/u rounded down and the rounding kind (0 exact or down, 1 up, 2 halfway,
// 3 a alone reaches the top of the binade), and the term's map
__device__ __forceinline__ ParityMap term_map(double a, int e, unsigned long long &q, int &kind) {
    const unsigned long long ab = (unsigned long long)__double_as_longlong(a);
    const int ea = (int)((ab >> 52) & 0x7ff);
    ParityMap m;
    if (ea > e) {
        q = kTwo53u;
        kind = 3;
        m.d0 = m.d1 = kTwo53u;
        m.par = 0u;
        return m;
    }
    const unsigned long long ma = (ab & ((1ull << 52) - 1)) | (ea ? (1ull << 52) : 0ull);
    const int sh = e - max(ea, 1);  // a / u = ma / 2^sh
    kind = 0;
    if (sh == 0) {
        q = ma;
    } else if (sh > 54) {  // below half a unit
        q = 0ull;
    } else {
        q = ma >> sh;
        const unsigned long long rem = ma & ((1ull << sh) - 1), half = 1ull << (sh - 1);
        kind = rem > half ? 1 : (rem == half ? 2 : 0);
    }
    if (kind == 2) {  // the even neighbour for either parity: parity 0 after
        m.d0 = q + (q & 1ull);
        m.d1 = q + 1ull - (q & 1ull);
        m.par = 0u;
    } else {
        const unsigned long long R = q + (unsigned long long)kind;
        const unsigned b = (unsigned)(R & 1ull);
        m.d0 = m.d1 = R;
        m.par = b | ((b ^ 1u) << 1);
    }
    return m;
}

// map of a run of terms, as stored between the phases of a window
struct alignas(16) RunMap {
    unsigned long long d0, d1;
    unsigned long long par;
};

constexpr int kKeys = 2048;    // binade keys max(exponent field, 1)
constexpr int kMaxSegs = 256;  // binades the resolution of a predicted pass holds

// A binade of the running sum in the predicted pass: its first term (the one
// whose sum enters it, added in plain FP64) and, once resolved, the sum there.
struct SegSlot {
    unsigned int gen;         // the pass that claimed the slot
    int prev;                 // key of the binade before (-1: the first term)
    long long b;              // the first term
    double a;                 // its value
    RunMap mprev;             // map of the terms of the binade before, after its first
    unsigned long long s0;    // resolved: sum after term b in units of the binade's ulp
    double scross;            // resolved: sum after term b
};

// Control block of the cooperative table launch.
struct TableCtl {
    GridBarrier bar;
    uint32_t status;
    uint32_t conflict;   // the predicted pass found its binades inconsistent
    long long kstar[2];  // first term of the window that leaves the binade (one slot per window parity)
    long long pos;       // positions pos, pos - 1, ..., 1 remain
    double s;            // running sum before them
    long long fail_b;    // predicted pass: terms before this one are resolved
    int klast;           // predicted pass: key of the last term
    int pad2;
    RunMap mlast;        // predicted pass: map of the last binade's terms after its first
    RunMap agg[kMaxTableBlocks];
    RunMap sagg[kMaxTableBlocks];  // predicted pass: segmented run of each block (flag in par bit 2)
    double bsum[kMaxTableBlocks];  // predicted pass: FP64 sum of each block's terms
    int blast[kMaxTableBlocks];    // predicted pass: key after each block's last term
    SegSlot seg[kKeys];
};

__device__ __forceinline__ ParityMap run_load(const RunMap *p) {
    ParityMap m;
    m.d0 = __ldcg(&p->d0);
    m.d1 = __ldcg(&p->d1);
    m.par = (unsigned)__ldcg(&p->par);
    return m;
}

__device__ __forceinline__ int sum_key(double v) {
    const int ef = (int)(((unsigned long long)__double_as_longlong(v) >> 52) & 0x7ff);
    return ef > 1 ? ef : 1;
}

// segmented runs: f = the run holds the first term of a binade (the map then
// covers the terms after the last such term)
struct SegRun {
    ParityMap m;
    unsigned f;
};

__device__ __forceinline__ SegRun sr_identity() { return SegRun{pm_identity(), 0u}; }

__device__ __forceinline__ SegRun sr_then(const SegRun &x, const SegRun &y) {
    SegRun r;
    r.f = x.f | y.f;
    r.m = y.f ? y.m : pm_then(x.m, y.m);
    return r;
}

__device__ __forceinline__ SegRun sr_shfl_up(const SegRun &v, int off) {
    SegRun o;
    o.m = pm_shfl_up(v.m, off);
    o.f = __shfl_up_sync(0xffffffffu, v.f, off);
    return o;
}

__device__ __forceinline__ RunMap sr_store(const SegRun &v) {
    RunMap r;
    r.d0 = v.m.d0;
    r.d1 = v.m.d1;
    r.par = (unsigned long long)(v.m.par | (v.f << 2));
    return r;
}

__device__ __forceinline__ SegRun sr_load(const RunMap *p) {
    SegRun v;
    v.m.d0 = __ldcg(&p->d0);
    v.m.d1 = __ldcg(&p->d1);
    const unsigned par = (unsigned)__ldcg(&p->par);
    v.m.par = par & 3u;
    v.f = (par >> 2) & 1u;
    return v;
}

// Predicted pass over the same running sums, in a few grid barriers: a plain
// FP64 prefix sum of the terms (any order) predicts the binade every term's
// sum falls in; every binade's run of terms after its first is then one
// segment of a segmented scan of the per-term maps, all binades at once; one
// thread walks the binades in order, adds each first term in plain FP64 from
// the sum before it and checks that it lands in the predicted binade and that
// the binade's run stays below its top; every term before the first failed
// check gets its exact sum.  The prediction only chooses the segments: each
// binade's result is checked against the sequential definition, and the terms
// from the first failure on (a sum within rounding of a binade's edge, more
// than kMaxSegs binades) are left to the windowed scan, which starts from
// ctl->pos and ctl->s.
__device__ bool running_sum_predicted(const double *src, int64_t soff, double *dst, int64_t m, TableCtl *ctl,
                                      uint64_t budget_ns, unsigned gen) {
    constexpr int nw = kScanThreads / 32;
    __shared__ double s_wd[nw];
    __shared__ SegRun s_wr[nw];
    __shared__ int s_lastkey[kScanThreads];
    __shared__ double s_bc;
    __shared__ SegRun s_bsr;
    __shared__ int s_key[kMaxSegs];
    __shared__ int s_pc[nw];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long nth = (long long)gridDim.x * kScanThreads;
    const long long T = (m + nth - 1) / nth;
    const long long g = (long long)blockIdx.x * kScanThreads + tid;
    const long long k0 = min((long long)m, g * T), k1 = min((long long)m, k0 + T);
    // term k of the scan (k = 0 is position m)
    auto term = [&](long long k) { return __ldcg(&src[m - k + soff]); };

    // 1. the prediction: exclusive FP64 prefix of the threads' sums
    if (blockIdx.x == 0 && tid == 0) ctl->conflict = 0u;  // (set only after the barrier below)
    double ts = 0.0;
    for (long long k = k0; k < k1; ++k) ts = __dadd_rn(ts, term(k));
    double inc = warp_inclusive_scan(ts);
    double exc = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) exc = 0.0;
    if (lane == 31) s_wd[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const double v = lane < nw ? s_wd[lane] : 0.0;
        const double vi = warp_inclusive_scan(v);
        double ve = __shfl_up_sync(0xffffffffu, vi, 1);
        if (lane == 0) ve = 0.0;
        if (lane < nw) s_wd[lane] = ve;
        if (lane == 31) ctl->bsum[blockIdx.x] = vi;
    }
    if (!grid_sync(&ctl->bar, &ctl->status, budget_ns)) return false;
    if (warp == 0) {
        double c = 0.0;
        for (int b0 = 0; b0 < (int)blockIdx.x; b0 += 32)
            c = __dadd_rn(c, __shfl_sync(0xffffffffu,
                                         warp_inclusive_scan(b0 + lane < (int)blockIdx.x ? __ldcg(&ctl->bsum[b0 + lane])
                                                                                         : 0.0),
                                         31));
        if (lane == 0) s_bc = c;
    }
    __syncthreads();
    const double pin = __dadd_rn(__dadd_rn(s_bc, s_wd[warp]), exc);

    // 2. binades: a term whose predicted sum has another key than the one before
    // starts a binade (term 0 always); the segmented run of every thread
    const int key_in = k0 == 0 ? -1 : sum_key(pin);
    int before = key_in;
    double P = pin;
    SegRun agg = sr_identity();
    ParityMap lfirst = pm_identity();  // the thread's terms before its first binade start
    int efirst = -1;
    for (long long k = k0; k < k1; ++k) {
        const double a = term(k);
        P = __dadd_rn(P, a);
        const int E = sum_key(P);
        if (E != before) {
            SegSlot *sg = &ctl->seg[E];
            if (atomicExch(&sg->gen, gen) == gen) atomicOr(&ctl->conflict, 1u);  // a binade entered twice
            sg->b = k;
            sg->a = a;
            sg->prev = before;
            if (efirst >= 0) sg->mprev = RunMap{agg.m.d0, agg.m.d1, (unsigned long long)agg.m.par};
            else {
                efirst = E;
                lfirst = agg.m;
            }
            agg.m = pm_identity();
            agg.f = 1u;
            before = E;
        } else {
            unsigned long long q;
            int kind;
            agg.m = pm_then(agg.m, term_map(a, E, q, kind));
        }
    }
    s_lastkey[tid] = before;
    // segmented scan of the runs: the warp, the block, then the blocks before
    SegRun sinc = agg;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const SegRun o = sr_shfl_up(sinc, off);
        if (lane >= off) sinc = sr_then(o, sinc);
    }
    SegRun sexc = sr_shfl_up(sinc, 1);
    if (lane == 0) sexc = sr_identity();
    if (lane == 31) s_wr[warp] = sinc;
    __syncthreads();
    // the key the thread's first term starts from must be the one the thread
    // before ended on (both predicted, in different summation orders)
    if (tid > 0 && k0 < k1 && key_in != s_lastkey[tid - 1]) atomicOr(&ctl->conflict, 1u);
    if (warp == 0) {
        SegRun v = lane < nw ? s_wr[lane] : sr_identity();
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const SegRun o = sr_shfl_up(v, off);
            if (lane >= off) v = sr_then(o, v);
        }
        SegRun ve = sr_shfl_up(v, 1);
        if (lane == 0) ve = sr_identity();
        if (lane < nw) s_wr[lane] = ve;
        if (lane == 31) ctl->sagg[blockIdx.x] = sr_store(v);
        if (lane == 0) ctl->blast[blockIdx.x] = s_lastkey[kScanThreads - 1];
    }
    if (!grid_sync(&ctl->bar, &ctl->status, budget_ns)) return false;
    if (warp == 0) {
        SegRun bp = sr_identity();
        for (int b0 = 0; b0 < (int)blockIdx.x; b0 += 32) {
            SegRun v = b0 + lane < (int)blockIdx.x ? sr_load(&ctl->sagg[b0 + lane]) : sr_identity();
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const SegRun o = sr_shfl_up(v, off);
                if (lane >= off) v = sr_then(o, v);
            }
            SegRun last;
            last.m.d0 = __shfl_sync(0xffffffffu, v.m.d0, 31);
            last.m.d1 = __shfl_sync(0xffffffffu, v.m.d1, 31);
            last.m.par = __shfl_sync(0xffffffffu, v.m.par, 31);
            last.f = __shfl_sync(0xffffffffu, v.f, 31);
            bp = sr_then(bp, last);
        }
        if (lane == 0) {
            s_bsr = bp;
            if (blockIdx.x > 0 && k0 < k1 && key_in != __ldcg(&ctl->blast[blockIdx.x - 1]))
                atomicOr(&ctl->conflict, 1u);
        }
    }
    __syncthreads();
    const SegRun cin = sr_then(s_bsr, sr_then(s_wr[warp], sexc));  // the run since the binade start before k0
    if (efirst >= 0) {
        const ParityMap mp = pm_then(cin.m, lfirst);
        ctl->seg[efirst].mprev = RunMap{mp.d0, mp.d1, (unsigned long long)mp.par};
    }
    if (k1 == m && k0 < k1) {
        const ParityMap ml = efirst >= 0 ? agg.m : pm_then(cin.m, agg.m);
        ctl->mlast = RunMap{ml.d0, ml.d1, (unsigned long long)ml.par};
        ctl->klast = before;
    }
    if (!grid_sync(&ctl->bar, &ctl->status, budget_ns)) return false;

    // 3. resolution, in block 0: the binades present, in key order, then one
    // thread walks them from s = +0
    if (blockIdx.x == 0) {
        const int E0 = 2 * tid, E1 = E0 + 1;
        const int p0 = __ldcg(&ctl->seg[E0].gen) == gen, p1 = __ldcg(&ctl->seg[E1].gen) == gen;
        const int c = p0 + p1;
        int ci = c;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int o = __shfl_up_sync(0xffffffffu, ci, off);
            if (lane >= off) ci += o;
        }
        if (lane == 31) s_pc[warp] = ci;
        __syncthreads();
        int base = 0, total = 0;
        for (int q = 0; q < nw; ++q) {
            if (q < warp) base += s_pc[q];
            total += s_pc[q];
        }
        const int at = base + ci - c;
        if (total <= kMaxSegs) {
            if (p0) s_key[at] = E0;
            if (p1) s_key[at + p0] = E1;
        }
        __syncthreads();
        if (tid == 0) {
            long long fail = m;
            double S = 0.0;
            if (__ldcg(&ctl->conflict) || total > kMaxSegs || total < 1 || __ldcg(&ctl->klast) != s_key[total - 1])
                fail = 0;
            for (int i = 0; fail == m && i < total; ++i) {
                const int E = s_key[i];
                SegSlot *sg = &ctl->seg[E];
                const long long b = __ldcg(&sg->b);
                if ((i == 0) != (b == 0) || __ldcg(&sg->prev) != (i == 0 ? -1 : s_key[i - 1])) {
                    fail = i == 0 ? 0 : b;
                    break;
                }
                const double sc = __dadd_rn(S, __ldcg(&sg->a));
                if (sum_key(sc) != E) {  // the first term did not land in the predicted binade
                    fail = b;
                    break;
                }
                const unsigned long long sb = (unsigned long long)__double_as_longlong(sc);
                const int es = (int)((sb >> 52) & 0x7ff);
                const unsigned long long S0 = (sb & ((1ull << 52) - 1)) | (es ? (1ull << 52) : 0ull);
                const RunMap *mr = i + 1 < total ? &ctl->seg[s_key[i + 1]].mprev : &ctl->mlast;
                const unsigned long long d = (S0 & 1ull) ? __ldcg(&mr->d1) : __ldcg(&mr->d0);
                if (S0 + d >= kTwo53u) {  // the run leaves the binade before the next predicted start
                    fail = b;
                    break;
                }
                sg->s0 = S0;
                sg->scross = sc;
                S = __longlong_as_double((long long)(((unsigned long long)(E - 1) << 52) + S0 + d));
            }
            ctl->fail_b = fail;
            ctl->pos = m - fail;
            ctl->s = S;  // the sum before term `fail` (every binade before it resolved)
        }
    }
    if (!grid_sync(&ctl->bar, &ctl->status, budget_ns)) return false;

    // 4. every term before the first failure: its binade's sum after the first
    // term plus the integer its run added, under that sum's parity
    const long long fail = __ldcg(&ctl->fail_b);
    if (k0 < fail) {
        const long long kend = min(k1, fail);
        int cur = key_in;
        unsigned long long S0 = 0ull, top = 0ull;
        if (cur >= 1) {
            S0 = __ldcg(&ctl->seg[cur].s0);
            top = (unsigned long long)(cur - 1) << 52;
        }
        ParityMap pre = cin.m;
        P = pin;
        for (long long k = k0; k < kend; ++k) {
            const double a = term(k);
            P = __dadd_rn(P, a);
            const int E = sum_key(P);
            if (E != cur) {
                cur = E;
                S0 = __ldcg(&ctl->seg[E].s0);
                top = (unsigned long long)(E - 1) << 52;
                pre = pm_identity();
                dst[m - k] = __ldcg(&ctl->seg[E].scross);
            } else {
                unsigned long long q;
                int kind;
                pre = pm_then(pre, term_map(a, E, q, kind));
                dst[m - k] = __longlong_as_double((long long)(top + S0 + ((S0 & 1ull) ? pre.d1 : pre.d0)));
            }
        }
    }
    return grid_sync(&ctl->bar, &ctl->status, budget_ns);
}

// Running sums s_i = fl(s_{i+1} + a_i) for i = m down to 1 (s_{m+1} = +0), with
// a_i = src[i + soff] >= 0, written to dst[i]; *sum = s_1 (+0 when m = 0).  Every
// block of the cooperative launch calls it; false when a grid barrier timed out.
__device__ bool grid_running_sum(const double *src, int64_t soff, double *dst, int64_t m, TableCtl *ctl,
                                 uint64_t budget_ns, unsigned gen, double *sum) {
    __shared__ ParityMap s_wmap[kScanThreads / 32];
    __shared__ ParityMap s_bpre;
    __shared__ unsigned s_first;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int G = gridDim.x;
    static_assert((long long)kMaxTableBlocks * kScanChunk < 0xffffffffll, "window indexes fit 32 bits");
    if (tid == 0) s_first = 0xffffffffu;
    if (blockIdx.x == 0 && tid == 0) {
        ctl->pos = m;
        ctl->s = 0.0;
        ctl->kstar[0] = ctl->kstar[1] = kNoTerm;
    }
    if (!grid_sync(&ctl->bar, &ctl->status, budget_ns)) return false;
    // the predicted pass resolves what it can; windows of the terms left
    if (m > 0 && !running_sum_predicted(src, soff, dst, m, ctl, budget_ns, gen)) return false;
    for (int pass = 0;; ++pass) {
        const long long pos = __ldcg(&ctl->pos);
        const double s = __ldcg(&ctl->s);
        if (pos <= 0) break;  // the same in every block
        const long long window = pos < (long long)G * kScanChunk ? pos : (long long)G * kScanChunk;
        const long long kb = (long long)blockIdx.x * kScanChunk;  // window index of the block's first term
        const unsigned long long sb = (unsigned long long)__double_as_longlong(s);
        const int es = (int)((sb >> 52) & 0x7ff);
        const int e = max(es, 1);
        const unsigned long long S0 = (sb & ((1ull << 52) - 1)) | (es ? (1ull << 52) : 0ull);
        const unsigned long long top = (unsigned long long)(e - 1) << 52;  // bits of u * S are top + S
        double a[kScanPer];
        unsigned long long q[kScanPer];
        int kind[kScanPer];
        ParityMap mine = pm_identity();
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            const long long k = kb + tid * kScanPer + j;
            a[j] = k < window ? __ldcg(&src[pos - k + soff]) : 0.0;  // written by other blocks (c_i)
            mine = pm_then(mine, term_map(a[j], e, q[j], kind[j]));
        }
        // scan of the maps: within the warp, then over the warps, then over the blocks
        ParityMap inc = mine;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const ParityMap o = pm_shfl_up(inc, off);
            if (lane >= off) inc = pm_then(o, inc);
        }
        ParityMap exc = pm_shfl_up(inc, 1);
        if (lane == 0) exc = pm_identity();
        if (lane == 31) s_wmap[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            ParityMap wm = lane < kScanThreads / 32 ? s_wmap[lane] : pm_identity();
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const ParityMap o = pm_shfl_up(wm, off);
                if (lane >= off) wm = pm_then(o, wm);
            }
            ParityMap we = pm_shfl_up(wm, 1);
            if (lane == 0) we = pm_identity();
            if (lane < kScanThreads / 32) s_wmap[lane] = we;  // runs of the warps before each warp
            if (lane == 31) {  // the block's whole run
                RunMap *g = &ctl->agg[blockIdx.x];
                g->d0 = wm.d0;
                g->d1 = wm.d1;
                g->par = wm.par;
            }
        }
        if (!grid_sync(&ctl->bar, &ctl->status, budget_ns)) return false;
        if (warp == 0) {  // the run of the blocks before this one
            ParityMap bp = pm_identity();
            for (int b0 = 0; b0 < (int)blockIdx.x; b0 += 32) {
                ParityMap bm = b0 + lane < (int)blockIdx.x ? run_load(&ctl->agg[b0 + lane]) : pm_identity();
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const ParityMap o = pm_shfl_up(bm, off);
                    if (lane >= off) bm = pm_then(o, bm);
                }
                ParityMap last;
                last.d0 = __shfl_sync(0xffffffffu, bm.d0, 31);
                last.d1 = __shfl_sync(0xffffffffu, bm.d1, 31);
                last.par = __shfl_sync(0xffffffffu, bm.par, 31);
                bp = pm_then(bp, last);
            }
            if (lane == 0) s_bpre = bp;
        }
        __syncthreads();
        const ParityMap pre = pm_then(s_bpre, pm_then(s_wmap[warp], exc));
        // this thread's terms under the true parity of S0
        const unsigned p0 = (unsigned)(S0 & 1ull);
        unsigned p = (pre.par >> p0) & 1u;
        unsigned long long acc = p0 ? pre.d1 : pre.d0;  // integer added before this thread's terms
        unsigned long long before[kScanPer];
        long long first = kNoTerm;
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            const long long k = kb + tid * kScanPer + j;
            before[j] = acc;
            unsigned long long R;
            if (kind[j] == 2) {
                R = q[j] + ((q[j] ^ (unsigned long long)p) & 1ull);
                p = 0u;
            } else {
                R = q[j] + (unsigned long long)(kind[j] & 1);
                p ^= (unsigned)(R & 1ull);
            }
            acc += R;
            // sums before the first term that leaves the binade stay below 2^54: no wrap
            if (k < window && first == kNoTerm && (kind[j] == 3 || S0 + acc >= kTwo53u)) first = k;
        }
        // the window's first crossing: minimum over the warp, the block, then one
        // global atomic per block (window indexes fit 32 bits)
        const int slot = pass & 1;
        unsigned fm = __reduce_min_sync(0xffffffffu, first == kNoTerm ? 0xffffffffu : (unsigned)first);
        if (lane == 0 && fm != 0xffffffffu) atomicMin(&s_first, fm);
        __syncthreads();
        if (tid == 0 && s_first != 0xffffffffu) atomicMin(&ctl->kstar[slot], (long long)s_first);
        if (!grid_sync(&ctl->bar, &ctl->status, budget_ns)) return false;
        if (tid == 0) s_first = 0xffffffffu;  // read by thread 0 alone, before the barrier above
        const long long ks = __ldcg(&ctl->kstar[slot]);
        const long long kstar = ks < window ? ks : window;  // terms before kstar stay in the binade
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            const long long k = kb + tid * kScanPer + j;
            const unsigned long long after = j + 1 < kScanPer ? before[j + 1] : acc;
            if (k < kstar) dst[pos - k] = __longlong_as_double((long long)(top + S0 + after));
            if (k == kstar - 1 && kstar == window) ctl->s = __longlong_as_double((long long)(top + S0 + after));
            if (k == kstar && kstar < window) {
                // the term that leaves the binade: one hardware add from the sum before it
                const double prev = k == 0 ? s : __longlong_as_double((long long)(top + S0 + before[j]));
                const double nv = __dadd_rn(prev, a[j]);
                dst[pos - k] = nv;
                ctl->s = nv;
            }
        }
        if (blockIdx.x == 0 && tid == 0) {
            ctl->kstar[slot ^ 1] = kNoTerm;  // for the next window
            ctl->pos = pos - (kstar < window ? kstar + 1 : window);
        }
        if (!grid_sync(&ctl->bar, &ctl->status, budget_ns)) return false;
    }
    *sum = __ldcg(&ctl->s);
    return true;
}

// Number of non-zero sorted states (xs is non-increasing and >= 0, so the
// zeros form a suffix), by bisection, into the int64 word at dscal + 2.
__global__ void k_nonzero_prefix(const double *xs, int64_t n, double *dscal) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t lo = 0, hi = n;  // first zero in [lo, hi]
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (xs[mid] == 0.0) hi = mid;
        else lo = mid + 1;
    }
    *reinterpret_cast<long long *>(dscal + 2) = (long long)lo;
}

// Cooperative launch of G blocks (all co-resident): w, then c_i, then r.
__global__ void __launch_bounds__(kScanThreads) k_tables(const double *xs, int64_t n, double *w, double *ci,
                                                         double *r, double *dscal, TableCtl *ctl,
                                                         uint64_t budget_ns) {
    // positions past the last non-zero state: x_i = 0 and every sum before them
    // is +0, so w_i = c_i = r_i = 0 exactly; the scans start at the last non-zero one
    const int64_t nz = *reinterpret_cast<const long long *>(dscal + 2);
    const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = nz + 1 + gt; i <= n + 1; i += gs) w[i] = ci[i] = r[i] = 0.0;
    if (gt == 0) w[0] = r[0] = ci[0] = 0.0;
    // w_i over x_i = xs[i - 1]
    double wsum;
    if (!grid_running_sum(xs, -1, w, nz, ctl, budget_ns, 1u, &wsum)) return;
    for (int64_t i = 1 + gt; i <= nz; i += gs) {
        const double t = __dmul_rn((double)(n - i + 1), xs[i - 1]);
        const double cv = __dsub_rn(t, __ldcg(&w[i]));
        ci[i] = __double_as_longlong(cv) < 0 ? 0.0 : cv;  // max(0, .), -0 -> +0
    }
    if (!grid_sync(&ctl->bar, &ctl->status, budget_ns)) return;
    double c;
    if (!grid_running_sum(ci, 0, r, nz, ctl, budget_ns, 2u, &c)) return;
    if (gt == 0) dscal[0] = c;  // c = r_1
}

// C_v = c - A_v with A_i = (w_1 - w_i) - (i-1) x_i + (n-i) x_i - w_{i+1} for
// sorted position i (the closed form of sum_u |x_i - x_u|), lambda = c / C_v.
__global__ void k_cv_lambda(const double *xs, const int32_t *perm, const double *w, const double *dscal, int64_t n,
                            double *Cv, double *lam, uint32_t *status) {
    const double c = dscal[0];
    const double w1 = w[1];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; i <= n; i += stride) {
        const double xi = xs[i - 1];
        double a = __dsub_rn(w1, w[i]);
        a = __dsub_rn(a, __dmul_rn((double)(i - 1), xi));
        a = __dadd_rn(a, __dmul_rn((double)(n - i), xi));
        a = __dsub_rn(a, w[i + 1]);
        const double cv = __dsub_rn(c, a);
        const int32_t v = perm[i - 1];
        Cv[v] = cv;
        if (cv > 0.0) {
            lam[v] = __ddiv_rn(c, cv);
        } else {
            lam[v] = __longlong_as_double(0x7ff0000000000000LL);
            atomicOr(status, DEV_DEGENERATE);
        }
    }
}

__device__ __forceinline__ void atomic_max_pos_double(double *addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

__global__ void k_max_lambda(const double *lam, int64_t n, double *dscal) {
    double m = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) m = fmax(m, lam[v]);
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomic_max_pos_double(&dscal[1], m);
}

// Tie groups of the sorted states: positions [lo, hi] (1-based) with equal x.
__global__ void k_groups(const double *xs, int64_t n, int32_t *glo, int32_t *ghi) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double v = xs[i];
        // xs is non-increasing: first index with xs <= v, last index with xs >= v
        int64_t lo = 0, hi = i;
        while (lo < hi) {
            const int64_t m = (lo + hi) >> 1;
            if (xs[m] > v) lo = m + 1;
            else hi = m;
        }
        int64_t a = i, b = n - 1;
        while (a < b) {
            const int64_t m = (a + b + 1) >> 1;
            if (xs[m] < v) b = m - 1;
            else a = m;
        }
        glo[i] = (int32_t)(lo + 1);
        ghi[i] = (int32_t)(a + 1);
    }
}

// ------------------------------------------------------------- transpose

// key(v) = (highest-degree out-neighbour of v, ties to the smallest id) << 32 | v;
// vertices without neighbours use themselves.
__global__ void k_hub_keys(const int64_t *rp, const int32_t *col, int64_t n, uint64_t *keys, int32_t *vals) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        int32_t best = (int32_t)v;
        int64_t bdeg = -1;
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
            const int32_t u = col[e];
            const int64_t d = rp[u + 1] - rp[u];
            if (d > bdeg || (d == bdeg && u < best)) {
                bdeg = d;
                best = u;
            }
        }
        keys[v] = ((uint64_t)(uint32_t)best << 32) | (uint32_t)v;
        vals[v] = (int32_t)v;
    }
}


}  // namespace

// Lane order of batched sources: vertices sorted by (highest-degree neighbour,
// id).  Only the batched form needs it, so it is built on first use.
percis_status prep_vorder(percis_ctx *ctx) {
    if (ctx->vorder_ready) return PERCIS_OK;
    const int64_t n = ctx->n;
    {
        PERCIS_TRY(ensure(ctx, ctx->vorder, sizeof(int32_t) * n, "vertex order"));
        DevBuf k1, k2, v2;
        cudaError_t e = cudaMalloc(&k1.p, sizeof(uint64_t) * n);
        if (e == cudaSuccess) e = cudaMalloc(&k2.p, sizeof(uint64_t) * n);
        if (e == cudaSuccess) e = cudaMalloc(&v2.p, sizeof(int32_t) * n);
        percis_status rs = PERCIS_OK;
        if (e != cudaSuccess) {
            cudaGetLastError();
            rs = set_err(ctx, PERCIS_E_OOM, "vertex order scratch");
        } else {
            k_hub_keys<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(ctx->rp.as<int64_t>(), ctx->col.as<int32_t>(),
                                                                     n, k1.as<uint64_t>(), ctx->vorder.as<int32_t>());
            ctx->launches++;
            // (the low word is the vertex id, already in order: a stable sort by the high word suffices)
            rs = radix_sort_u64(ctx, k1.as<uint64_t>(), ctx->vorder.as<int32_t>(), k2.as<uint64_t>(),
                                v2.as<int32_t>(), n, 32, 32);
        }
        cudaStreamSynchronize(ctx->stream);
        cudaFree(k1.p);
        cudaFree(k2.p);
        cudaFree(v2.p);
        if (rs != PERCIS_OK) return rs;
    }
    ctx->vorder_ready = true;
    return PERCIS_OK;
}

percis_status prep_graph(percis_ctx *ctx) {
    const int64_t n = ctx->n, nnz = ctx->nnz;
    PERCIS_TRY(ensure(ctx, ctx->status, 64, "status"));
    uint32_t *st = ctx->status.as<uint32_t>();
    PERCIS_CUDA(ctx, cudaMemsetAsync(st, 0, 64, ctx->stream));
    unsigned long long *desc = reinterpret_cast<unsigned long long *>(ctx->status.as<char>() + 8);
    // the largest out- and in-degree (read on the device by the bidirectional form's
    // default heavy-level rule)
    PERCIS_TRY(ensure(ctx, ctx->graph_info, 64, "graph info"));
    ctx->max_degree_host = -1;
    unsigned long long *md = ctx->graph_info.as<unsigned long long>();
    PERCIS_CUDA(ctx, cudaMemsetAsync(md, 0, sizeof(unsigned long long), ctx->stream));
    k_check_rows<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(ctx->rp.as<int64_t>(), ctx->col.as<int32_t>(), n,
                                                                 nnz, st, desc, md);
    PERCIS_CHECK_LAUNCH(ctx, "check rows");
    unsigned long long hst[3] = {0ull, 0ull, 0ull};
    PERCIS_CUDA(ctx, cudaMemcpyAsync(hst, st, sizeof(hst), cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if ((uint32_t)hst[0]) return set_err(ctx, PERCIS_E_INVALID, "malformed CSR (row_ptr not monotone)");
    if (ctx->directed) {
        // the in-adjacency's sort on the second stream, after everything issued so far
        // (earlier work may still read the previous one), while the columns are checked
        // here; the sort's digits are masked, so it reads and writes in bounds whatever
        // the columns hold.  Its last step (the offsets, indexed by column) waits for the
        // check.  The states can be prepared on this stream meanwhile.
        if (!ctx->aux) {
            PERCIS_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->aux, cudaStreamNonBlocking));
            PERCIS_CUDA(ctx, cudaEventCreateWithFlags(&ctx->aux_go, cudaEventDisableTiming));
            PERCIS_CUDA(ctx, cudaEventCreateWithFlags(&ctx->graph_ready, cudaEventDisableTiming));
        }
        PERCIS_CUDA(ctx, cudaEventRecord(ctx->aux_go, ctx->stream));
        PERCIS_CUDA(ctx, cudaStreamWaitEvent(ctx->aux, ctx->aux_go, 0));
    }
    // the column check first, so that it starts before the sort's launches are issued
    k_check_cols<<<grid_for(ctx, nnz, 256), 256, 0, ctx->stream>>>(ctx->col.as<int32_t>(), n, nnz, st, desc);
    PERCIS_CHECK_LAUNCH(ctx, "check columns");
    if (ctx->directed) {
        AuxScope scope(ctx);
        PERCIS_TRY(transpose_sort(ctx));
    }
    PERCIS_CUDA(ctx, cudaMemcpyAsync(hst, st, sizeof(hst), cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if ((uint32_t)hst[0]) return set_err(ctx, PERCIS_E_INVALID, "malformed CSR (column out of range)");
    ctx->rows_sorted = hst[1] == hst[2];  // (the in-lists of a stable transpose are then sorted too)
    if (ctx->directed) {
        percis_status tst;
        {
            AuxScope scope(ctx);
            tst = transpose_finish(ctx);
            if (tst == PERCIS_OK) {
                k_max_degree<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(ctx->irp.as<int64_t>(), n, md);
                tst = cudaGetLastError() == cudaSuccess ? PERCIS_OK : set_err(ctx, PERCIS_E_CUDA, "max in-degree");
                ctx->launches++;
            }
        }
        PERCIS_TRY(tst);
        PERCIS_CUDA(ctx, cudaEventRecord(ctx->graph_ready, ctx->aux));
        ctx->graph_pending = true;
    }
    ctx->vorder_ready = false;  // built on first use by the batched form
    if (!ctx->skip_diam) {
        int64_t D = 0;
        PERCIS_TRY(vertex_diam_ub(ctx, &D));
        ctx->vertex_diam = D;
    }
    return PERCIS_OK;
}

percis_status wait_graph(percis_ctx *ctx) {
    if (ctx->graph_pending) {
        PERCIS_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->graph_ready, 0));
        ctx->graph_pending = false;
    }
    return PERCIS_OK;
}

percis_status prep_states(percis_ctx *ctx) {
    const int64_t n = ctx->n;
    uint32_t *st = ctx->status.as<uint32_t>();
    PERCIS_CUDA(ctx, cudaMemsetAsync(st, 0, 64, ctx->stream));
    k_check_states<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(ctx->x.as<double>(), n, st);
    PERCIS_CHECK_LAUNCH(ctx, "check states");

    PERCIS_TRY(ensure(ctx, ctx->xs, sizeof(double) * n, "xs"));
    PERCIS_TRY(ensure(ctx, ctx->perm, sizeof(int32_t) * n, "perm"));
    PERCIS_TRY(ensure(ctx, ctx->w, sizeof(double) * (n + 2), "w"));
    PERCIS_TRY(ensure(ctx, ctx->ci, sizeof(double) * (n + 2), "ci"));
    PERCIS_TRY(ensure(ctx, ctx->r, sizeof(double) * (n + 2), "r"));
    PERCIS_TRY(ensure(ctx, ctx->Cv, sizeof(double) * n, "Cv"));
    PERCIS_TRY(ensure(ctx, ctx->lam, sizeof(double) * n, "lambda"));
    PERCIS_TRY(ensure(ctx, ctx->dscal, 64, "scalars"));
    // sort scratch: keys, keys2, vals2 (reuse the sigma buffer space if large)
    PERCIS_TRY(ensure(ctx, ctx->pc_tmp, (sizeof(uint64_t) * 2 + sizeof(int32_t)) * n + 64, "sort scratch"));
    uint64_t *k1 = ctx->pc_tmp.as<uint64_t>();
    uint64_t *k2 = k1 + n;
    int32_t *v2 = (int32_t *)(k2 + n);
    int32_t *perm = ctx->perm.as<int32_t>();
    const int g = grid_for(ctx, n, 256);
    k_state_keys<<<g, 256, 0, ctx->stream>>>(ctx->x.as<double>(), n, k1, perm);
    PERCIS_CHECK_LAUNCH(ctx, "state keys");
    PERCIS_TRY(radix_sort_u64(ctx, k1, perm, k2, v2, n, 0, 64));
    k_gather_sorted<<<g, 256, 0, ctx->stream>>>(ctx->x.as<double>(), perm, n, ctx->xs.as<double>());
    PERCIS_CHECK_LAUNCH(ctx, "gather sorted");
    k_nonzero_prefix<<<1, 32, 0, ctx->stream>>>(ctx->xs.as<double>(), n, ctx->dscal.as<double>());
    PERCIS_CHECK_LAUNCH(ctx, "non-zero states");
    {
        // as many co-resident blocks as the non-zero states fill (read back: the launch
        // size is set on the host)
        long long nz = 0;
        PERCIS_CUDA(ctx, cudaMemcpyAsync(&nz, ctx->dscal.as<double>() + 2, sizeof(nz), cudaMemcpyDeviceToHost,
                                         ctx->stream));
        PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (ctx->table_grid == 0) {
            int per_sm = 0;
            PERCIS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tables, kScanThreads, 0));
            ctx->table_grid = std::min(kMaxTableBlocks, std::max(1, per_sm) * ctx->num_sms);
        }
        const int G = (int)std::max<long long>(1, std::min<long long>(ctx->table_grid, (nz + kScanChunk - 1) / kScanChunk));
        PERCIS_TRY(ensure(ctx, ctx->table_ctl, sizeof(TableCtl), "table control"));
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->table_ctl.p, 0, sizeof(TableCtl), ctx->stream));
        const double *xs = ctx->xs.as<double>();
        double *w = ctx->w.as<double>(), *ci = ctx->ci.as<double>(), *r = ctx->r.as<double>();
        double *dscal = ctx->dscal.as<double>();
        TableCtl *tctl = ctx->table_ctl.as<TableCtl>();
        uint64_t budget = (uint64_t)(ctx->opt.timeout_s * 1e9);
        int64_t nn = n;
        void *args[] = {&xs, &nn, &w, &ci, &r, &dscal, &tctl, &budget};
        PERCIS_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)k_tables, dim3(G), dim3(kScanThreads), args, 0,
                                                     ctx->stream));
        ctx->launches++;
        uint32_t tst = 0;
        PERCIS_CUDA(ctx, cudaMemcpyAsync(&tst, &tctl->status, 4, cudaMemcpyDeviceToHost, ctx->stream));
        PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (tst & DEV_TIMEOUT) return set_err(ctx, PERCIS_E_TIMEOUT, "table scan wait exceeded its budget");
    }
    PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->dscal.as<double>() + 1, 0, sizeof(double), ctx->stream));
    k_cv_lambda<<<g, 256, 0, ctx->stream>>>(ctx->xs.as<double>(), perm, ctx->w.as<double>(), ctx->dscal.as<double>(),
                                            n, ctx->Cv.as<double>(), ctx->lam.as<double>(), st);
    PERCIS_CHECK_LAUNCH(ctx, "cv lambda");
    k_max_lambda<<<g, 256, 0, ctx->stream>>>(ctx->lam.as<double>(), n, ctx->dscal.as<double>());
    PERCIS_CHECK_LAUNCH(ctx, "max lambda");
    ctx->groups_ready = false;  // built by the first backward pass that needs them
    double sc[2];
    uint32_t hst = 0;
    PERCIS_CUDA(ctx, cudaMemcpyAsync(sc, ctx->dscal.p, sizeof(sc), cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaMemcpyAsync(&hst, st, 4, cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (hst & DEV_BAD_STATE) return set_err(ctx, PERCIS_E_INVALID, "states must lie in [0,1] (no NaN)");
    ctx->c_host = sc[0];
    ctx->dhat_host = sc[1];
    if (hst & DEV_DEGENERATE)
        return set_err(ctx, PERCIS_E_DEGENERATE, "some C_v <= 0: percolation centrality undefined (all other states equal)");
    return PERCIS_OK;
}

// Tie groups of the sorted states (the backward pass's sums over C_u run over
// strictly smaller and strictly larger states), once per set of states.
percis_status prep_groups(percis_ctx *ctx) {
    if (ctx->groups_ready) return PERCIS_OK;
    const int64_t n = ctx->n;
    PERCIS_TRY(ensure(ctx, ctx->grp_lo, sizeof(int32_t) * n, "groups"));
    PERCIS_TRY(ensure(ctx, ctx->grp_hi, sizeof(int32_t) * n, "groups"));
    k_groups<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(ctx->xs.as<double>(), n, ctx->grp_lo.as<int32_t>(),
                                                             ctx->grp_hi.as<int32_t>());
    PERCIS_CHECK_LAUNCH(ctx, "tie groups");
    ctx->groups_ready = true;
    return PERCIS_OK;
}

}  // namespace percis
