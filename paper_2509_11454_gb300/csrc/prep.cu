// Preprocessing kernels: CSR validation and transpose, the stable sort of
// the percolation states, Algorithm 2's tables, C_v, lambda_v and d^.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace percis {

namespace {

// ------------------------------------------------------------- validation

__global__ void k_check_csr(const int64_t *rp, const int32_t *col, int64_t n, int64_t nnz, uint32_t *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (rp[v] > rp[v + 1] || rp[v] < 0 || rp[v + 1] > nnz) atomicOr(status, 1u);
        if (v == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicOr(status, 1u);
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const int32_t c = col[e];
        if (c < 0 || (int64_t)c >= n) atomicOr(status, 1u);
    }
}

__global__ void k_check_states(const double *x, int64_t n, uint32_t *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const double a = x[v];
        if (!(a >= 0.0 && a <= 1.0)) atomicOr(status, DEV_BAD_STATE);
    }
}

// ----------------------------------------------------------- merge sort
// Stable bottom-up merge sort of (key, val) pairs: in a pass of width w an
// element of the left run lands at (its rank in its run) + (number of
// right-run keys < key); an element of the right run at (its rank) +
// (number of left-run keys <= key).  Equal keys keep their input order.

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t *a, int64_t lo, int64_t hi, uint64_t key) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t upper_bound_u64(const uint64_t *a, int64_t lo, int64_t hi, uint64_t key) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] <= key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_merge_pass(const uint64_t *kin, const int32_t *vin, uint64_t *kout, int32_t *vout, int64_t n,
                             int64_t w) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t run = i / w;
        const uint64_t key = kin[i];
        int64_t out;
        if ((run & 1) == 0) {
            const int64_t a0 = run * w;
            const int64_t b0 = a0 + w;
            const int64_t b1 = min(b0 + w, n);
            const int64_t rank = b0 < n ? lower_bound_u64(kin, b0, b1, key) - b0 : 0;
            out = a0 + (i - a0) + rank;
        } else {
            const int64_t b0 = run * w;
            const int64_t a0 = b0 - w;
            out = a0 + (i - b0) + (upper_bound_u64(kin, a0, b0, key) - a0);
        }
        kout[out] = key;
        vout[out] = vin[i];
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
//    associatively, so one block-wide scan over them gives every running sum of a
//    chunk of terms at once.
//  - the first term whose sum reaches the top of the binade is added with one
//    hardware FP64 add, and the chunk restarts after it in the new binade (a
//    non-decreasing sum enters each binade once).
// Both evaluations give the correctly rounded sum of the same operands in the same
// order (IEEE 754 round to nearest, ties to even) at every step, hence equal results.
constexpr int kScanThreads = 1024;
constexpr int kScanPer = 4;  // terms per thread and chunk
constexpr int kScanChunk = kScanThreads * kScanPer;
constexpr unsigned long long kTwo53u = 1ull << 53;
constexpr int kNoTerm = 0x7fffffff;

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

// Running sums s_i = fl(s_{i+1} + a_i) for i = m down to 1 (s_{m+1} = +0), with
// a_i = src[i + soff] >= 0, written to dst[i]; returns s_1 (+0 when m = 0).  The
// whole block calls it.
__device__ double exact_running_sum(const double *src, int64_t soff, double *dst, int64_t m) {
    __shared__ ParityMap s_wmap[kScanThreads / 32];
    __shared__ int s_kstar[2];
    __shared__ double s_sum;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_kstar[0] = s_kstar[1] = kNoTerm;
    __syncthreads();
    double s = 0.0;
    int64_t pos = m;  // positions pos, pos - 1, ..., 1 remain; term k of a chunk sits at pos - k
    for (int pass = 0; pos > 0; ++pass) {
        const int cnt = pos < (int64_t)kScanChunk ? (int)pos : kScanChunk;
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
            const int k = tid * kScanPer + j;
            a[j] = k < cnt ? src[pos - k + soff] : 0.0;
            mine = pm_then(mine, term_map(a[j], e, q[j], kind[j]));
        }
        // scan of the maps: within the warp, then over the warps
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
        }
        __syncthreads();
        const ParityMap pre = pm_then(s_wmap[warp], exc);
        // this thread's terms under the true parity of S0
        const unsigned p0 = (unsigned)(S0 & 1ull);
        unsigned p = (pre.par >> p0) & 1u;
        unsigned long long acc = p0 ? pre.d1 : pre.d0;  // integer added before this thread's terms
        unsigned long long before[kScanPer];
        int first = kNoTerm;
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            const int k = tid * kScanPer + j;
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
            if (k < cnt && first == kNoTerm && (kind[j] == 3 || S0 + acc >= kTwo53u)) first = k;
        }
        const int slot = pass & 1;
        if (first != kNoTerm) atomicMin(&s_kstar[slot], first);
        __syncthreads();
        const int kstar = min(s_kstar[slot], cnt);  // terms before kstar stay in the binade
#pragma unroll
        for (int j = 0; j < kScanPer; ++j) {
            const int k = tid * kScanPer + j;
            const unsigned long long after = j + 1 < kScanPer ? before[j + 1] : acc;
            if (k < kstar) dst[pos - k] = __longlong_as_double((long long)(top + S0 + after));
            if (k == kstar - 1 && kstar == cnt) s_sum = __longlong_as_double((long long)(top + S0 + after));
            if (k == kstar && kstar < cnt) {
                // the term that leaves the binade: one hardware add from the sum before it
                const double prev = k == 0 ? s : __longlong_as_double((long long)(top + S0 + before[j]));
                const double nv = __dadd_rn(prev, a[j]);
                dst[pos - k] = nv;
                s_sum = nv;
            }
        }
        if (tid == 0) s_kstar[slot ^ 1] = kNoTerm;  // for the next pass
        __syncthreads();
        s = s_sum;
        pos -= kstar < cnt ? kstar + 1 : cnt;
    }
    return s;
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

__global__ void __launch_bounds__(kScanThreads) k_tables(const double *xs, int64_t n, double *w, double *ci,
                                                         double *r, double *dscal) {
    // positions past the last non-zero state: x_i = 0 and every sum before them
    // is +0, so w_i = c_i = r_i = 0 exactly; the scans start at the last non-zero one
    const int64_t nz = *reinterpret_cast<const long long *>(dscal + 2);
    for (int64_t i = nz + 1 + threadIdx.x; i <= n + 1; i += blockDim.x) w[i] = ci[i] = r[i] = 0.0;
    if (threadIdx.x == 0) w[0] = r[0] = ci[0] = 0.0;
    // w_i over x_i = xs[i - 1]
    exact_running_sum(xs, -1, w, nz);
    __syncthreads();
    for (int64_t i = 1 + threadIdx.x; i <= nz; i += blockDim.x) {
        const double t = __dmul_rn((double)(n - i + 1), xs[i - 1]);
        const double cv = __dsub_rn(t, w[i]);
        ci[i] = __double_as_longlong(cv) < 0 ? 0.0 : cv;  // max(0, .), -0 -> +0
    }
    __syncthreads();
    const double c = exact_running_sum(ci, 0, r, nz);
    if (threadIdx.x == 0) dscal[0] = c;  // c = r_1
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

__global__ void k_edge_keys(const int64_t *rp, const int32_t *col, int64_t n, uint64_t *keys, int32_t *vals) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
            keys[e] = ((uint64_t)(uint32_t)col[e] << 32) | (uint32_t)u;
            vals[e] = (int32_t)u;
        }
    }
}

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


__global__ void k_indeg(const int32_t *col, int64_t nnz, long long *cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
        atomicAdd((unsigned long long *)&cnt[col[e]], 1ULL);
}

}  // namespace

// Stable sort of (keys, vals) in place using the given scratch (same sizes).
static percis_status merge_sort(percis_ctx *ctx, uint64_t *keys, int32_t *vals, uint64_t *k2, int32_t *v2, int64_t n) {
    uint64_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    const int grid = grid_for(ctx, n, 256);
    for (int64_t w = 1; w < n; w <<= 1) {
        k_merge_pass<<<grid, 256, 0, ctx->stream>>>(ka, va, kb, vb, n, w);
        PERCIS_CHECK_LAUNCH(ctx, "merge pass");
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        PERCIS_CUDA(ctx, cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        PERCIS_CUDA(ctx, cudaMemcpyAsync(vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return PERCIS_OK;
}

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
            rs = merge_sort(ctx, k1.as<uint64_t>(), ctx->vorder.as<int32_t>(), k2.as<uint64_t>(), v2.as<int32_t>(), n);
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
    k_check_csr<<<grid_for(ctx, std::max(n, nnz), 256), 256, 0, ctx->stream>>>(ctx->rp.as<int64_t>(),
                                                                             ctx->col.as<int32_t>(), n, nnz, st);
    PERCIS_CHECK_LAUNCH(ctx, "check csr");
    uint32_t hst = 0;
    PERCIS_CUDA(ctx, cudaMemcpyAsync(&hst, st, 4, cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (hst) return set_err(ctx, PERCIS_E_INVALID, "malformed CSR (row_ptr not monotone or column out of range)");

    if (ctx->directed) {
        PERCIS_TRY(ensure(ctx, ctx->irp, sizeof(int64_t) * (n + 1), "in-CSR offsets"));
        PERCIS_TRY(ensure(ctx, ctx->icol, sizeof(int32_t) * std::max<int64_t>(nnz, 1), "in-CSR columns"));
        DevBuf k1, k2, v2;
        size_t kb = sizeof(uint64_t) * std::max<int64_t>(nnz, 1);
        cudaError_t e = cudaMalloc(&k1.p, kb);
        if (e == cudaSuccess) e = cudaMalloc(&k2.p, kb);
        if (e == cudaSuccess) e = cudaMalloc(&v2.p, sizeof(int32_t) * std::max<int64_t>(nnz, 1));
        percis_status rs = PERCIS_OK;
        if (e != cudaSuccess) {
            rs = set_err(ctx, PERCIS_E_OOM, "transpose scratch");
        } else {
            int32_t *icol = ctx->icol.as<int32_t>();
            k_edge_keys<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(ctx->rp.as<int64_t>(), ctx->col.as<int32_t>(),
                                                                      n, k1.as<uint64_t>(), icol);
            ctx->launches++;
            rs = merge_sort(ctx, k1.as<uint64_t>(), icol, k2.as<uint64_t>(), v2.as<int32_t>(), nnz);
            if (rs == PERCIS_OK) {
                long long *cnt = (long long *)ctx->irp.as<int64_t>();
                // in-degree counts into a temporary, then exclusive scan into irp
                DevBuf tmp;
                e = cudaMalloc(&tmp.p, sizeof(long long) * (n + 1));
                if (e != cudaSuccess) rs = set_err(ctx, PERCIS_E_OOM, "in-degree scratch");
                else {
                    cudaMemsetAsync(tmp.p, 0, sizeof(long long) * (n + 1), ctx->stream);
                    k_indeg<<<grid_for(ctx, nnz, 256), 256, 0, ctx->stream>>>(ctx->col.as<int32_t>(), nnz,
                                                                            tmp.as<long long>());
                    ctx->launches++;
                    rs = scan_exclusive_i64(ctx, tmp.as<int64_t>(), (int64_t *)cnt, n);
                    cudaStreamSynchronize(ctx->stream);
                    cudaFree(tmp.p);
                }
            }
        }
        cudaStreamSynchronize(ctx->stream);
        cudaFree(k1.p);
        cudaFree(k2.p);
        cudaFree(v2.p);
        if (rs != PERCIS_OK) return rs;
        PERCIS_CUDA(ctx, cudaGetLastError());
    }
    ctx->vorder_ready = false;  // built on first use by the batched form
    if (!ctx->skip_diam) {
        int64_t D = 0;
        PERCIS_TRY(vertex_diam_ub(ctx, &D));
        ctx->vertex_diam = D;
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
    PERCIS_TRY(ensure(ctx, ctx->grp_lo, sizeof(int32_t) * n, "groups"));
    PERCIS_TRY(ensure(ctx, ctx->grp_hi, sizeof(int32_t) * n, "groups"));
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
    PERCIS_TRY(merge_sort(ctx, k1, perm, k2, v2, n));
    k_gather_sorted<<<g, 256, 0, ctx->stream>>>(ctx->x.as<double>(), perm, n, ctx->xs.as<double>());
    PERCIS_CHECK_LAUNCH(ctx, "gather sorted");
    k_nonzero_prefix<<<1, 32, 0, ctx->stream>>>(ctx->xs.as<double>(), n, ctx->dscal.as<double>());
    PERCIS_CHECK_LAUNCH(ctx, "non-zero states");
    k_tables<<<1, kScanThreads, 0, ctx->stream>>>(ctx->xs.as<double>(), n, ctx->w.as<double>(),
                                                         ctx->ci.as<double>(), ctx->r.as<double>(),
                                                         ctx->dscal.as<double>());
    PERCIS_CHECK_LAUNCH(ctx, "tables");
    PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->dscal.as<double>() + 1, 0, sizeof(double), ctx->stream));
    k_cv_lambda<<<g, 256, 0, ctx->stream>>>(ctx->xs.as<double>(), perm, ctx->w.as<double>(), ctx->dscal.as<double>(),
                                            n, ctx->Cv.as<double>(), ctx->lam.as<double>(), st);
    PERCIS_CHECK_LAUNCH(ctx, "cv lambda");
    k_max_lambda<<<g, 256, 0, ctx->stream>>>(ctx->lam.as<double>(), n, ctx->dscal.as<double>());
    PERCIS_CHECK_LAUNCH(ctx, "max lambda");
    k_groups<<<g, 256, 0, ctx->stream>>>(ctx->xs.as<double>(), n, ctx->grp_lo.as<int32_t>(),
                                         ctx->grp_hi.as<int32_t>());
    PERCIS_CHECK_LAUNCH(ctx, "tie groups");
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

}  // namespace percis
