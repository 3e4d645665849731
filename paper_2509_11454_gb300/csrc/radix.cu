// Stable sorts of (key, int32 value) pairs -- an LSD radix sort, and a merge
// sort for small arrays -- and the directed graph's in-adjacency built with them.
//
// Each pass orders the pairs by one 8-bit digit of the key, stably, in three
// launches: per-tile digit counts (tiles of 4096 pairs), one exclusive scan of
// the counts laid out digit-major (so the scan gives every (digit, tile) its
// first output slot), and a scatter in which every tile ranks its pairs among
// equal digits in index order (per-warp ballot groups and counters), regroups
// them by digit in shared memory and writes each digit's run contiguously.
// Passes run from the lowest digit up, so the result is ordered by the key's
// sorted bits and, among equal keys, by input position.
//
// The in-adjacency of a directed CSR is the stable sort of its edges by
// target: the edges arrive ordered by source, so every in-list comes out
// ordered by source (the order the backtrack scans predecessors in).
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace percis {

namespace {

// tile shape (build-time tuning constants): threads per block, pairs per thread,
// resident scatter blocks per SM
#ifndef PERCIS_RADIX_BLOCK
#define PERCIS_RADIX_BLOCK 256
#endif
#ifndef PERCIS_RADIX_ROUNDS
#define PERCIS_RADIX_ROUNDS 16
#endif
#ifndef PERCIS_RADIX_MINB
#define PERCIS_RADIX_MINB 3
#endif
constexpr int kRadixBlock = PERCIS_RADIX_BLOCK;
constexpr int kRadixRounds = PERCIS_RADIX_ROUNDS;
constexpr int kRadixTile = kRadixBlock * kRadixRounds;
constexpr int kRadixBins = 256;
constexpr int kRadixWarps = kRadixBlock / 32;
static_assert(kRadixBlock % kRadixBins == 0, "every digit has a thread in the count scan");

template <class K>
__device__ __forceinline__ int digit_of(K key, int shift) {
    return (int)((key >> shift) & (K)(kRadixBins - 1));
}

// counts[d * ntiles + tile] = pairs of the tile whose digit is d.  A block takes
// kCountGroup consecutive tiles at a time, so each digit's counts of the group
// are written together (one sector instead of one per tile).
constexpr int kCountGroup = 4;

template <class K>
__global__ void __launch_bounds__(kRadixBlock) k_radix_count(const K *keys, int64_t n, int shift, int64_t ntiles,
                                                             long long *counts) {
    __shared__ int s_hist[kCountGroup][kRadixBins];
    const int64_t ngroups = (ntiles + kCountGroup - 1) / kCountGroup;
    for (int64_t grp = blockIdx.x; grp < ngroups; grp += gridDim.x) {
        for (int j = threadIdx.x; j < kCountGroup * kRadixBins; j += kRadixBlock) (&s_hist[0][0])[j] = 0;
        __syncthreads();
        const int64_t t0 = grp * kCountGroup;
        for (int g = 0; g < kCountGroup && t0 + g < ntiles; ++g) {
            const int64_t base = (t0 + g) * kRadixTile;
            K kk[kRadixRounds];  // the tile's keys loaded first, all in flight together
#pragma unroll
            for (int r = 0; r < kRadixRounds; ++r) {
                const int64_t i = base + (int64_t)r * kRadixBlock + threadIdx.x;
                kk[r] = i < n ? keys[i] : K(0);
            }
#pragma unroll
            for (int r = 0; r < kRadixRounds; ++r)
                if (base + (int64_t)r * kRadixBlock + threadIdx.x < n) atomicAdd(&s_hist[g][digit_of(kk[r], shift)], 1);
        }
        __syncthreads();
        for (int d = threadIdx.x; d < kRadixBins; d += kRadixBlock)
            for (int g = 0; g < kCountGroup && t0 + g < ntiles; ++g) counts[(int64_t)d * ntiles + t0 + g] = s_hist[g][d];
        __syncthreads();
    }
}

// Pairs of each tile to offs[d * ntiles + tile] + (rank among the tile's earlier
// pairs of digit d).  Warp w ranks the tile's pairs [512 w, 512 w + 512) among
// equal digits with warp-private counters (no block barrier), the per-digit
// counts of the warps then give every pair its place in the tile ordered by
// digit, stably; the pairs are regrouped so in shared memory and written out
// in that order, so the writes of one digit's run are contiguous.
template <class K>
constexpr size_t scatter_smem() {
    return (sizeof(K) + sizeof(int32_t)) * kRadixTile + sizeof(int) * kRadixWarps * kRadixBins +
           sizeof(long long) * kRadixBins + sizeof(int) * kRadixBins + sizeof(int) * kRadixWarps;
}

template <class K>
__global__ void __launch_bounds__(kRadixBlock, PERCIS_RADIX_MINB) k_radix_scatter(const K *kin, const int32_t *vin, K *kout,
                                                                  int32_t *vout, int64_t n, int shift,
                                                                  int64_t ntiles, const long long *offs) {
    extern __shared__ __align__(16) unsigned char s_raw[];
    K *sk = reinterpret_cast<K *>(s_raw);
    int32_t *sv = reinterpret_cast<int32_t *>(sk + kRadixTile);
    int *s_wc = reinterpret_cast<int *>(sv + kRadixTile);  // [warp][digit]
    long long *s_base = reinterpret_cast<long long *>(s_wc + kRadixWarps * kRadixBins);
    int *s_lpre = reinterpret_cast<int *>(s_base + kRadixBins);
    int *s_wtot = s_lpre + kRadixBins;
    constexpr int kPerWarp = kRadixTile / kRadixWarps;
    constexpr int kRounds = kPerWarp / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    int *wc = s_wc + warp * kRadixBins;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * kRadixTile;
        const int64_t wbase = base + (int64_t)warp * kPerWarp;
        for (int d = lane; d < kRadixBins; d += 32) wc[d] = 0;
        K key[kRounds];
        int32_t val[kRounds];
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            const int64_t i = wbase + r * 32 + lane;
            key[r] = i < n ? kin[i] : K(0);
            val[r] = i < n ? vin[i] : 0;
        }
        __syncwarp();
        int rk[kRounds];
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            const bool valid = wbase + r * 32 + lane < n;
            const int d = valid ? digit_of(key[r], shift) : 0;
            // lanes with the same digit (and validity): one ballot per digit bit
            const unsigned vm = __ballot_sync(0xffffffffu, valid);
            unsigned peers = valid ? vm : ~vm;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const unsigned bb = __ballot_sync(0xffffffffu, (d >> b) & 1);
                peers &= ((d >> b) & 1) ? bb : ~bb;
            }
            const int lead = __ffs(peers) - 1;
            int run = (valid && lane == lead) ? wc[d] : 0;
            run = __shfl_sync(0xffffffffu, run, lead);
            rk[r] = run + __popc(peers & lt);
            __syncwarp();
            if (valid && lane == lead) wc[d] = run + __popc(peers);
            __syncwarp();
        }
        __syncthreads();
        {
            // digit d = this thread (the first kRadixBins threads): its count in the
            // tile, its first place in the tile (exclusive scan over the digits), and
            // each warp's first place among it
            const int d = threadIdx.x;
            const bool dt = d < kRadixBins;  // (whole warps)
            int wpre[kRadixWarps];
            int c = 0, inc = 0;
            if (dt) {
#pragma unroll
                for (int w = 0; w < kRadixWarps; ++w) {
                    wpre[w] = c;
                    c += s_wc[w * kRadixBins + d];
                }
                inc = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int t2 = __shfl_up_sync(0xffffffffu, inc, o);
                    if (lane >= o) inc += t2;
                }
                if (lane == 31) s_wtot[warp] = inc;
                s_base[d] = offs[(int64_t)d * ntiles + tile];
            }
            __syncthreads();
            if (dt) {
                int lp = inc - c;
                for (int q = 0; q < warp; ++q) lp += s_wtot[q];
                s_lpre[d] = lp;
#pragma unroll
                for (int w = 0; w < kRadixWarps; ++w) s_wc[w * kRadixBins + d] = lp + wpre[w];
            }
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            if (wbase + r * 32 + lane < n) {
                const int pos = wc[digit_of(key[r], shift)] + rk[r];
                sk[pos] = key[r];
                sv[pos] = val[r];
            }
        }
        __syncthreads();
        const int cnt = (int)(n - base < (int64_t)kRadixTile ? n - base : (int64_t)kRadixTile);
        for (int p = threadIdx.x; p < cnt; p += kRadixBlock) {
            const K k = sk[p];
            const int d = digit_of(k, shift);
            const long long g = s_base[d] + (p - s_lpre[d]);
            kout[g] = k;
            vout[g] = sv[p];
        }
        __syncthreads();  // the tile's shared arrays are reused by the next
    }
}

// src[e] = the row of edge e: a warp takes 32 consecutive rows (their offsets
// loaded together) and writes them one after the other, all lanes on each row,
// so long rows are spread over the lanes and short ones cost one step each
__global__ void k_edge_rows(const int64_t *rp, int64_t n, int32_t *src) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; u0 < n; u0 += warps * 32) {
        const int64_t u = u0 + lane;
        const int64_t b = u < n ? rp[u] : 0, e = u < n ? rp[u + 1] : 0;
        for (int r = 0; r < 32; ++r) {
            const int64_t e0 = __shfl_sync(0xffffffffu, b, r), e1 = __shfl_sync(0xffffffffu, e, r);
            for (int64_t x = e0 + lane; x < e1; x += 32) src[x] = (int32_t)(u0 + r);
        }
    }
}

// irp[v] = first position of target v in the sorted targets (= nnz past the last):
// position e writes irp[v] for every v in (tgt[e-1], tgt[e]], and e = nnz the tail
__global__ void k_offsets_from_sorted(const uint32_t *tgt, int64_t nnz, int64_t n, int64_t *irp) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e <= nnz; e += stride) {
        const int64_t lo = e == 0 ? 0 : (int64_t)tgt[e - 1] + 1;
        const int64_t hi = e == nnz ? n : (int64_t)tgt[e];
        for (int64_t v = lo; v <= hi; ++v) irp[v] = e;
    }
}

// Small arrays: a bottom-up merge sort of whole 64-bit keys (log2 n passes of
// one launch each) beats eight radix passes of five launches.  In a pass of
// width w every element finds its output slot by a binary search in the
// neighbouring run (ties: the left run first, so the sort is stable).
__device__ __forceinline__ int64_t lower_bound_u64(const unsigned long long *a, int64_t lo, int64_t hi,
                                                   unsigned long long key) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t upper_bound_u64(const unsigned long long *a, int64_t lo, int64_t hi,
                                                   unsigned long long key) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] <= key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_merge_pass(const unsigned long long *kin, const int32_t *vin, unsigned long long *kout,
                             int32_t *vout, int64_t n, int64_t w) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t run = i / w;
        const unsigned long long key = kin[i];
        int64_t out;
        if ((run & 1) == 0) {  // left run: after the right run's keys that are smaller
            const int64_t a0 = run * w, b0 = a0 + w, b1 = min(b0 + w, n);
            out = i + (b0 < n ? lower_bound_u64(kin, b0, b1, key) - b0 : 0);
        } else {  // right run: after the left run's keys that are not larger
            const int64_t b0 = run * w, a0 = b0 - w;
            out = a0 + (i - b0) + (upper_bound_u64(kin, a0, b0, key) - a0);
        }
        kout[out] = key;
        vout[out] = vin[i];
    }
}

constexpr int64_t kMergeMaxN = 1 << 18;

int radix_grid(percis_ctx *ctx, int64_t ntiles) {
    const int64_t cap = (int64_t)ctx->num_sms * 8;
    return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, cap));
}

// keys_in, when given, is the first pass's input instead of keys (which is then
// only scratch): the pass does not modify its input.
template <class K>
percis_status radix_sort_impl(percis_ctx *ctx, K *keys, int32_t *vals, K *tk, int32_t *tv, int64_t n, int lo_bit,
                              int bits, K **out_keys, int32_t **out_vals, const K *keys_in = nullptr) {
    *out_keys = keys_in ? const_cast<K *>(keys_in) : keys;
    *out_vals = vals;
    if (n <= 1 || bits <= 0) return PERCIS_OK;
    const int64_t ntiles = (n + kRadixTile - 1) / kRadixTile;
    const int64_t nc = ntiles * kRadixBins;
    PERCIS_TRY(ensure(ctx, ctx->radix_counts, sizeof(long long) * (size_t)(nc + 1), "radix counts"));
    long long *counts = ctx->radix_counts.as<long long>();
    const int grid = radix_grid(ctx, ntiles);
    if (scatter_smem<K>() > 48 * 1024)
        PERCIS_CUDA(ctx, cudaFuncSetAttribute(k_radix_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)scatter_smem<K>()));
    K *ka = keys, *kb = tk;
    int32_t *va = vals, *vb = tv;
    for (int shift = lo_bit; shift < lo_bit + bits; shift += 8) {
        const K *kin = (shift == lo_bit && keys_in) ? keys_in : ka;
        k_radix_count<K><<<grid, kRadixBlock, 0, ctx->stream>>>(kin, n, shift, ntiles, counts);
        PERCIS_CHECK_LAUNCH(ctx, "radix count");
        PERCIS_TRY(scan_exclusive_i64(ctx, (const int64_t *)counts, (int64_t *)counts, nc));
        k_radix_scatter<K><<<grid, kRadixBlock, scatter_smem<K>(), ctx->stream>>>(kin, va, kb, vb, n, shift, ntiles,
                                                                                   counts);
        PERCIS_CHECK_LAUNCH(ctx, "radix scatter");
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    *out_keys = ka;
    *out_vals = va;
    return PERCIS_OK;
}

}  // namespace

percis_status radix_sort_u64(percis_ctx *ctx, uint64_t *keys, int32_t *vals, uint64_t *tk, int32_t *tv, int64_t n,
                             int lo_bit, int bits) {
    uint64_t *ok = keys;
    int32_t *ov = vals;
    if (n <= kMergeMaxN && lo_bit == 0 && bits == 64) {
        unsigned long long *ka = (unsigned long long *)keys, *kb = (unsigned long long *)tk;
        int32_t *va = vals, *vb = tv;
        const int grid = grid_for(ctx, n, 256);
        for (int64_t w = 1; w < n; w <<= 1) {
            k_merge_pass<<<grid, 256, 0, ctx->stream>>>(ka, va, kb, vb, n, w);
            PERCIS_CHECK_LAUNCH(ctx, "merge pass");
            std::swap(ka, kb);
            std::swap(va, vb);
        }
        ok = (uint64_t *)ka;
        ov = va;
    } else {
        PERCIS_TRY(radix_sort_impl<unsigned long long>(ctx, (unsigned long long *)keys, vals,
                                                       (unsigned long long *)tk, tv, n, lo_bit, bits,
                                                       (unsigned long long **)&ok, &ov));
    }
    if (ok != keys) {
        PERCIS_CUDA(ctx, cudaMemcpyAsync(keys, ok, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        PERCIS_CUDA(ctx, cudaMemcpyAsync(vals, ov, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return PERCIS_OK;
}

// In-adjacency of the loaded directed CSR: irp (int64[n+1]) and icol (int32[nnz],
// every in-list ordered by source).
// The in-adjacency in two steps: the sort of the edges by target (valid row
// offsets needed; any column values are sorted in bounds), then the offsets
// (valid columns needed).
percis_status transpose_sort(percis_ctx *ctx) {
    const int64_t n = ctx->n, nnz = ctx->nnz;
    PERCIS_TRY(ensure(ctx, ctx->irp, sizeof(int64_t) * (n + 1), "in-CSR offsets"));
    PERCIS_TRY(ensure(ctx, ctx->icol, sizeof(int32_t) * std::max<int64_t>(nnz, 1), "in-CSR columns"));
    if (nnz == 0) {
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->irp.p, 0, sizeof(int64_t) * (n + 1), ctx->stream));
        return PERCIS_OK;
    }
    // scratch (grow-only, kept in the context): two key arrays and one value array
    const size_t kb = sizeof(uint32_t) * (size_t)nnz;
    PERCIS_TRY(ensure(ctx, ctx->sort_a, 2 * kb, "transpose keys"));
    PERCIS_TRY(ensure(ctx, ctx->sort_b, kb, "transpose values"));
    int bits = 1;
    while (bits < 32 && (1ll << bits) < n) ++bits;
    // the values ping-pong between icol and the scratch array once per pass: start
    // them where an even number of passes leaves them in icol (no final copy)
    const int passes = (bits + 7) / 8;
    uint32_t *k1 = ctx->sort_a.as<uint32_t>(), *k2 = k1 + nnz;
    int32_t *v1 = ctx->icol.as<int32_t>(), *v2 = ctx->sort_b.as<int32_t>();
    if (passes & 1) std::swap(v1, v2);
    k_edge_rows<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(ctx->rp.as<int64_t>(), n, v1);
    PERCIS_CHECK_LAUNCH(ctx, "edge rows");
    uint32_t *ok;
    int32_t *ov;
    // the columns are the first pass's keys as they are
    PERCIS_TRY(radix_sort_impl<unsigned int>(ctx, k1, v1, k2, v2, nnz, 0, bits, &ok, &ov,
                                             reinterpret_cast<const uint32_t *>(ctx->col.as<int32_t>())));
    if (ov != ctx->icol.as<int32_t>())
        PERCIS_CUDA(ctx, cudaMemcpyAsync(ctx->icol.as<int32_t>(), ov, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice,
                                         ctx->stream));
    ctx->tr_sorted_keys = ok;
    return PERCIS_OK;
}

percis_status transpose_finish(percis_ctx *ctx) {
    const int64_t n = ctx->n, nnz = ctx->nnz;
    if (nnz == 0) return PERCIS_OK;  // (irp zeroed by transpose_sort)
    k_offsets_from_sorted<<<grid_for(ctx, nnz + 1, 256), 256, 0, ctx->stream>>>(ctx->tr_sorted_keys, nnz, n,
                                                                               ctx->irp.as<int64_t>());
    PERCIS_CHECK_LAUNCH(ctx, "in-CSR offsets");
    return PERCIS_OK;
}

}  // namespace percis
