// Exclusive prefix scans (reduce-then-scan, three kernels) used to group
// samples by source and by the backward pass.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace percis {

namespace {

constexpr int kScanBlock = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanBlock * kScanItems;

template <class T>
__device__ __forceinline__ T warp_incl(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        T o = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v += o;
    }
    return v;
}

// Exclusive scan of one value per thread across the block; *total = sum.
template <class T>
__device__ __forceinline__ T block_excl(T v, T *total) {
    __shared__ T ws[kScanBlock / 32];
    __shared__ T s_tot;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const T inc = warp_incl(v);
    T ex = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) ex = T(0);
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        const T s = lane < kScanBlock / 32 ? ws[lane] : T(0);
        const T si = warp_incl(s);
        T se = __shfl_up_sync(0xffffffffu, si, 1);
        if (lane == 0) se = T(0);
        if (lane < kScanBlock / 32) ws[lane] = se;
        if (lane == 31) s_tot = si;
    }
    __syncthreads();
    const T r = ws[warp] + ex;
    if (threadIdx.x == 0) *total = s_tot;
    __syncthreads();
    return r;
}

template <class T>
__global__ void k_tile_sums(const T *in, int64_t n, T *partial) {
    __shared__ T tot;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    block_excl(s, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <class T>
__global__ void k_scan_partials(T *partial, int64_t m, T *grand) {
    __shared__ T tot;
    T carry = 0;
    for (int64_t b = 0; b < m; b += kScanBlock) {
        const int64_t i = b + threadIdx.x;
        T v = i < m ? partial[i] : T(0);
        T ex = block_excl(v, &tot);
        if (i < m) partial[i] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && grand) *grand = carry;
}

template <class T>
__global__ void k_tile_scan(const T *in, T *out, int64_t n, const T *partial) {
    __shared__ T tot;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    T v[kScanItems];
    T s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? in[base + k] : T(0);
        s += v[k];
    }
    T ex = block_excl(s, &tot) + partial[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = ex;
        ex += v[k];
    }
}

template <class T>
percis_status scan_impl(percis_ctx *ctx, const T *in, T *out, int64_t n) {
    // out has n+1 slots: out[n] = total
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    PERCIS_TRY(ensure(ctx, ctx->scratch, sizeof(T) * (size_t)(tiles + 1) + 64, "scan scratch"));
    T *partial = ctx->scratch.as<T>();
    if (n == 0) {
        PERCIS_CUDA(ctx, cudaMemsetAsync(out, 0, sizeof(T), ctx->stream));
        return PERCIS_OK;
    }
    k_tile_sums<T><<<(unsigned)tiles, kScanBlock, 0, ctx->stream>>>(in, n, partial);
    PERCIS_CHECK_LAUNCH(ctx, "scan tile sums");
    k_scan_partials<T><<<1, kScanBlock, 0, ctx->stream>>>(partial, tiles, out + n);
    PERCIS_CHECK_LAUNCH(ctx, "scan partials");
    k_tile_scan<T><<<(unsigned)tiles, kScanBlock, 0, ctx->stream>>>(in, out, n, partial);
    PERCIS_CHECK_LAUNCH(ctx, "scan tiles");
    return PERCIS_OK;
}

}  // namespace

percis_status scan_exclusive_i64(percis_ctx *ctx, const int64_t *in, int64_t *out, int64_t n) {
    return scan_impl<long long>(ctx, (const long long *)in, (long long *)out, n);
}

percis_status scan_exclusive_f64(percis_ctx *ctx, const double *in, double *out, int64_t n) {
    return scan_impl<double>(ctx, in, out, n);
}

int grid_for(percis_ctx *ctx, int64_t work, int block) {
    int64_t g = (work + block - 1) / block;
    const int64_t cap = (int64_t)ctx->num_sms * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace percis
