// Exact percolation centrality (Definition 1): every vertex is a source once.
// Sources go through the batched sigma-BFS in groups of up to 512 lanes (full
// traversals); then, level by level from the deepest, the dependencies of the
// extended Brandes recurrence
//   delta_s(v) = sum over w in out(v) at the next level of
//                (sigma_sv / sigma_sw) (R(x_s - x_w) + delta_s(w))
// are pulled over out-neighbours (one warp per vertex, lanes spread over the
// warp), and p(v) = sum_{s != v} delta_s(v) / C_v.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "internal.h"

namespace percis {

namespace {

template <int K, int SM>
__global__ void k_dependency(int64_t n, const int64_t *rp, const int32_t *col, const uint64_t *fh, int32_t L,
                             const void *sigma_v, double *delta, const double *x, const int32_t *lane_src,
                             int32_t nlanes, double *num) {
    constexpr int W = 64 * K;
    using ST = typename SigmaMode<SM>::ST;
    const ST *sigma = static_cast<const ST *>(sigma_v);
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nk = n * K;
    const uint64_t *fL = fh + (int64_t)L * nk;
    const uint64_t *fN = fh + (int64_t)(L + 1) * nk;
    for (int64_t v = gwarp; v < n; v += nwarps) {
        double vsum = 0.0;
        for (int w = 0; w < K; ++w) {
            const uint64_t bits = fL[v * K + w];
            if (!bits) continue;
            const int j0 = 64 * w + lane, j1 = j0 + 32;
            const bool b0 = (bits >> lane) & 1ull, b1 = (bits >> (lane + 32)) & 1ull;
            const double xs0 = (b0 && j0 < nlanes) ? x[lane_src[j0]] : 0.0;
            const double xs1 = (b1 && j1 < nlanes) ? x[lane_src[j1]] : 0.0;
            const double sv0 = b0 ? (double)sigma[v * W + j0] : 0.0;
            const double sv1 = b1 ? (double)sigma[v * W + j1] : 0.0;
            double a0 = 0.0, a1 = 0.0;
            for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
                const int32_t c = col[e];
                const uint64_t m = bits & fN[(int64_t)c * K + w];
                if (!m) continue;
                if ((m >> lane) & 1ull) {
                    const double cf = fmax(0.0, xs0 - x[c]) + delta[(int64_t)c * W + j0];
                    a0 += sv0 / (double)sigma[(int64_t)c * W + j0] * cf;
                }
                if ((m >> (lane + 32)) & 1ull) {
                    const double cf = fmax(0.0, xs1 - x[c]) + delta[(int64_t)c * W + j1];
                    a1 += sv1 / (double)sigma[(int64_t)c * W + j1] * cf;
                }
            }
            if (b0) delta[v * W + j0] = a0;
            if (b1) delta[v * W + j1] = a1;
            // sources contribute nothing to their own centrality
            if (b0 && j0 < nlanes && lane_src[j0] != v) vsum += a0;
            if (b1 && j1 < nlanes && lane_src[j1] != v) vsum += a1;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) vsum += __shfl_xor_sync(0xffffffffu, vsum, off);
        if (lane == 0 && vsum != 0.0) num[v] += vsum;
    }
}

__global__ void k_iota(int32_t *a, int64_t lo, int64_t cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += stride) a[i] = (int32_t)(lo + i);
}

__global__ void k_divide(const double *num, const double *Cv, int64_t n, double *pc) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) pc[v] = num[v] / Cv[v];
}

template <int K>
percis_status dependency_levels(percis_ctx *ctx, int levels, const void *sig, double *delta, const int32_t *src,
                                int32_t nlanes, double *num) {
    const int grid = grid_for(ctx, ctx->n * 32, 256);
    for (int L = levels; L >= 0; --L) {
        if (ctx->sigma_mode == 2)
            k_dependency<K, 2><<<grid, 256, 0, ctx->stream>>>(ctx->n, ctx->rp.as<int64_t>(), ctx->col.as<int32_t>(),
                                                            ctx->fhist.as<uint64_t>(), L, sig, delta,
                                                            ctx->x.as<double>(), src, nlanes, num);
        else if (ctx->sigma_mode == 1)
            k_dependency<K, 1><<<grid, 256, 0, ctx->stream>>>(ctx->n, ctx->rp.as<int64_t>(), ctx->col.as<int32_t>(),
                                                            ctx->fhist.as<uint64_t>(), L, sig, delta,
                                                            ctx->x.as<double>(), src, nlanes, num);
        else
            k_dependency<K, 0><<<grid, 256, 0, ctx->stream>>>(ctx->n, ctx->rp.as<int64_t>(), ctx->col.as<int32_t>(),
                                                            ctx->fhist.as<uint64_t>(), L, sig, delta,
                                                            ctx->x.as<double>(), src, nlanes, num);
        PERCIS_CHECK_LAUNCH(ctx, "dependency");
    }
    return PERCIS_OK;
}

}  // namespace

percis_status exact_pc(percis_ctx *ctx, double *pc) {
    const int64_t n = ctx->n;
    const int W = n >= 512 ? 512 : (n > 256 ? 512 : n > 128 ? 256 : n > 64 ? 128 : 64);
    PERCIS_TRY(ensure(ctx, ctx->pc_tmp, sizeof(double) * (size_t)n * (W + 1) + sizeof(int32_t) * 512, "exact scratch"));
    double *num = ctx->pc_tmp.as<double>();
    double *delta = num + n;
    int32_t *src = (int32_t *)(delta + (size_t)n * W);
    PERCIS_CUDA(ctx, cudaMemsetAsync(num, 0, sizeof(double) * n, ctx->stream));
    for (int64_t lo = 0; lo < n; lo += W) {
        const int32_t cnt = (int32_t)std::min<int64_t>(W, n - lo);
        k_iota<<<1, 512, 0, ctx->stream>>>(src, lo, cnt);
        PERCIS_CHECK_LAUNCH(ctx, "iota");
        // full traversals; msbfs_full rounds the lane width up to a power of two >= cnt
        PERCIS_TRY(msbfs_full(ctx, cnt, src, nullptr, nullptr));
        MsCtl hc;
        PERCIS_CUDA(ctx, cudaMemcpyAsync(&hc, ctx->ms_ctl.p, sizeof(hc), cudaMemcpyDeviceToHost, ctx->stream));
        PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        int Wl = 64;
        while (Wl < cnt) Wl *= 2;
        const int levels = hc.level;
        percis_status st;
        switch (Wl / 64) {
            case 1: st = dependency_levels<1>(ctx, levels, ctx->sigmaW.p, delta, src, cnt, num); break;
            case 2: st = dependency_levels<2>(ctx, levels, ctx->sigmaW.p, delta, src, cnt, num); break;
            case 4: st = dependency_levels<4>(ctx, levels, ctx->sigmaW.p, delta, src, cnt, num); break;
            default: st = dependency_levels<8>(ctx, levels, ctx->sigmaW.p, delta, src, cnt, num); break;
        }
        if (st != PERCIS_OK) return st;
    }
    k_divide<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(num, ctx->Cv.as<double>(), n, pc);
    PERCIS_CHECK_LAUNCH(ctx, "divide");
    return PERCIS_OK;
}

}  // namespace percis
