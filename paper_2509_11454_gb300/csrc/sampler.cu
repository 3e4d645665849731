// Algorithm 2 pair sampling on the device and grouping of the sampled pairs
// by source (one BFS lane per distinct source in the batched form).
#include "common.cuh"
#include "internal.h"

namespace percis {

namespace {

// One thread per sample: Philox4x32-10 gives (u_s, u_t); two binary searches
// exactly as Algorithm 2 (appendix) over the 1-based tables, evaluated with
// explicit round-to-nearest operations so no multiply-add is fused.
__global__ void k_sample_pairs(int64_t n, const double *__restrict__ xs, const int32_t *__restrict__ perm,
                               const double *__restrict__ w, const double *__restrict__ ci,
                               const double *__restrict__ r, const double *__restrict__ dscal,
                               const double *__restrict__ x, uint64_t seed, const uint64_t *seed_dev, uint32_t tag,
                               int64_t i0, int64_t count, int32_t *s_out, int32_t *t_out, int32_t *kind) {
    const double c = dscal[0];
    if (seed_dev) seed = *seed_dev;  // a recorded launch reads the seed of the current call
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
        double us, ut;
        uniforms2(seed, (uint64_t)(i0 + k), tag, 0u, us, ut);
        int64_t a = 1, b = n, d = (a + b) >> 1;
        while (a <= b) {
            const double kk = __ddiv_rn(__dsub_rn(c, r[d + 1]), c);
            if (us <= kk) b = d - 1;
            else a = d + 1;
            d = (a + b) >> 1;
        }
        const int64_t s = b + 1;
        const double xss = xs[s - 1], wss = w[s], css = ci[s];
        a = s;
        b = n;
        d = (a + b) >> 1;
        while (a <= b) {
            const double num = __dadd_rn(__dsub_rn(__dmul_rn((double)(d - s + 1), xss), wss), w[d + 1]);
            const double kk = __ddiv_rn(num, css);
            if (ut <= kk) b = d - 1;
            else a = d + 1;
            d = (a + b) >> 1;
        }
        // t <= n whenever c_s > 0, which holds for every s the first search can
        // return; the clamp only keeps the index in bounds.
        const int64_t t = b + 1 <= n ? b + 1 : n;
        const int32_t sn = perm[s - 1], tn = perm[t - 1];
        if (s_out) s_out[k] = sn;
        if (t_out) t_out[k] = tn;
        if (kind) kind[k] = (__dsub_rn(x[sn], x[tn]) > 0.0) ? 0 : 1;
    }
}

__global__ void k_count_sources(const int32_t *s, const int32_t *kind, int64_t count, long long *src_count) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        if (kind[i] == 0) atomicAdd((unsigned long long *)&src_count[s[i]], 1ULL);
}

__global__ void k_head_flags(const long long *src_count, int64_t n, long long *head) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        head[v] = src_count[v] > 0 ? 1 : 0;
}

// Per-vertex quantities permuted into lane order (perm = vorder) and back.
__global__ void k_gather_ll(const long long *in, const int32_t *perm, int64_t n, long long *out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) out[k] = in[perm[k]];
}

__global__ void k_scatter_ll(const long long *in, const int32_t *perm, int64_t n, long long *out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += stride) out[perm[k]] = in[k];
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = in[n];
}

__global__ void k_scatter_samples(const int32_t *s, const int32_t *t, const int32_t *kind, int64_t count,
                                  const long long *src_off, const long long *lane_of_v, int32_t *src_fill,
                                  int32_t *sorted_samples, int32_t *samp_t, int32_t *samp_lane) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        if (kind[i] != 0) continue;
        const int32_t sv = s[i];
        const long long pos = src_off[sv] + atomicAdd(&src_fill[sv], 1);
        sorted_samples[pos] = (int32_t)i;
        samp_t[pos] = t[i];
        samp_lane[pos] = (int32_t)lane_of_v[sv];
    }
}

__global__ void k_lane_tables(const long long *src_count, const long long *src_off, const long long *lane_of_v,
                              int64_t n, int32_t *lane_src, long long *lane_off) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (src_count[v] > 0) {
            const long long lane = lane_of_v[v];
            lane_src[lane] = (int32_t)v;
            lane_off[lane] = src_off[v];
        }
        if (v == 0) lane_off[lane_of_v[n]] = src_off[n];
    }
}

}  // namespace

percis_status sample_pairs(percis_ctx *ctx, uint64_t seed, uint32_t tag, int64_t i0, int64_t count, int32_t *s,
                           int32_t *t, int32_t *kind, const uint64_t *seed_dev, cudaStream_t stream) {
    if (count <= 0) return PERCIS_OK;
    const int block = 256;
    k_sample_pairs<<<grid_for(ctx, count, block), block, 0, stream ? stream : ctx->stream>>>(
        ctx->n, ctx->xs.as<double>(), ctx->perm.as<int32_t>(), ctx->w.as<double>(), ctx->ci.as<double>(),
        ctx->r.as<double>(), ctx->dscal.as<double>(), ctx->x.as<double>(), seed, seed_dev, tag, i0, count, s, t,
        kind);
    PERCIS_CHECK_LAUNCH(ctx, "sample pairs");
    return PERCIS_OK;
}

// Group the valid samples of the last phase (pair_s, pair_t, kind) by source.
// Lane j (0 <= j < U) is the j-th distinct source in lane order (vertex id
// order, or the load-time vertex order that groups vertices by their
// highest-degree neighbour); its samples sit at positions lane_off[j] ..
// lane_off[j+1]-1 of sorted_samples.
percis_status group_by_source(percis_ctx *ctx, int64_t count, int64_t *n_sources, int64_t *n_valid) {
    const int64_t n = ctx->n;
    PERCIS_TRY(ensure(ctx, ctx->src_count, sizeof(long long) * (n + 1), "src count"));
    PERCIS_TRY(ensure(ctx, ctx->src_off, sizeof(long long) * (n + 1), "src off"));
    PERCIS_TRY(ensure(ctx, ctx->lane_of_v, sizeof(long long) * (n + 1), "lane of v"));
    PERCIS_TRY(ensure(ctx, ctx->src_fill, sizeof(int32_t) * (n + 1), "src fill"));
    PERCIS_TRY(ensure(ctx, ctx->sorted_samples, sizeof(int32_t) * (count + 1), "sorted samples"));
    PERCIS_TRY(ensure(ctx, ctx->samp_t, sizeof(int32_t) * (count + 1), "samp t"));
    PERCIS_TRY(ensure(ctx, ctx->samp_lane, sizeof(int32_t) * (count + 1), "samp lane"));
    PERCIS_TRY(ensure(ctx, ctx->lane_src, sizeof(int32_t) * (count + 1), "lane src"));
    PERCIS_TRY(ensure(ctx, ctx->lane_off, sizeof(long long) * (count + 2), "lane off"));
    long long *cnt = ctx->src_count.as<long long>();
    long long *off = ctx->src_off.as<long long>();
    long long *lov = ctx->lane_of_v.as<long long>();
    PERCIS_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(long long) * (n + 1), ctx->stream));
    PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->src_fill.p, 0, sizeof(int32_t) * (n + 1), ctx->stream));
    const int block = 256;
    k_count_sources<<<grid_for(ctx, count, block), block, 0, ctx->stream>>>(ctx->pair_s.as<int32_t>(),
                                                                          ctx->kind.as<int32_t>(), count, cnt);
    PERCIS_CHECK_LAUNCH(ctx, "count sources");
    PERCIS_TRY(ensure(ctx, ctx->red, sizeof(long long) * (2 * n + 2), "head scan"));
    long long *tmp = ctx->red.as<long long>();  // n+1 scratch
    long long *tmp2 = tmp + n + 1;              // n+1 scratch
    if (ctx->opt.lane_order == 1) {
        // sources in lane order: offsets and lane ids are scans over vorder
        PERCIS_TRY(prep_vorder(ctx));
        const int32_t *perm = ctx->vorder.as<int32_t>();
        k_gather_ll<<<grid_for(ctx, n, block), block, 0, ctx->stream>>>(cnt, perm, n, tmp2);
        PERCIS_CHECK_LAUNCH(ctx, "gather counts");
        PERCIS_TRY(scan_exclusive_i64(ctx, (const int64_t *)tmp2, (int64_t *)tmp, n));
        k_scatter_ll<<<grid_for(ctx, n, block), block, 0, ctx->stream>>>(tmp, perm, n, off);
        PERCIS_CHECK_LAUNCH(ctx, "scatter offsets");
        k_head_flags<<<grid_for(ctx, n, block), block, 0, ctx->stream>>>(tmp2, n, tmp2);
        PERCIS_CHECK_LAUNCH(ctx, "head flags");
        PERCIS_TRY(scan_exclusive_i64(ctx, (const int64_t *)tmp2, (int64_t *)tmp, n));
        k_scatter_ll<<<grid_for(ctx, n, block), block, 0, ctx->stream>>>(tmp, perm, n, lov);
        PERCIS_CHECK_LAUNCH(ctx, "scatter lanes");
    } else {
        PERCIS_TRY(scan_exclusive_i64(ctx, (const int64_t *)cnt, (int64_t *)off, n));
        k_head_flags<<<grid_for(ctx, n, block), block, 0, ctx->stream>>>(cnt, n, tmp2);
        PERCIS_CHECK_LAUNCH(ctx, "head flags");
        PERCIS_TRY(scan_exclusive_i64(ctx, (const int64_t *)tmp2, (int64_t *)lov, n));
    }
    k_scatter_samples<<<grid_for(ctx, count, block), block, 0, ctx->stream>>>(
        ctx->pair_s.as<int32_t>(), ctx->pair_t.as<int32_t>(), ctx->kind.as<int32_t>(), count, off, lov,
        ctx->src_fill.as<int32_t>(), ctx->sorted_samples.as<int32_t>(), ctx->samp_t.as<int32_t>(),
        ctx->samp_lane.as<int32_t>());
    PERCIS_CHECK_LAUNCH(ctx, "scatter samples");
    k_lane_tables<<<grid_for(ctx, n, block), block, 0, ctx->stream>>>(cnt, off, lov, n, ctx->lane_src.as<int32_t>(),
                                                                    ctx->lane_off.as<long long>());
    PERCIS_CHECK_LAUNCH(ctx, "lane tables");
    long long h[2];
    PERCIS_CUDA(ctx, cudaMemcpyAsync(&h[0], lov + n, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaMemcpyAsync(&h[1], off + n, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *n_sources = h[0];
    *n_valid = h[1];
    return PERCIS_OK;
}

}  // namespace percis
