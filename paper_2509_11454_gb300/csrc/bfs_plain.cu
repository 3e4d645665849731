// Plain form of RandomSP (Section III-B): for every sampled pair one
// cooperative launch runs a level-synchronous sigma-counting BFS from s over
// the whole GPU (frontier queues, warp per frontier vertex), truncated once
// t's level is discovered, then one single-warp launch backtracks a uniform
// shortest path.  This is the baseline the batched form is measured against.
// It also serves VertexDiamUB and the single-source BFS inspection call.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace percis {

namespace {

constexpr int kPlainBlock = 256;

struct PlainArgs {
    int64_t n;
    const int64_t *rp;
    const int32_t *col;
    const int64_t *irp;
    const int32_t *icol;
    int32_t *ep;  // epoch stamp: vertex discovered in the current BFS iff ep[v] == epoch
    int32_t *lvl;
    double *sigma;
    int32_t *qa;
    int32_t *qb;
    PlainCtl *ctl;
    const int32_t *s_dev;
    const int32_t *t_dev;
    const int32_t *kind;
    int64_t idx;
    int32_t s_host, t_host;
    int32_t epoch;
    int32_t levels_only;  // levels (eccentricity) only: no path counts
    uint64_t budget_ns;
};

__global__ void __launch_bounds__(kPlainBlock) k_plain_bfs(PlainArgs a) {
    const int32_t s = a.s_dev ? a.s_dev[a.idx] : a.s_host;
    const int32_t t = a.t_dev ? a.t_dev[a.idx] : a.t_host;
    if (a.kind && a.kind[a.idx] != 0) return;  // zero-weight pair: no path needed (uniform over the grid)
    PlainCtl *ctl = a.ctl;
    GridBarrier *bar = reinterpret_cast<GridBarrier *>(ctl);
    uint32_t *status = &ctl->status;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ep[s] = a.epoch;
        a.lvl[s] = 0;
        a.sigma[s] = 1.0;
        a.qa[0] = s;
        ctl->qsize[0] = 1;
        ctl->qsize[1] = 0;
        ctl->qsize[2] = 0;
        ctl->level = 0;
        ctl->found = 0;
    }
    if (!grid_sync(bar, status, a.budget_ns)) return;
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int32_t *cur = a.qa, *nxt = a.qb;
    int L = 0, ecc = 0;
    // a target equal to the source is settled at level 0: nothing to expand
    for (; t < 0 || t != s;) {
        const int nq = (int)ld_relaxed_u32((const uint32_t *)&ctl->qsize[L % 3]);
        // the slot level L + 2 will fill: last read before the previous barrier
        if (blockIdx.x == 0 && threadIdx.x == 0) ctl->qsize[(L + 2) % 3] = 0;
        // expand level L: claim undiscovered out-neighbours
        for (int64_t k = gwarp; k < nq; k += nwarps) {
            const int32_t u = __ldcg(&cur[k]);
            const int64_t e0 = a.rp[u], e1 = a.rp[u + 1];
            for (int64_t base = e0; base < e1; base += 32) {
                const int64_t e = base + lane;
                bool mine = false;
                int32_t v = 0;
                if (e < e1) {
                    v = a.col[e];
                    if (__ldcg(&a.ep[v]) != a.epoch) mine = atomicMax(&a.ep[v], a.epoch) < a.epoch;
                }
                const unsigned m = __ballot_sync(0xffffffffu, mine);
                if (m) {
                    const int leader = __ffs(m) - 1;
                    int base_pos = 0;
                    if (lane == leader) base_pos = atomicAdd(&ctl->qsize[(L + 1) % 3], __popc(m));
                    base_pos = __shfl_sync(0xffffffffu, base_pos, leader);
                    if (mine) {
                        const int pos = base_pos + __popc(m & ((1u << lane) - 1u));
                        nxt[pos] = v;
                        a.lvl[v] = L + 1;
                    }
                }
            }
        }
        if (!grid_sync(bar, status, a.budget_ns)) return;
        const int nn = (int)ld_relaxed_u32((const uint32_t *)&ctl->qsize[(L + 1) % 3]);
        // sigma of the new level: pull over in-neighbours at level L
        for (int64_t k = gwarp; k < nn && !a.levels_only; k += nwarps) {
            const int32_t wv = __ldcg(&nxt[k]);
            const int64_t e0 = a.irp[wv], e1 = a.irp[wv + 1];
            double acc = 0.0;
            for (int64_t e = e0 + lane; e < e1; e += 32) {
                const int32_t u = a.icol[e];
                if (__ldcg(&a.ep[u]) == a.epoch && __ldcg(&a.lvl[u]) == L) acc += __ldcg(&a.sigma[u]);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) {
                a.sigma[wv] = acc;
                if (acc >= kTwo53) atomicOr(status, DEV_SIGMA_OVERFLOW);
                if (wv == t) atomicExch(&ctl->found, 1);
            }
        }
        // (levels only: no target, so the exit test below reads nn alone)
        if (!a.levels_only && !grid_sync(bar, status, a.budget_ns)) return;
        ++L;
        if (nn > 0) ecc = L;
        if (nn == 0) break;
        // Exit tests read only values that stay fixed until every block has
        // passed the next barrier: qsize of this level and the sticky found
        // flag (ep[t] itself may be claimed by a faster block in the next
        // level's expansion, which would split the grid).
        if (t >= 0 && ld_relaxed_u32((const uint32_t *)&ctl->found)) break;
        int32_t *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->level = ecc;
        ctl->qsize[0] = 0;
        ctl->qsize[1] = 0;
        ctl->qsize[2] = 0;
    }
}

// Backtrack of one sample with one warp: from w = t, draw u in (0,1] and
// move to the first predecessor (in-adjacency order) whose running sigma sum
// reaches u * sigma_w.  The running sums are exact (integers below 2^53), so a
// warp-parallel scan picks the same predecessor as a sequential scan.
__global__ void k_plain_backtrack(const int64_t *irp, const int32_t *icol, const int32_t *ep, const int32_t *lvl,
                                  const double *sigma, int32_t epoch, const int32_t *s_arr, const int32_t *t_arr,
                                  int32_t *kind, int64_t idx, uint64_t seed, uint32_t tag, int32_t *ilen,
                                  long long *path_off, int32_t *arena, unsigned long long *arena_top,
                                  int64_t arena_cap, unsigned long long *cnt, uint32_t *status) {
    const int lane = threadIdx.x & 31;
    const int32_t s = s_arr[idx], t = t_arr[idx];
    if (kind[idx] != 0 || ep[t] != epoch) {
        if (lane == 0) {
            if (kind[idx] == 0) kind[idx] = 2;
            ilen[idx] = 0;
            path_off[idx] = 0;
        }
        return;
    }
    const int32_t d = lvl[t];
    const int32_t len = d - 1;
    unsigned long long off = 0;
    if (lane == 0) {
        off = atomicAdd(arena_top, (unsigned long long)len);
        ilen[idx] = len;
        path_off[idx] = (long long)off;
        if ((int64_t)(off + len) > arena_cap) atomicOr(status, DEV_ARENA_OVERFLOW);
    }
    off = __shfl_sync(0xffffffffu, off, 0);
    const bool store = (int64_t)(off + len) <= arena_cap;
    int32_t w = t;
    int32_t lw = d;
    uint32_t step = 0;
    int32_t k = 0;
    while (w != s) {
        const double target = __dmul_rn(uniform_at(seed, (uint64_t)idx, tag, step), sigma[w]);
        const int64_t e0 = irp[w], e1 = irp[w + 1];
        double carry = 0.0;
        int32_t pick = -1;
        for (int64_t base = e0; base < e1 && pick < 0; base += 32) {
            const int64_t e = base + lane;
            int32_t p = -1;
            double val = 0.0;
            if (e < e1) {
                p = icol[e];
                if (ep[p] == epoch && lvl[p] == lw - 1) val = sigma[p];
            }
            const double cum = __dadd_rn(carry, warp_inclusive_scan(val));
            const unsigned hit = __ballot_sync(0xffffffffu, val > 0.0 && cum >= target);
            if (hit) pick = __shfl_sync(0xffffffffu, p, __ffs(hit) - 1);
            carry = __shfl_sync(0xffffffffu, cum, 31);
        }
        if (pick < 0) {
            if (lane == 0) atomicOr(status, DEV_BAD_PATH);
            return;
        }
        if (pick != s) {
            if (lane == 0) {
                if (store) arena[off + k] = pick;
                atomicAdd(&cnt[pick], 1ULL);
            }
            ++k;
        }
        w = pick;
        --lw;
        ++step;
    }
}

__global__ void k_dist_sigma(const int32_t *ep, const int32_t *lvl, const double *sigma, int32_t epoch, int64_t n,
                             int32_t *dist, double *sig) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const bool in = ep[v] == epoch;
        if (dist) dist[v] = in ? lvl[v] : -1;
        if (sig) sig[v] = in ? sigma[v] : 0.0;
    }
}

__global__ void k_argmax_degree(const int64_t *rp, const int32_t *ep, const int32_t *seen_epoch_lo, int64_t n,
                                unsigned long long *best) {
    // key = (degree << 32) | (~v): max degree, ties to the smallest id
    unsigned long long m = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t dg = rp[v + 1] - rp[v];
        if (dg > 0 && ep[v] < *seen_epoch_lo) {
            const unsigned long long key = ((unsigned long long)dg << 32) | (0xffffffffu - (uint32_t)v);
            m = m > key ? m : key;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, off);
        m = m > o ? m : o;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(best, m);
}

}  // namespace

static percis_status ensure_plain(percis_ctx *ctx) {
    const int64_t n = ctx->n;
    const bool fresh = ctx->ep.bytes < sizeof(int32_t) * (size_t)n;
    PERCIS_TRY(ensure(ctx, ctx->ep, sizeof(int32_t) * n, "ep"));
    PERCIS_TRY(ensure(ctx, ctx->lvl, sizeof(int32_t) * n, "lvl"));
    PERCIS_TRY(ensure(ctx, ctx->sigma1, sizeof(double) * n, "sigma"));
    PERCIS_TRY(ensure(ctx, ctx->qa, sizeof(int32_t) * n, "queue"));
    PERCIS_TRY(ensure(ctx, ctx->qb, sizeof(int32_t) * n, "queue"));
    PERCIS_TRY(ensure(ctx, ctx->plain_ctl, 256, "plain ctl"));
    if (fresh || ctx->epoch <= 0 || ctx->epoch > (1 << 30)) {
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->ep.p, 0, sizeof(int32_t) * n, ctx->stream));
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->plain_ctl.p, 0, 256, ctx->stream));
        ctx->epoch = 0;
    }
    if (ctx->plain_grid == 0) {  // co-resident blocks on this context's device
        int per_sm = 0;
        PERCIS_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plain_bfs, kPlainBlock, 0));
        ctx->plain_grid = std::max(1, per_sm) * ctx->num_sms;
    }
    return PERCIS_OK;
}

percis_status plain_bfs(percis_ctx *ctx, const int32_t *s_dev, const int32_t *t_dev, int64_t idx, int32_t s_host,
                        int32_t t_host, bool levels_only) {
    PERCIS_TRY(ensure_plain(ctx));
    ctx->epoch++;
    PlainArgs a;
    a.n = ctx->n;
    a.rp = ctx->rp.as<int64_t>();
    a.col = ctx->col.as<int32_t>();
    a.irp = ctx->directed ? ctx->irp.as<int64_t>() : ctx->rp.as<int64_t>();
    a.icol = ctx->directed ? ctx->icol.as<int32_t>() : ctx->col.as<int32_t>();
    a.ep = ctx->ep.as<int32_t>();
    a.lvl = ctx->lvl.as<int32_t>();
    a.sigma = ctx->sigma1.as<double>();
    a.qa = ctx->qa.as<int32_t>();
    a.qb = ctx->qb.as<int32_t>();
    a.ctl = ctx->plain_ctl.as<PlainCtl>();
    a.s_dev = s_dev;
    a.t_dev = t_dev;
    a.kind = s_dev ? ctx->kind.as<int32_t>() : nullptr;
    a.idx = idx;
    a.s_host = s_host;
    a.t_host = t_host;
    a.epoch = ctx->epoch;
    a.levels_only = levels_only ? 1 : 0;
    a.budget_ns = (uint64_t)(ctx->opt.timeout_s * 1e9);
    void *args[] = {&a};
    PERCIS_CUDA(ctx, cudaLaunchCooperativeKernel((const void *)k_plain_bfs, dim3(ctx->plain_grid), dim3(kPlainBlock),
                                                 args, 0, ctx->stream));
    ctx->launches++;
    return PERCIS_OK;
}

percis_status plain_backtrack(percis_ctx *ctx, uint64_t seed, uint32_t tag, int64_t idx) {
    k_plain_backtrack<<<1, 32, 0, ctx->stream>>>(
        ctx->directed ? ctx->irp.as<int64_t>() : ctx->rp.as<int64_t>(),
        ctx->directed ? ctx->icol.as<int32_t>() : ctx->col.as<int32_t>(), ctx->ep.as<int32_t>(),
        ctx->lvl.as<int32_t>(), ctx->sigma1.as<double>(), ctx->epoch, ctx->pair_s.as<int32_t>(),
        ctx->pair_t.as<int32_t>(), ctx->kind.as<int32_t>(), idx, seed, tag, ctx->ilen.as<int32_t>(),
        ctx->path_off.as<long long>(), ctx->arena.as<int32_t>(), ctx->arena_top.as<unsigned long long>(),
        ctx->arena_cap, ctx->cnt.as<unsigned long long>(), &ctx->plain_ctl.as<PlainCtl>()->status);
    PERCIS_CHECK_LAUNCH(ctx, "plain backtrack");
    return PERCIS_OK;
}

percis_status plain_phase(percis_ctx *ctx, uint64_t seed, uint32_t tag_path, int64_t count) {
    for (int64_t i = 0; i < count; ++i) {
        PERCIS_TRY(plain_bfs(ctx, ctx->pair_s.as<int32_t>(), ctx->pair_t.as<int32_t>(), i, 0, 0));
        PERCIS_TRY(plain_backtrack(ctx, seed, tag_path, i));
    }
    return PERCIS_OK;
}

percis_status plain_dist_sigma(percis_ctx *ctx, int32_t *dist, double *sigma) {
    k_dist_sigma<<<grid_for(ctx, ctx->n, 256), 256, 0, ctx->stream>>>(
        ctx->ep.as<int32_t>(), ctx->lvl.as<int32_t>(), ctx->sigma1.as<double>(), ctx->epoch, ctx->n, dist, sigma);
    PERCIS_CHECK_LAUNCH(ctx, "dist sigma");
    return PERCIS_OK;
}

// VertexDiamUB: for undirected graphs, one full BFS from the largest-degree
// vertex of every component (ties to the smallest id); D = max(2 ecc - 1, 0).
// Directed graphs: D = n - 2.
percis_status vertex_diam_ub(percis_ctx *ctx, int64_t *D) {
    const int64_t n = ctx->n;
    if (ctx->directed) {
        *D = n >= 2 ? n - 2 : 0;
        return PERCIS_OK;
    }
    PERCIS_TRY(ensure_plain(ctx));
    PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->plain_ctl.p, 0, sizeof(PlainCtl), ctx->stream));
    // vertices of earlier components carry epochs >= first_epoch
    const int32_t first_epoch = ctx->epoch + 1;
    PERCIS_TRY(ensure(ctx, ctx->red, 64, "argmax"));
    int32_t *lo_dev = (int32_t *)(ctx->red.as<unsigned long long>() + 1);
    PERCIS_CUDA(ctx, cudaMemcpyAsync(lo_dev, &first_epoch, sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    int64_t best_D = 0;
    for (int64_t comp = 0; comp < n; ++comp) {
        unsigned long long key = 0;
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->red.p, 0, sizeof(unsigned long long), ctx->stream));
        k_argmax_degree<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(
            ctx->rp.as<int64_t>(), ctx->ep.as<int32_t>(), lo_dev, n, ctx->red.as<unsigned long long>());
        PERCIS_CHECK_LAUNCH(ctx, "argmax degree");
        PERCIS_CUDA(ctx, cudaMemcpyAsync(&key, ctx->red.p, sizeof(key), cudaMemcpyDeviceToHost, ctx->stream));
        PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (key == 0) break;
        const int32_t v = (int32_t)(0xffffffffu - (uint32_t)(key & 0xffffffffu));
        PERCIS_TRY(plain_bfs(ctx, nullptr, nullptr, 0, v, -1, true));
        PlainCtl hc;
        PERCIS_CUDA(ctx, cudaMemcpyAsync(&hc, ctx->plain_ctl.p, sizeof(hc), cudaMemcpyDeviceToHost, ctx->stream));
        PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        if (hc.status & DEV_TIMEOUT) return set_err(ctx, PERCIS_E_TIMEOUT, "VertexDiamUB BFS timed out");
        const int64_t b = 2 * (int64_t)hc.level - 1;
        best_D = std::max(best_D, b);
    }
    *D = best_D;
    return PERCIS_OK;
}

}  // namespace percis
