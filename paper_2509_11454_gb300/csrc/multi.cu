// Many independent graphs in one context.  Each graph is its own instance of
// the problem of Section II (own C, lambda, d^, vertex-diameter bound, l1 and
// l), kept in a sub-context that does its own state preprocessing, pair
// sampling, bounds, finalisation and backward pass with the single-graph
// kernels.  The union context holds the block-diagonal CSR and runs the
// sigma-counting BFS of all graphs together: the sampled sources of every
// graph are grouped into lanes, and consecutive lanes share one batched
// launch over the vertex range of their graphs.
//
// Sample numbering: in each phase, graph g's samples carry the indices
// off_g .. off_g + count_g - 1, off_g being the sum of the sample counts of
// graphs 0 .. g-1, in the Philox counters of the pair and path draws.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace percis {

struct MultiGraph {
    int32_t G = 0;
    std::vector<int64_t> vptr;          // G + 1 vertex offsets
    std::vector<percis_ctx *> subs;     // one context per graph (shares the union's stream)
    std::vector<int64_t> counts, soff;  // per-graph sample counts of the current phase, offsets (G + 1)
    std::vector<int32_t> lane_src_host;
    int64_t range = 0;                  // vertex range of the batch buffers
    DevBuf gid;                         // graph of every vertex
    DevBuf vptr_dev;                    // first vertex id of every graph (device)
    int64_t largest = 0;
    DevBuf soff_dev, ell_dev, stats, pmax;
    bool paths_scattered = false;
    // recorded per-graph sampling launches of each phase (pair tag 0 / 1), the
    // counts they were recorded for, and the device word they read the seed from
    cudaGraphExec_t samp_exec[2] = {nullptr, nullptr};
    std::vector<int64_t> samp_key[2];
    DevBuf seed_dev;
    int64_t graph_launches = 0, graph_records = 0;
};

namespace {

void drop_graph(MultiGraph *m, int k) {
    if (m->samp_exec[k]) cudaGraphExecDestroy(m->samp_exec[k]);
    m->samp_exec[k] = nullptr;
    m->samp_key[k].clear();
}

__global__ void k_offset_ids(int32_t *s, int32_t *t, int64_t count, int32_t delta) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        s[i] += delta;
        t[i] += delta;
    }
}

__device__ __forceinline__ int32_t graph_of_sample(const long long *soff, int32_t G, long long i) {
    int32_t lo = 0, hi = G;  // soff[lo] <= i < soff[hi]
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (soff[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

// per graph: sum |I|, sum |I|^2, zero-weight samples, unreachable targets
__global__ void k_stats_multi(int64_t count, const long long *soff, int32_t G, const int32_t *kind,
                              const int32_t *ilen, unsigned long long *acc) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const int32_t g = graph_of_sample(soff, G, i);
        const int32_t k = kind[i];
        const unsigned long long l = (unsigned long long)ilen[i];
        if (k == 0) {
            if (l) {
                atomicAdd(&acc[4 * g + 0], l);
                atomicAdd(&acc[4 * g + 1], l * l);
            }
        } else if (k == 1) {
            atomicAdd(&acc[4 * g + 2], 1ull);
        } else {
            atomicAdd(&acc[4 * g + 3], 1ull);
        }
    }
}

// per graph: max_v lambda_v cnt_v / l_g (non-negative, so the bit patterns order like the values)
__global__ void k_pmax_multi(const double *lam, const unsigned long long *cnt, const double *acc, const int32_t *gid,
                             const double *ell, int64_t n, unsigned long long *pmax) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int32_t g = gid[v];
        const double p = lam[v] * (acc ? acc[v] : (double)cnt[v]) / ell[g];
        if (p > 0.0) atomicMax(&pmax[g], (unsigned long long)__double_as_longlong(p));
    }
}

__global__ void k_finalize_multi(const double *lam, const unsigned long long *cnt, const double *acc,
                                 const int32_t *gid, const double *ell, int64_t n, double *pc) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        pc[v] = lam[v] * (acc ? acc[v] : (double)cnt[v]) / ell[gid[v]];
}

// a graph's samples of the last phase in its own context: local ids, paths
// re-packed in sample order
__global__ void k_local_paths(const int32_t *ilen, const long long *src_off, const int32_t *arena, int64_t count,
                              const long long *dst_off, int32_t *dst, int32_t delta) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const int32_t l = ilen[i];
        const long long a = src_off[i], b = dst_off[i];
        for (int32_t k = 0; k < l; ++k) dst[b + k] = arena[a + k] - delta;
    }
}

__global__ void k_ilen64(const int32_t *ilen, int64_t count, long long *out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) out[i] = ilen[i];
}

}  // namespace

void multi_free(percis_ctx *ctx) {
    if (!ctx->multi) return;
    MultiGraph *m = ctx->multi;
    drop_graph(m, 0);
    drop_graph(m, 1);
    for (percis_ctx *sub : m->subs) percis_destroy(sub);
    DevBuf *bufs[] = {&m->gid, &m->soff_dev, &m->ell_dev, &m->stats, &m->pmax, &m->seed_dev, &m->vptr_dev};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    delete m;
    ctx->multi = nullptr;
}

int64_t multi_range(percis_ctx *ctx) { return ctx->multi ? ctx->multi->range : ctx->n; }

void multi_graph_view(percis_ctx *ctx, const int32_t **gid, const int64_t **vbase, int64_t *largest) {
    MultiGraph *m = ctx->multi;
    *gid = m->gid.as<int32_t>();
    *vbase = m->vptr_dev.as<int64_t>();
    *largest = m->largest;
}

void multi_set_options(percis_ctx *ctx) {
    if (!ctx->multi) return;
    for (percis_ctx *sub : ctx->multi->subs) sub->opt = ctx->opt;
}

namespace {

// the per-graph launches of one phase's pair sampling
percis_status issue_sampling(percis_ctx *ctx, uint64_t seed, uint32_t tag, const uint64_t *seed_dev) {
    MultiGraph *m = ctx->multi;
    for (int32_t g = 0; g < m->G; ++g) {
        const int64_t c = m->counts[g];
        if (c == 0) continue;
        int32_t *s = ctx->pair_s.as<int32_t>() + m->soff[g];
        int32_t *t = ctx->pair_t.as<int32_t>() + m->soff[g];
        int32_t *kd = ctx->kind.as<int32_t>() + m->soff[g];
        percis_ctx *sub = m->subs[g];
        const percis_status st = sample_pairs(sub, seed, tag, m->soff[g], c, s, t, kd, seed_dev, ctx->stream);
        if (st != PERCIS_OK) return set_err(ctx, st, "graph " + std::to_string(g) + ": " + sub->err);
        k_offset_ids<<<grid_for(ctx, c, 256), 256, 0, ctx->stream>>>(s, t, c, (int32_t)m->vptr[g]);
        PERCIS_CHECK_LAUNCH(ctx, "offset ids");
    }
    return PERCIS_OK;
}

}  // namespace

percis_status multi_sample_pairs(percis_ctx *ctx, uint64_t seed, uint32_t tag) {
    MultiGraph *m = ctx->multi;
    if (!ctx->opt.cuda_graphs || tag > 1) return issue_sampling(ctx, seed, tag, nullptr);
    // CUDA graph: the G sampling launches (and their id offsets) recorded once per
    // count vector and replayed; the seed travels through a device word
    PERCIS_TRY(ensure(ctx, m->seed_dev, 64, "seed word"));
    PERCIS_CUDA(ctx, cudaMemcpyAsync(m->seed_dev.p, &seed, sizeof(seed), cudaMemcpyHostToDevice, ctx->stream));
    const int k = (int)tag;
    // the recorded launches bake in the buffers' addresses: re-record when counts or buffers change
    std::vector<int64_t> key = m->counts;
    key.push_back((int64_t)(uintptr_t)ctx->pair_s.p);
    key.push_back((int64_t)(uintptr_t)ctx->pair_t.p);
    key.push_back((int64_t)(uintptr_t)ctx->kind.p);
    if (!m->samp_exec[k] || m->samp_key[k] != key) {
        drop_graph(m, k);
        cudaGraph_t graph = nullptr;
        PERCIS_CUDA(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        const percis_status st = issue_sampling(ctx, seed, tag, m->seed_dev.as<uint64_t>());
        const cudaError_t ec = cudaStreamEndCapture(ctx->stream, &graph);
        if (st != PERCIS_OK) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        if (ec != cudaSuccess) return cuda_err(ctx, ec, "end of the sampling capture");
        const cudaError_t ei = cudaGraphInstantiate(&m->samp_exec[k], graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            m->samp_exec[k] = nullptr;
            return cuda_err(ctx, ei, "instantiating the sampling graph");
        }
        m->samp_key[k] = key;
        m->graph_records++;
    }
    PERCIS_CUDA(ctx, cudaGraphLaunch(m->samp_exec[k], ctx->stream));
    m->graph_launches++;
    return PERCIS_OK;
}

percis_status multi_plan_batches(percis_ctx *ctx, int64_t n_sources, int W, std::vector<LaneBatch> *out) {
    MultiGraph *m = ctx->multi;
    m->lane_src_host.resize((size_t)n_sources);
    PERCIS_CUDA(ctx, cudaMemcpyAsync(m->lane_src_host.data(), ctx->lane_src.p, sizeof(int32_t) * n_sources,
                                     cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    out->clear();
    auto graph_of = [&](int32_t v) {
        return (int32_t)(std::upper_bound(m->vptr.begin(), m->vptr.end(), (int64_t)v) - m->vptr.begin() - 1);
    };
    int64_t j = 0;
    while (j < n_sources) {
        // lanes come in lane order, which keeps each graph's sources together
        const int32_t g0 = graph_of(m->lane_src_host[j]);
        int32_t glast = g0;
        int64_t k = j + 1;
        while (k < n_sources && k - j < W) {
            const int32_t g = graph_of(m->lane_src_host[k]);
            const int32_t lo = std::min(g0, g), hi = std::max(glast, g);
            if (m->vptr[hi + 1] - m->vptr[lo] > m->range) break;
            glast = std::max(glast, g);
            ++k;
        }
        int32_t glo = g0, ghi = g0;
        for (int64_t q = j; q < k; ++q) {
            const int32_t g = graph_of(m->lane_src_host[q]);
            glo = std::min(glo, g);
            ghi = std::max(ghi, g);
        }
        out->push_back({(int32_t)j, (int32_t)(k - j), (int32_t)m->vptr[glo], m->vptr[ghi + 1] - m->vptr[glo]});
        j = k;
    }
    return PERCIS_OK;
}

}  // namespace percis

using namespace percis;

namespace {

percis_status need_multi(percis_ctx *ctx, bool states) {
    if (!ctx) return PERCIS_E_INVALID;
    if (!ctx->multi) return set_err(ctx, PERCIS_E_STATE, "no graphs loaded with percis_load_graphs");
    if (states && !ctx->have_states) return set_err(ctx, PERCIS_E_STATE, "no states set");
    return PERCIS_OK;
}

// per-graph statistics of the phase just run (counts already in the union context)
percis_status multi_stats(percis_ctx *ctx, const std::vector<double> &ell, std::vector<unsigned long long> *acc,
                          std::vector<double> *pmax) {
    MultiGraph *m = ctx->multi;
    const int32_t G = m->G;
    PERCIS_TRY(ensure(ctx, m->stats, sizeof(unsigned long long) * 4 * G, "graph stats"));
    PERCIS_TRY(ensure(ctx, m->pmax, sizeof(unsigned long long) * G, "graph pmax"));
    PERCIS_TRY(ensure(ctx, m->ell_dev, sizeof(double) * G, "graph l"));
    PERCIS_CUDA(ctx, cudaMemsetAsync(m->stats.p, 0, sizeof(unsigned long long) * 4 * G, ctx->stream));
    PERCIS_CUDA(ctx, cudaMemsetAsync(m->pmax.p, 0, sizeof(unsigned long long) * G, ctx->stream));
    PERCIS_CUDA(ctx, cudaMemcpyAsync(m->ell_dev.p, ell.data(), sizeof(double) * G, cudaMemcpyHostToDevice, ctx->stream));
    const int64_t total = m->soff[G];
    if (total > 0) {
        k_stats_multi<<<grid_for(ctx, total, 256), 256, 0, ctx->stream>>>(
            total, m->soff_dev.as<long long>(), G, ctx->kind.as<int32_t>(), ctx->ilen.as<int32_t>(),
            m->stats.as<unsigned long long>());
        PERCIS_CHECK_LAUNCH(ctx, "graph stats");
    }
    k_pmax_multi<<<grid_for(ctx, ctx->n, 256), 256, 0, ctx->stream>>>(
        ctx->lam.as<double>(), ctx->cnt.as<unsigned long long>(),
        ctx->opt.estimator == 1 ? ctx->acc_ap.as<double>() : nullptr, m->gid.as<int32_t>(), m->ell_dev.as<double>(),
        ctx->n, m->pmax.as<unsigned long long>());
    PERCIS_CHECK_LAUNCH(ctx, "graph pmax");
    acc->resize(4 * (size_t)G);
    std::vector<unsigned long long> pb((size_t)G);
    PERCIS_CUDA(ctx, cudaMemcpyAsync(acc->data(), m->stats.p, sizeof(unsigned long long) * 4 * G,
                                     cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaMemcpyAsync(pb.data(), m->pmax.p, sizeof(unsigned long long) * G, cudaMemcpyDeviceToHost,
                                     ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    pmax->resize((size_t)G);
    for (int32_t g = 0; g < G; ++g) memcpy(&(*pmax)[g], &pb[g], sizeof(double));
    return PERCIS_OK;
}

percis_status multi_phase(percis_ctx *ctx, uint64_t seed, int phase, const std::vector<int64_t> &counts,
                          PhaseOut *po) {
    MultiGraph *m = ctx->multi;
    m->counts = counts;
    m->soff.assign((size_t)m->G + 1, 0);
    for (int32_t g = 0; g < m->G; ++g) m->soff[g + 1] = m->soff[g] + counts[g];
    PERCIS_TRY(ensure(ctx, m->soff_dev, sizeof(long long) * (m->G + 1), "sample offsets"));
    PERCIS_CUDA(ctx, cudaMemcpyAsync(m->soff_dev.p, m->soff.data(), sizeof(long long) * (m->G + 1),
                                     cudaMemcpyHostToDevice, ctx->stream));
    m->paths_scattered = false;
    const int64_t total = m->soff[m->G];
    return run_phase(ctx, seed, phase, std::max<int64_t>(total, 1), po);
}

}  // namespace

extern "C" percis_status percis_load_graphs(percis_ctx *ctx, int32_t num_graphs, const int64_t *graph_vptr, int64_t n,
                                            int64_t nnz, const int64_t *row_ptr, const int32_t *col, int directed) {
    if (!ctx) return PERCIS_E_INVALID;
    if (num_graphs < 1 || !graph_vptr || !row_ptr || (nnz > 0 && !col))
        return set_err(ctx, PERCIS_E_INVALID, "need num_graphs >= 1 and host arrays");
    if (graph_vptr[0] != 0 || graph_vptr[num_graphs] != n)
        return set_err(ctx, PERCIS_E_INVALID, "graph_vptr must run from 0 to n");
    for (int32_t g = 0; g < num_graphs; ++g)
        if (graph_vptr[g + 1] - graph_vptr[g] < 2)
            return set_err(ctx, PERCIS_E_INVALID, "graph " + std::to_string(g) + " has fewer than 2 vertices");
    if (row_ptr[0] != 0 || row_ptr[n] != nnz) return set_err(ctx, PERCIS_E_INVALID, "row_ptr must run from 0 to nnz");
    for (int32_t g = 0; g < num_graphs; ++g) {
        const int64_t lo = graph_vptr[g], hi = graph_vptr[g + 1];
        for (int64_t v = lo; v < hi; ++v) {
            if (row_ptr[v + 1] < row_ptr[v]) return set_err(ctx, PERCIS_E_INVALID, "row_ptr not monotone");
            for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e)
                if (col[e] < lo || col[e] >= hi)
                    return set_err(ctx, PERCIS_E_INVALID,
                                   "edge leaves its graph (graph " + std::to_string(g) + ", vertex " +
                                       std::to_string(v) + ")");
        }
    }
    multi_free(ctx);
    // the union: block-diagonal CSR for the batched BFS (its own bound is the max over graphs)
    ctx->skip_diam = true;
    percis_status st = percis_load_csr(ctx, n, nnz, row_ptr, col, directed, 0);
    ctx->skip_diam = false;
    if (st != PERCIS_OK) return st;
    ctx->have_graph = false;
    MultiGraph *m = new MultiGraph();
    m->G = num_graphs;
    m->vptr.assign(graph_vptr, graph_vptr + num_graphs + 1);
    int64_t D = 0, largest = 0;
    std::vector<int64_t> lrp;
    for (int32_t g = 0; g < num_graphs && st == PERCIS_OK; ++g) {
        const int64_t lo = graph_vptr[g], hi = graph_vptr[g + 1], ng = hi - lo;
        largest = std::max(largest, ng);
        percis_ctx *sub = nullptr;
        st = percis_create(&sub, ctx->device, ctx->stream);
        if (st != PERCIS_OK) break;
        m->subs.push_back(sub);
        sub->opt = ctx->opt;
        lrp.resize((size_t)ng + 1);
        for (int64_t v = 0; v <= ng; ++v) lrp[v] = row_ptr[lo + v] - row_ptr[lo];
        std::vector<int32_t> lcol((size_t)std::max<int64_t>(1, lrp[ng]));
        for (int64_t e = 0; e < lrp[ng]; ++e) lcol[e] = col[row_ptr[lo] + e] - (int32_t)lo;
        st = percis_load_csr(sub, ng, lrp[ng], lrp.data(), lcol.data(), directed, 0);
        if (st != PERCIS_OK) st = set_err(ctx, st, "graph " + std::to_string(g) + ": " + sub->err);
        else D = std::max(D, sub->vertex_diam);
    }
    if (st != PERCIS_OK) {
        ctx->multi = m;
        multi_free(ctx);
        return st;
    }
    ctx->vertex_diam = D;
    // batch buffers span at least the largest graph (and small graphs together)
    m->range = std::min<int64_t>(n, std::max<int64_t>(largest, 1 << 18));
    std::vector<int32_t> gid((size_t)n);
    for (int32_t g = 0; g < num_graphs; ++g)
        std::fill(gid.begin() + graph_vptr[g], gid.begin() + graph_vptr[g + 1], g);
    ctx->multi = m;
    m->largest = largest;
    PERCIS_TRY(ensure(ctx, m->gid, sizeof(int32_t) * n, "graph ids"));
    PERCIS_CUDA(ctx, cudaMemcpyAsync(m->gid.p, gid.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, ctx->stream));
    PERCIS_TRY(ensure(ctx, m->vptr_dev, sizeof(int64_t) * (num_graphs + 1), "graph offsets"));
    PERCIS_CUDA(ctx, cudaMemcpyAsync(m->vptr_dev.p, graph_vptr, sizeof(int64_t) * (num_graphs + 1),
                                     cudaMemcpyHostToDevice, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->have_graph = true;
    return PERCIS_OK;
}

extern "C" int32_t percis_num_graphs(percis_ctx *ctx) { return ctx && ctx->multi ? ctx->multi->G : 0; }

percis_status percis::percis_multi_set_states(percis_ctx *ctx, const double *x, int on_device) {
    PERCIS_TRY(need_multi(ctx, false));
    MultiGraph *m = ctx->multi;
    ctx->have_states = false;
    ctx->have_paths = false;
    const int64_t n = ctx->n;
    PERCIS_TRY(ensure(ctx, ctx->x, sizeof(double) * n, "x"));
    PERCIS_TRY(ensure(ctx, ctx->lam, sizeof(double) * n, "lambda"));
    PERCIS_CUDA(ctx, cudaMemcpyAsync(ctx->x.p, x, sizeof(double) * n,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    for (int32_t g = 0; g < m->G; ++g) {
        percis_ctx *sub = m->subs[g];
        const int64_t lo = m->vptr[g], ng = m->vptr[g + 1] - lo;
        const percis_status st = percis_set_states(sub, ctx->x.as<double>() + lo, 1);
        if (st != PERCIS_OK) return set_err(ctx, st, "graph " + std::to_string(g) + ": " + sub->err);
        PERCIS_CUDA(ctx, cudaMemcpyAsync(ctx->lam.as<double>() + lo, sub->lam.p, sizeof(double) * ng,
                                         cudaMemcpyDeviceToDevice, ctx->stream));
    }
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->have_states = true;
    return PERCIS_OK;
}

extern "C" percis_status percis_estimate_graphs(percis_ctx *ctx, double eps, double delta, uint64_t seed,
                                                double *pc_out, int pc_on_device, percis_info *info) {
    PERCIS_TRY(need_multi(ctx, true));
    if (!(eps > 0.0 && eps < 1.0) || !(delta > 0.0 && delta < 1.0) || !pc_out)
        return set_err(ctx, PERCIS_E_INVALID, "eps and delta must lie in (0,1); pc_out must be non-NULL");
    if (ctx->opt.form == PERCIS_FORM_PLAIN)
        return set_err(ctx, PERCIS_E_INVALID, "many graphs run in the batched or bidirectional form");
    MultiGraph *m = ctx->multi;
    const int32_t G = m->G;
    const int64_t launches0 = ctx->launches;
    const bool di = ctx->opt.data_independent != 0;
    const int64_t ell1 = di ? 0 : (ctx->opt.ell1 > 0 ? ctx->opt.ell1 : ell1_default(eps, delta));
    std::vector<percis_info> inf((size_t)G);
    memset(inf.data(), 0, sizeof(percis_info) * G);
    std::vector<unsigned long long> acc;
    std::vector<double> pmax((size_t)G, 0.0);
    PhaseOut po1, po2;
    if (!di) {
        PERCIS_TRY(multi_phase(ctx, seed, 0, std::vector<int64_t>((size_t)G, ell1), &po1));
        PERCIS_TRY(multi_stats(ctx, std::vector<double>((size_t)G, (double)ell1), &acc, &pmax));
    } else {
        acc.assign(4 * (size_t)G, 0ull);
    }
    std::vector<int64_t> ells((size_t)G);
    for (int32_t g = 0; g < G; ++g) {
        percis_ctx *sub = m->subs[g];
        percis_info &f = inf[g];
        f.n = sub->n;
        f.nnz = sub->nnz;
        f.C = sub->c_host;
        f.dhat = sub->dhat_host;
        const int64_t D = ctx->opt.vertex_diam >= 0 ? ctx->opt.vertex_diam : sub->vertex_diam;
        f.vertex_diam = D;
        f.ell1 = ell1;
        f.zero_weight[0] = (int64_t)acc[4 * g + 2];
        f.unreachable[0] = (int64_t)acc[4 * g + 3];
        f.sum_internal[0] = (int64_t)acc[4 * g + 0];
        const Bounds b = compute_bounds(eps, delta, sub->dhat_host, D, ell1, (int64_t)acc[4 * g + 0],
                                        (int64_t)acc[4 * g + 1], pmax[g], di ? 1 : 0);
        f.rho_tilde = b.rho_tilde;
        f.Lambda = b.Lambda;
        f.rho_hat = b.rho_hat;
        f.v_hat = b.v_hat;
        f.x_hat = b.x_hat;
        f.p1_max = pmax[g];
        ells[g] = ctx->opt.ell > 0 ? ctx->opt.ell : b.ell;
        f.ell = ells[g];
    }
    PERCIS_TRY(multi_phase(ctx, seed, 1, ells, &po2));
    std::vector<double> elld(ells.begin(), ells.end());
    std::vector<unsigned long long> acc2;
    std::vector<double> pm2;
    PERCIS_TRY(multi_stats(ctx, elld, &acc2, &pm2));
    double *dst = pc_out;
    if (!pc_on_device) {
        PERCIS_TRY(ensure(ctx, ctx->pc_tmp, sizeof(double) * ctx->n, "pc staging"));
        dst = ctx->pc_tmp.as<double>();
    }
    k_finalize_multi<<<grid_for(ctx, ctx->n, 256), 256, 0, ctx->stream>>>(
        ctx->lam.as<double>(), ctx->cnt.as<unsigned long long>(),
        ctx->opt.estimator == 1 ? ctx->acc_ap.as<double>() : nullptr, m->gid.as<int32_t>(), m->ell_dev.as<double>(),
        ctx->n, dst);
    PERCIS_CHECK_LAUNCH(ctx, "finalize graphs");
    if (!pc_on_device)
        PERCIS_CUDA(ctx, cudaMemcpyAsync(pc_out, dst, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->last_ell = 1;
    ctx->last_seed = seed;
    if (info) {
        for (int32_t g = 0; g < G; ++g) {
            percis_info &f = inf[g];
            f.zero_weight[1] = (int64_t)acc2[4 * g + 2];
            f.unreachable[1] = (int64_t)acc2[4 * g + 3];
            f.sum_internal[1] = (int64_t)acc2[4 * g + 0];
            // launches are shared by all graphs: every entry reports the totals
            f.sources[0] = po1.sources;
            f.sources[1] = po2.sources;
            f.batches[0] = po1.batches;
            f.batches[1] = po2.batches;
            f.bfs_ms[0] = po1.bfs_ms;
            f.bfs_ms[1] = po2.bfs_ms;
            f.bfs_launches[0] = po1.bfs_launches;
            f.bfs_launches[1] = po2.bfs_launches;
            f.sigma_overflow = po1.overflow | po2.overflow;
            f.lanes = ctx->lanes_alloc;
            f.kernel_launches = ctx->launches - launches0;
            info[g] = f;
        }
    }
    return PERCIS_OK;
}

// Backward of the last many-graph estimate: each graph's samples move to its
// context (local ids, paths in sample order), then the single-graph adjoint.
percis_status percis::percis_multi_backward(percis_ctx *ctx, const double *grad_pc, double *grad_x, int on_device) {
    PERCIS_TRY(need_multi(ctx, true));
    MultiGraph *m = ctx->multi;
    if (!ctx->have_paths || ctx->last_phase != 1)
        return set_err(ctx, PERCIS_E_NO_SAMPLE, "backward needs a completed estimate of the one-path form");
    const int64_t n = ctx->n;
    const double *gd = grad_pc;
    double *gx = grad_x;
    if (!on_device) {
        PERCIS_TRY(ensure(ctx, ctx->grad_tmp, sizeof(double) * 2 * n, "gradient staging"));
        PERCIS_CUDA(ctx, cudaMemcpyAsync(ctx->grad_tmp.p, grad_pc, sizeof(double) * n, cudaMemcpyHostToDevice,
                                         ctx->stream));
        gd = ctx->grad_tmp.as<double>();
        gx = ctx->grad_tmp.as<double>() + n;
    }
    for (int32_t g = 0; g < m->G; ++g) {
        percis_ctx *sub = m->subs[g];
        const int64_t lo = m->vptr[g], ng = m->vptr[g + 1] - lo;
        const int64_t c = m->counts[g], o = m->soff[g];
        if (!m->paths_scattered) {
            const int64_t cc = std::max<int64_t>(c, 1);
            PERCIS_TRY(ensure(sub, sub->pair_s, sizeof(int32_t) * cc, "pairs"));
            PERCIS_TRY(ensure(sub, sub->pair_t, sizeof(int32_t) * cc, "pairs"));
            PERCIS_TRY(ensure(sub, sub->kind, sizeof(int32_t) * cc, "kinds"));
            PERCIS_TRY(ensure(sub, sub->ilen, sizeof(int32_t) * cc, "ilen"));
            PERCIS_TRY(ensure(sub, sub->path_off, sizeof(long long) * (cc + 1), "path offsets"));
            PERCIS_TRY(ensure(sub, sub->cnt, sizeof(unsigned long long) * ng, "counts"));
            PERCIS_TRY(ensure(sub, sub->grad_tmp, sizeof(long long) * (cc + 1), "path lengths"));
            cudaStream_t s = ctx->stream;
            PERCIS_CUDA(ctx, cudaMemcpyAsync(sub->pair_s.p, ctx->pair_s.as<int32_t>() + o, sizeof(int32_t) * c,
                                             cudaMemcpyDeviceToDevice, s));
            PERCIS_CUDA(ctx, cudaMemcpyAsync(sub->pair_t.p, ctx->pair_t.as<int32_t>() + o, sizeof(int32_t) * c,
                                             cudaMemcpyDeviceToDevice, s));
            PERCIS_CUDA(ctx, cudaMemcpyAsync(sub->kind.p, ctx->kind.as<int32_t>() + o, sizeof(int32_t) * c,
                                             cudaMemcpyDeviceToDevice, s));
            PERCIS_CUDA(ctx, cudaMemcpyAsync(sub->ilen.p, ctx->ilen.as<int32_t>() + o, sizeof(int32_t) * c,
                                             cudaMemcpyDeviceToDevice, s));
            PERCIS_CUDA(ctx, cudaMemcpyAsync(sub->cnt.p, ctx->cnt.as<unsigned long long>() + lo,
                                             sizeof(unsigned long long) * ng, cudaMemcpyDeviceToDevice, s));
            if (c > 0) {
                k_offset_ids<<<grid_for(ctx, c, 256), 256, 0, s>>>(sub->pair_s.as<int32_t>(), sub->pair_t.as<int32_t>(),
                                                                 c, -(int32_t)lo);
                PERCIS_CHECK_LAUNCH(ctx, "local ids");
                long long *len64 = sub->grad_tmp.as<long long>();
                k_ilen64<<<grid_for(ctx, c, 256), 256, 0, s>>>(sub->ilen.as<int32_t>(), c, len64);
                PERCIS_CHECK_LAUNCH(ctx, "path lengths");
                PERCIS_TRY(scan_exclusive_i64(sub, (const int64_t *)len64, sub->path_off.as<int64_t>(), c));
            }
            long long tot = 0;
            PERCIS_CUDA(ctx, cudaMemcpyAsync(&tot, sub->path_off.as<long long>() + c, sizeof(tot),
                                             cudaMemcpyDeviceToHost, s));
            PERCIS_CUDA(ctx, cudaStreamSynchronize(s));
            if (c == 0) tot = 0;
            PERCIS_TRY(ensure(sub, sub->arena, sizeof(int32_t) * std::max<long long>(tot, 1), "path arena"));
            sub->arena_cap = std::max<long long>(tot, 1);
            if (c > 0) {
                k_local_paths<<<grid_for(ctx, c, 256), 256, 0, s>>>(
                    sub->ilen.as<int32_t>(), ctx->path_off.as<long long>() + o, ctx->arena.as<int32_t>(), c,
                    sub->path_off.as<long long>(), sub->arena.as<int32_t>(), (int32_t)lo);
                PERCIS_CHECK_LAUNCH(ctx, "local paths");
            }
            sub->phase_count = c;
            sub->last_phase = 1;
            sub->last_seed = ctx->last_seed;
            sub->last_ell = c;
            sub->have_paths = true;
        }
        const percis_status st = percis_backward(sub, gd + lo, gx + lo, 1);
        if (st != PERCIS_OK) return set_err(ctx, st, "graph " + std::to_string(g) + ": " + sub->err);
    }
    m->paths_scattered = true;
    if (!on_device)
        PERCIS_CUDA(ctx, cudaMemcpyAsync(grad_x, gx, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PERCIS_OK;
}
