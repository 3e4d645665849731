// C ABI of libpercis and the Algorithm 1 driver (host side).  Every step of
// the estimator runs in the kernels of this library; the host only sizes
// buffers, launches, and evaluates the scalar bound of Theorem 1 from four
// reduced statistics.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"
#include "internal.h"

namespace percis {

percis_status set_err(percis_ctx *ctx, percis_status st, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return st;
}

percis_status cuda_err(percis_ctx *ctx, cudaError_t e, const char *where) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_err(ctx, PERCIS_E_OOM, buf);
    }
    return set_err(ctx, PERCIS_E_CUDA, buf);
}

percis_status ensure(percis_ctx *ctx, DevBuf &b, size_t bytes, const char *what) {
    if (bytes < 16) bytes = 16;
    if (b.bytes >= bytes) return PERCIS_OK;
    if (b.p) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
    }
    const size_t want = bytes + bytes / 16;
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return set_err(ctx, PERCIS_E_OOM, std::string("cudaMalloc failed for ") + what);
    }
    b.bytes = want;
    return PERCIS_OK;
}

cudaEvent_t next_event(percis_ctx *ctx) {
    if (ctx->ev_next >= ctx->ev_pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ctx->ev_pool.push_back(e);
    }
    return ctx->ev_pool[ctx->ev_next++];
}

double events_elapsed_ms(percis_ctx *ctx) {
    double tot = 0.0;
    for (size_t k = 0; k + 1 < ctx->ev_next; k += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, ctx->ev_pool[k], ctx->ev_pool[k + 1]) == cudaSuccess) tot += ms;
        else cudaGetLastError();
    }
    return tot;
}

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Per-phase statistics: sum |I|, sum |I|^2, zero-weight and unreachable
// counts, and max_v lambda_v cnt_v / l.
struct alignas(16) PhaseStats {
    long long s1, s2, zero_w, unreach;
    unsigned long long pmax_bits;
    long long pad[3];
};

__global__ void k_phase_stats(int64_t count, const int32_t *kind, const int32_t *ilen, int64_t n, const double *lam,
                              const unsigned long long *cnt, const double *acc, PhaseStats *out) {
    long long s1 = 0, s2 = 0, zw = 0, un = 0;
    double pm = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const long long l = ilen[i];
        s1 += l;
        s2 += l * l;
        zw += kind[i] == 1;
        un += kind[i] == 2;
    }
    // the largest lambda_v cnt_v (the division by l is monotone, so it is applied
    // once to the maximum, on the host); zero counts skip the FP64 product
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const double c = acc ? acc[v] : (double)cnt[v];
        if (c != 0.0) pm = fmax(pm, __dmul_rn(lam[v], c));
    }
    for (int off = 16; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
        zw += __shfl_xor_sync(0xffffffffu, zw, off);
        un += __shfl_xor_sync(0xffffffffu, un, off);
        pm = fmax(pm, __shfl_xor_sync(0xffffffffu, pm, off));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd((unsigned long long *)&out->s1, (unsigned long long)s1);
        atomicAdd((unsigned long long *)&out->s2, (unsigned long long)s2);
        atomicAdd((unsigned long long *)&out->zero_w, (unsigned long long)zw);
        atomicAdd((unsigned long long *)&out->unreach, (unsigned long long)un);
        atomicMax(&out->pmax_bits, (unsigned long long)__double_as_longlong(pm));
    }
}

// p~(v) = lambda_v cnt_v / l  (all-paths: lambda_v acc_v / l)
__global__ void k_finalize(const double *lam, const unsigned long long *cnt, const double *acc, int64_t n, double ell,
                           double *pc) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const double c = acc ? acc[v] : (double)cnt[v];
        pc[v] = c == 0.0 ? 0.0 : __ddiv_rn(__dmul_rn(lam[v], c), ell);  // (lambda is finite: 0 stays +0)
    }
}

__global__ void k_ilen_i64(const int32_t *ilen, int64_t count, long long *out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) out[i] = ilen[i];
}

__global__ void k_gather_paths(const int32_t *ilen, const long long *path_off, const int32_t *arena,
                               const long long *ptr, int64_t count, int32_t *nodes) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const long long o = path_off[i], d = ptr[i];
        for (int q = 0; q < ilen[i]; ++q) nodes[d + q] = arena[o + q];
    }
}

__global__ void k_u64_to_i64(const unsigned long long *a, int64_t n, long long *b) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) b[i] = (long long)a[i];
}

percis_status need_graph(percis_ctx *ctx) {
    if (!ctx) return PERCIS_E_INVALID;
    if (!ctx->have_graph) return set_err(ctx, PERCIS_E_STATE, "no graph loaded");
    return PERCIS_OK;
}

percis_status need_states(percis_ctx *ctx) {
    PERCIS_TRY(need_graph(ctx));
    if (!ctx->have_states) return set_err(ctx, PERCIS_E_STATE, "no states set");
    return PERCIS_OK;
}

// Pinned host words (status at 0, phase statistics at 64): asynchronous copies
// there complete with the stream, so one synchronisation reads them all.
char *host_mirror(percis_ctx *ctx) {
    if (!ctx->hmirror && cudaMallocHost(&ctx->hmirror, 256) != cudaSuccess) {
        cudaGetLastError();
        ctx->hmirror = nullptr;
    }
    return static_cast<char *>(ctx->hmirror);
}

uint32_t read_status(percis_ctx *ctx) {
    char *hm = host_mirror(ctx);
    uint32_t st = 0, st2 = 0;
    uint32_t *d1 = hm ? reinterpret_cast<uint32_t *>(hm) : &st, *d2 = hm ? reinterpret_cast<uint32_t *>(hm) + 1 : &st2;
    *d1 = 0u;
    *d2 = 0u;
    if (ctx->ms_ctl.p)
        cudaMemcpyAsync(d1, &ctx->ms_ctl.as<MsCtl>()->status, 4, cudaMemcpyDeviceToHost, ctx->stream);
    if (ctx->plain_ctl.p)
        cudaMemcpyAsync(d2, &ctx->plain_ctl.as<PlainCtl>()->status, 4, cudaMemcpyDeviceToHost, ctx->stream);
    cudaStreamSynchronize(ctx->stream);
    return *d1 | *d2;
}

// The phase statistics kernel and the copy of its result to the host mirror
// (offset 64), without synchronising; want_pmax adds the max of lambda cnt over the vertices.
percis_status issue_phase_stats(percis_ctx *ctx, int64_t count, bool want_pmax) {
    PERCIS_TRY(ensure(ctx, ctx->red, sizeof(PhaseStats), "stats"));
    PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->red.p, 0, sizeof(PhaseStats), ctx->stream));
    const int64_t nv = want_pmax ? ctx->n : 0;
    k_phase_stats<<<grid_for(ctx, std::max<int64_t>(std::max<int64_t>(count, nv), 1), 256), 256, 0, ctx->stream>>>(
        count, ctx->kind.as<int32_t>(), ctx->ilen.as<int32_t>(), nv, ctx->lam.as<double>(),
        ctx->cnt.as<unsigned long long>(), ctx->opt.estimator == 1 ? ctx->acc_ap.as<double>() : nullptr,
        ctx->red.as<PhaseStats>());
    PERCIS_CHECK_LAUNCH(ctx, "phase stats");
    char *hm = host_mirror(ctx);
    if (!hm) return set_err(ctx, PERCIS_E_OOM, "pinned host words");
    PERCIS_CUDA(ctx, cudaMemcpyAsync(hm + 64, ctx->red.p, sizeof(PhaseStats), cudaMemcpyDeviceToHost, ctx->stream));
    return PERCIS_OK;
}

// The statistics copied by issue_phase_stats, once the stream has synchronised;
// pmax = max lambda cnt / ell (the IEEE division applied once to the largest product).
void read_phase_stats(percis_ctx *ctx, double ell, PhaseOut *po) {
    PhaseStats hs;
    memcpy(&hs, host_mirror(ctx) + 64, sizeof(hs));
    po->s1 = hs.s1;
    po->s2 = hs.s2;
    po->zero_w = hs.zero_w;
    po->unreach = hs.unreach;
    double pm;
    memcpy(&pm, &hs.pmax_bits, sizeof(pm));
    po->pmax = pm / ell;
}

// Reset status words and grid-barrier counters (a launch that gave up on a
// bounded wait may leave a barrier half-arrived).
void clear_status(percis_ctx *ctx) {
    if (ctx->ms_ctl.p) cudaMemsetAsync(ctx->ms_ctl.p, 0, sizeof(MsCtl), ctx->stream);
    if (ctx->plain_ctl.p) cudaMemsetAsync(ctx->plain_ctl.p, 0, sizeof(PlainCtl), ctx->stream);
}

}  // namespace

// One sampling phase (pair tag = phase, path tag = 2 + phase) of `count`
// samples.  Leaves pairs, kinds, |I|, paths and cnt in the context.
percis_status run_phase(percis_ctx *ctx, uint64_t seed, int phase, int64_t count, PhaseOut *po) {
    PERCIS_TRY(wait_graph(ctx));
    int64_t *sources = &po->sources, *batches = &po->batches;
    int32_t *overflow = &po->overflow;
    const int64_t n = ctx->n;
    const int64_t cap_count = std::max<int64_t>(count, 1);
    PERCIS_TRY(ensure(ctx, ctx->pair_s, sizeof(int32_t) * cap_count, "pairs"));
    PERCIS_TRY(ensure(ctx, ctx->pair_t, sizeof(int32_t) * cap_count, "pairs"));
    PERCIS_TRY(ensure(ctx, ctx->kind, sizeof(int32_t) * cap_count, "kinds"));
    PERCIS_TRY(ensure(ctx, ctx->ilen, sizeof(int32_t) * cap_count, "ilen"));
    PERCIS_TRY(ensure(ctx, ctx->path_off, sizeof(long long) * cap_count, "path offsets"));
    PERCIS_TRY(ensure(ctx, ctx->cnt, sizeof(unsigned long long) * n, "counts"));
    PERCIS_TRY(ensure(ctx, ctx->arena_top, 64, "arena top"));
    if (ctx->arena_cap < cap_count * 8) {
        const int64_t cap = cap_count * 8;
        PERCIS_TRY(ensure(ctx, ctx->arena, sizeof(int32_t) * cap, "path arena"));
        ctx->arena_cap = cap;
    }
    ctx->have_paths = false;
    if (ctx->opt.instrument) PERCIS_TRY(ensure(ctx, ctx->counters, sizeof(unsigned long long) * 8, "counters"));
    ctx->sigma_mode = 0;
    for (int attempt = 0; attempt < 24; ++attempt) {
        clear_status(ctx);
        ctx->ev_next = 0;
        if (ctx->opt.instrument)
            PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->counters.p, 0, sizeof(unsigned long long) * 8, ctx->stream));
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->cnt.p, 0, sizeof(unsigned long long) * n, ctx->stream));
        if (ctx->opt.estimator == 1) {
            PERCIS_TRY(ensure(ctx, ctx->acc_ap, sizeof(double) * n, "all-paths sums"));
            PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->acc_ap.p, 0, sizeof(double) * n, ctx->stream));
        }
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->arena_top.p, 0, 64, ctx->stream));
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->ilen.p, 0, sizeof(int32_t) * cap_count, ctx->stream));
        PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->path_off.p, 0, sizeof(long long) * cap_count, ctx->stream));
        if (ctx->multi)
            PERCIS_TRY(multi_sample_pairs(ctx, seed, (uint32_t)phase));
        else
            PERCIS_TRY(sample_pairs(ctx, seed, (uint32_t)phase, 0, count, ctx->pair_s.as<int32_t>(),
                                    ctx->pair_t.as<int32_t>(), ctx->kind.as<int32_t>()));
        *sources = 0;
        *batches = 0;
        if (ctx->opt.form == PERCIS_FORM_PLAIN) {
            cudaEvent_t e0 = next_event(ctx), e1 = next_event(ctx);
            if (e0) cudaEventRecord(e0, ctx->stream);
            PERCIS_TRY(plain_phase(ctx, seed, (uint32_t)(2 + phase), count));
            if (e1) cudaEventRecord(e1, ctx->stream);
            *batches = count;
        } else if (ctx->opt.form == PERCIS_FORM_BIDIR) {
            cudaEvent_t e0 = next_event(ctx), e1 = next_event(ctx);
            if (e0) cudaEventRecord(e0, ctx->stream);
            PERCIS_TRY(bidir_phase(ctx, seed, (uint32_t)(2 + phase), count));
            if (e1) cudaEventRecord(e1, ctx->stream);
            *batches = ctx->bi_launches;
        } else {
            int64_t U = 0, valid = 0;
            PERCIS_TRY(group_by_source(ctx, count, &U, &valid));
            *sources = U;
            if (U > 0) PERCIS_TRY(batched_phase(ctx, seed, (uint32_t)(2 + phase), count, U, batches));
        }
        if (po->want_stats) PERCIS_TRY(issue_phase_stats(ctx, count, po->stats_pmax));
        const uint32_t st = read_status(ctx);
        PERCIS_CUDA(ctx, cudaGetLastError());
        if (st & DEV_TIMEOUT) return set_err(ctx, PERCIS_E_TIMEOUT, "device wait exceeded its budget");
        if (st & DEV_NEED_LEVELS) {
            ctx->levels_alloc = std::max(ctx->levels_alloc, 32) * 2;
            continue;
        }
        if (st & DEV_ARENA_OVERFLOW) {
            unsigned long long top = 0;
            PERCIS_CUDA(ctx, cudaMemcpy(&top, ctx->arena_top.p, sizeof(top), cudaMemcpyDeviceToHost));
            const int64_t cap = (int64_t)top + (int64_t)top / 4 + 1024;
            PERCIS_TRY(ensure(ctx, ctx->arena, sizeof(int32_t) * cap, "path arena"));
            ctx->arena_cap = cap;
            continue;
        }
        if (ctx->opt.form == PERCIS_FORM_BIDIR && (st & DEV_SIGMA_OVERFLOW) && ctx->sigma_mode != 2) {
            ctx->sigma_mode = 2;  // counts reached 2^53: redo with FP64 counts
            continue;
        }
        if (ctx->opt.form == PERCIS_FORM_BATCHED) {
            if ((st & DEV_SIGMA_WIDE) && ctx->sigma_mode == 0) {
                ctx->sigma_mode = 1;  // a count reached 2^32: redo with 64-bit storage
                continue;
            }
            if ((st & DEV_SIGMA_OVERFLOW) && ctx->sigma_mode == 1) {
                ctx->sigma_mode = 2;  // a count reached 2^53: redo with FP64 counts
                continue;
            }
        }
        if ((st & DEV_BAD_PATH) && !(st & DEV_SIGMA_OVERFLOW))
            return set_err(ctx, PERCIS_E_CUDA, "backtrack found no predecessor");
        *overflow = (st & DEV_SIGMA_OVERFLOW) ? 1 : 0;
        po->bfs_ms = events_elapsed_ms(ctx);
        po->bfs_launches = *batches;
        if (po->want_stats) read_phase_stats(ctx, (double)count, po);
        if (ctx->opt.instrument && ctx->opt.form != PERCIS_FORM_PLAIN) {
            unsigned long long hc[8];
            PERCIS_CUDA(ctx, cudaMemcpy(hc, ctx->counters.p, sizeof(hc), cudaMemcpyDeviceToHost));
            for (int k = 0; k < 8; ++k) po->work[k] = (int64_t)hc[k];
        }
        ctx->phase_count = count;
        ctx->last_phase = phase;
        ctx->last_seed = seed;
        ctx->have_paths = ctx->opt.estimator == 0;  // the all-paths form stores no paths
        return PERCIS_OK;
    }
    return set_err(ctx, PERCIS_E_TOO_LARGE, "phase could not be sized (levels/arena)");
}

}  // namespace percis

using namespace percis;

extern "C" {

void percis_default_options(percis_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->form = PERCIS_FORM_BATCHED;
    opt->lanes = 0;
    opt->ell1 = 0;
    opt->ell = 0;
    opt->vertex_diam = -1;
    opt->keep_paths = 1;
    opt->data_independent = 0;
    opt->timeout_s = 10.0;
    opt->instrument = 0;
    opt->lane_order = 1;
    opt->direction = 2;
    opt->push_alpha = 0.0;
    opt->estimator = 0;
}

percis_status percis_create(percis_ctx **out, int device, void *stream) {
    if (!out) return PERCIS_E_INVALID;
    *out = nullptr;
    percis_ctx *ctx = new (std::nothrow) percis_ctx();
    if (!ctx) return PERCIS_E_OOM;
    ctx->device = device;
    DeviceGuard g(device);
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e != cudaSuccess) {
        delete ctx;
        cudaGetLastError();
        return PERCIS_E_CUDA;
    }
    if (stream) {
        ctx->stream = (cudaStream_t)stream;
    } else {
        e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete ctx;
            return PERCIS_E_CUDA;
        }
        ctx->own_stream = true;
    }
    percis_default_options(&ctx->opt);
    *out = ctx;
    return PERCIS_OK;
}

void percis_destroy(percis_ctx *ctx) {
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->aux) cudaStreamSynchronize(ctx->aux);
    DevBuf *bufs[] = {&ctx->rp, &ctx->col, &ctx->irp, &ctx->icol, &ctx->x, &ctx->xs, &ctx->perm, &ctx->w, &ctx->ci,
                      &ctx->r, &ctx->Cv, &ctx->lam, &ctx->grp_lo, &ctx->grp_hi, &ctx->dscal, &ctx->ep, &ctx->lvl,
                      &ctx->sigma1, &ctx->qa, &ctx->qb, &ctx->plain_ctl, &ctx->vis, &ctx->fhist, &ctx->sigmaW,
                      &ctx->ms_ctl, &ctx->remaining, &ctx->found, &ctx->pair_s, &ctx->pair_t, &ctx->kind,
                      &ctx->ilen, &ctx->path_off, &ctx->arena, &ctx->cnt, &ctx->arena_top, &ctx->src_count,
                      &ctx->src_fill, &ctx->src_off, &ctx->lane_of_v, &ctx->sorted_samples, &ctx->samp_lane,
                      &ctx->samp_t, &ctx->lane_src, &ctx->lane_off, &ctx->scratch, &ctx->red, &ctx->status,
                      &ctx->pc_tmp, &ctx->grad_tmp, &ctx->host_pinned, &ctx->vorder,
                      &ctx->fq0, &ctx->fq1, &ctx->acc_ap,
                      &ctx->ap_tau, &ctx->ap_stamp, &ctx->ap_list, &ctx->plan_dev, &ctx->bi_info,
                      &ctx->bi_queue, &ctx->radix_counts, &ctx->sort_a, &ctx->sort_b,
                      &ctx->table_ctl, &ctx->bi_hent, &ctx->bi_hq, &ctx->bi_hep, &ctx->bi_defer,
                      &ctx->bi_trace, &ctx->tr_counts, &ctx->tr_scratch, &ctx->graph_info};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    if (ctx->counters.p) cudaFree(ctx->counters.p);
    if (ctx->levdeg.p) cudaFree(ctx->levdeg.p);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    multi_free(ctx);
    if (ctx->aux) cudaStreamDestroy(ctx->aux);
    if (ctx->hmirror) cudaFreeHost(ctx->hmirror);
    if (ctx->aux_go) cudaEventDestroy(ctx->aux_go);
    if (ctx->graph_ready) cudaEventDestroy(ctx->graph_ready);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

percis_status percis_set_stream(percis_ctx *ctx, void *stream) {
    if (!ctx || !stream) return PERCIS_E_INVALID;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    ctx->own_stream = false;
    ctx->stream = (cudaStream_t)stream;
    return PERCIS_OK;
}

const char *percis_last_error(const percis_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t percis_launch_count(const percis_ctx *ctx) { return ctx ? ctx->launches : -1; }

percis_status percis_set_options(percis_ctx *ctx, const percis_options *opt) {
    if (!ctx || !opt) return PERCIS_E_INVALID;
    if (opt->form != PERCIS_FORM_BATCHED && opt->form != PERCIS_FORM_PLAIN && opt->form != PERCIS_FORM_BIDIR)
        return set_err(ctx, PERCIS_E_INVALID, "unknown form");
    if (opt->lanes != 0 && opt->lanes != 64 && opt->lanes != 128 && opt->lanes != 256 && opt->lanes != 512)
        return set_err(ctx, PERCIS_E_INVALID, "lanes must be 0, 64, 128, 256 or 512");
    if (opt->lane_order != 0 && opt->lane_order != 1) return set_err(ctx, PERCIS_E_INVALID, "lane_order must be 0 or 1");
    if (opt->direction < 0 || opt->direction > 2) return set_err(ctx, PERCIS_E_INVALID, "direction must be 0, 1 or 2");
    if (!(opt->push_alpha >= 0.0)) return set_err(ctx, PERCIS_E_INVALID, "push_alpha must be >= 0");
    if (opt->estimator != 0 && opt->estimator != 1) return set_err(ctx, PERCIS_E_INVALID, "estimator must be 0 or 1");
    if (opt->estimator == 1 && opt->form != PERCIS_FORM_BATCHED)
        return set_err(ctx, PERCIS_E_INVALID, "the all-paths estimator runs in the batched form");
    if (opt->ell1 < 0 || opt->ell1 == 1 || opt->ell < 0 || !(opt->timeout_s > 0.0))
        return set_err(ctx, PERCIS_E_INVALID, "bad sample sizes or timeout");
    ctx->opt = *opt;
    multi_set_options(ctx);
    return PERCIS_OK;
}

percis_status percis_load_csr(percis_ctx *ctx, int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                              int directed, int on_device) {
    if (!ctx) return PERCIS_E_INVALID;
    if (n < 2 || n > 0x7fffffffLL || nnz < 0 || !row_ptr || (nnz > 0 && !col))
        return set_err(ctx, PERCIS_E_INVALID, "need n >= 2 (int32 ids) and valid pointers");
    DeviceGuard g(ctx->device);
    multi_free(ctx);
    ctx->have_graph = false;
    ctx->have_states = false;
    ctx->have_paths = false;
    PERCIS_TRY(ensure(ctx, ctx->rp, sizeof(int64_t) * (n + 1), "row_ptr"));
    PERCIS_TRY(ensure(ctx, ctx->col, sizeof(int32_t) * std::max<int64_t>(nnz, 1), "col"));
    const cudaMemcpyKind kd = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    PERCIS_CUDA(ctx, cudaMemcpyAsync(ctx->rp.p, row_ptr, sizeof(int64_t) * (n + 1), kd, ctx->stream));
    if (nnz > 0) PERCIS_CUDA(ctx, cudaMemcpyAsync(ctx->col.p, col, sizeof(int32_t) * nnz, kd, ctx->stream));
    ctx->n = n;
    ctx->nnz = nnz;
    ctx->directed = directed ? 1 : 0;
    PERCIS_TRY(prep_graph(ctx));
    ctx->have_graph = true;
    return PERCIS_OK;
}

percis_status percis_set_states(percis_ctx *ctx, const double *x, int on_device) {
    if (ctx && ctx->multi && x) {
        DeviceGuard g(ctx->device);
        return percis_multi_set_states(ctx, x, on_device);
    }
    PERCIS_TRY(need_graph(ctx));
    if (!x) return set_err(ctx, PERCIS_E_INVALID, "x is NULL");
    DeviceGuard g(ctx->device);
    ctx->have_states = false;
    ctx->have_paths = false;
    PERCIS_TRY(ensure(ctx, ctx->x, sizeof(double) * ctx->n, "x"));
    PERCIS_CUDA(ctx, cudaMemcpyAsync(ctx->x.p, x, sizeof(double) * ctx->n,
                                     on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, ctx->stream));
    PERCIS_TRY(prep_states(ctx));
    ctx->have_states = true;
    return PERCIS_OK;
}

percis_status percis_estimate(percis_ctx *ctx, double eps, double delta, uint64_t seed, double *pc_out,
                              int pc_on_device, percis_info *info) {
    PERCIS_TRY(need_states(ctx));
    if (ctx->multi) return set_err(ctx, PERCIS_E_INVALID, "a context of many graphs estimates with percis_estimate_graphs");
    if (!(eps > 0.0 && eps < 1.0) || !(delta > 0.0 && delta < 1.0) || !pc_out)
        return set_err(ctx, PERCIS_E_INVALID, "eps and delta must lie in (0,1); pc_out must be non-NULL");
    DeviceGuard g(ctx->device);
    const int64_t launches0 = ctx->launches;
    percis_info inf;
    memset(&inf, 0, sizeof(inf));
    inf.n = ctx->n;
    inf.nnz = ctx->nnz;
    inf.C = ctx->c_host;
    inf.dhat = ctx->dhat_host;
    const int64_t D = ctx->opt.vertex_diam >= 0 ? ctx->opt.vertex_diam : ctx->vertex_diam;
    inf.vertex_diam = D;
    const bool di = ctx->opt.data_independent != 0;
    const int64_t ell1 = di ? 0 : (ctx->opt.ell1 > 0 ? ctx->opt.ell1 : ell1_default(eps, delta));
    inf.ell1 = ell1;
    auto record = [&](int ph, const PhaseOut &po) {
        inf.sources[ph] = po.sources;
        inf.batches[ph] = po.batches;
        inf.sigma_overflow |= po.overflow;
        inf.bfs_ms[ph] = po.bfs_ms;
        inf.bfs_launches[ph] = po.bfs_launches;
        for (int k = 0; k < 8; ++k) inf.work[ph][k] = po.work[k];
    };
    int64_t s1 = 0, s2 = 0;
    double p1_max = 0.0;
    if (!di) {
        PhaseOut po;
        po.want_stats = po.stats_pmax = true;  // read back with the phase's status
        PERCIS_TRY(run_phase(ctx, seed, 0, ell1, &po));
        record(0, po);
        inf.zero_weight[0] = po.zero_w;
        inf.unreachable[0] = po.unreach;
        inf.sum_internal[0] = po.s1;
        s1 = po.s1;
        s2 = po.s2;
        p1_max = po.pmax;
    }
    const Bounds b = compute_bounds(eps, delta, ctx->dhat_host, D, ell1, s1, s2, p1_max, di ? 1 : 0);
    inf.rho_tilde = b.rho_tilde;
    inf.Lambda = b.Lambda;
    inf.rho_hat = b.rho_hat;
    inf.v_hat = b.v_hat;
    inf.x_hat = b.x_hat;
    inf.p1_max = p1_max;
    const int64_t ell = ctx->opt.ell > 0 ? ctx->opt.ell : b.ell;
    inf.ell = ell;
    {
        PhaseOut po;
        PERCIS_TRY(run_phase(ctx, seed, 1, ell, &po));
        record(1, po);
    }
    ctx->last_ell = ell;
    double *dst = pc_out;
    if (!pc_on_device) {
        PERCIS_TRY(ensure(ctx, ctx->pc_tmp, sizeof(double) * ctx->n, "pc staging"));
        dst = ctx->pc_tmp.as<double>();
    }
    k_finalize<<<grid_for(ctx, ctx->n, 256), 256, 0, ctx->stream>>>(
        ctx->lam.as<double>(), ctx->cnt.as<unsigned long long>(),
        ctx->opt.estimator == 1 ? ctx->acc_ap.as<double>() : nullptr, ctx->n, (double)ell, dst);
    PERCIS_CHECK_LAUNCH(ctx, "finalize");
    if (info) PERCIS_TRY(issue_phase_stats(ctx, ell, false));  // read after the synchronisation below
    if (!pc_on_device)
        PERCIS_CUDA(ctx, cudaMemcpyAsync(pc_out, dst, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (info) {
        PhaseOut p2;
        read_phase_stats(ctx, (double)ell, &p2);
        inf.zero_weight[1] = p2.zero_w;
        inf.unreachable[1] = p2.unreach;
        inf.sum_internal[1] = p2.s1;
    }
    inf.lanes = ctx->opt.form == PERCIS_FORM_PLAIN ? 1 : ctx->lanes_alloc;
    inf.kernel_launches = ctx->launches - launches0;
    if (info) *info = inf;
    return PERCIS_OK;
}

percis_status percis_exact_small(percis_ctx *ctx, double *pc_out, int pc_on_device) {
    PERCIS_TRY(need_states(ctx));
    if (!pc_out) return set_err(ctx, PERCIS_E_INVALID, "pc_out is NULL");
    if ((double)ctx->n * (double)std::max<int64_t>(ctx->nnz, 1) > 1099511627776.0)
        return set_err(ctx, PERCIS_E_TOO_LARGE, "n * nnz above 2^40");
    DeviceGuard g(ctx->device);
    PERCIS_TRY(wait_graph(ctx));
    double *dst = pc_out;
    PERCIS_TRY(ensure(ctx, ctx->grad_tmp, sizeof(double) * ctx->n, "exact output"));
    if (!pc_on_device) dst = ctx->grad_tmp.as<double>();
    PERCIS_TRY(exact_pc(ctx, dst));
    if (!pc_on_device)
        PERCIS_CUDA(ctx, cudaMemcpyAsync(pc_out, dst, sizeof(double) * ctx->n, cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const uint32_t st = read_status(ctx);
    if (st & DEV_TIMEOUT) return set_err(ctx, PERCIS_E_TIMEOUT, "device wait exceeded its budget");
    return PERCIS_OK;
}

percis_status percis_backward(percis_ctx *ctx, const double *grad_pc, double *grad_x, int on_device) {
    PERCIS_TRY(need_states(ctx));
    if (!grad_pc || !grad_x) return set_err(ctx, PERCIS_E_INVALID, "NULL gradient buffer");
    if (ctx->multi) {
        DeviceGuard g(ctx->device);
        return percis_multi_backward(ctx, grad_pc, grad_x, on_device);
    }
    if (!ctx->have_paths || ctx->last_phase != 1 || ctx->last_ell <= 0)
        return set_err(ctx, PERCIS_E_NO_SAMPLE, "backward needs a completed estimate of the one-path form");
    DeviceGuard g(ctx->device);
    const int64_t n = ctx->n;
    const double *gin = grad_pc;
    double *gout = grad_x;
    if (!on_device) {
        PERCIS_TRY(ensure(ctx, ctx->pc_tmp, sizeof(double) * 2 * n, "backward staging"));
        double *tmp = ctx->pc_tmp.as<double>();
        PERCIS_CUDA(ctx, cudaMemcpyAsync(tmp, grad_pc, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream));
        gin = tmp;
        gout = tmp + n;
    }
    PERCIS_TRY(backward_fixed(ctx, gin, gout));
    if (!on_device)
        PERCIS_CUDA(ctx, cudaMemcpyAsync(grad_x, gout, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PERCIS_OK;
}

percis_status percis_get_prep(percis_ctx *ctx, int32_t *perm, double *xs, double *w, double *ci, double *r,
                              double *Cv, double *lambda, double *c, double *dhat, int64_t *vertex_diam) {
    PERCIS_TRY(need_graph(ctx));
    DeviceGuard g(ctx->device);
    if (vertex_diam) *vertex_diam = ctx->vertex_diam;
    if (!ctx->have_states) {
        if (perm || xs || w || ci || r || Cv || lambda) return set_err(ctx, PERCIS_E_STATE, "no states set");
        if (c) *c = 0.0;
        if (dhat) *dhat = 0.0;
        return PERCIS_OK;
    }
    const int64_t n = ctx->n;
    auto cp = [&](void *dst, const DevBuf &src, size_t bytes) -> percis_status {
        if (!dst) return PERCIS_OK;
        PERCIS_CUDA(ctx, cudaMemcpyAsync(dst, src.p, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        return PERCIS_OK;
    };
    PERCIS_TRY(cp(perm, ctx->perm, sizeof(int32_t) * n));
    PERCIS_TRY(cp(xs, ctx->xs, sizeof(double) * n));
    PERCIS_TRY(cp(w, ctx->w, sizeof(double) * (n + 2)));
    PERCIS_TRY(cp(ci, ctx->ci, sizeof(double) * (n + 2)));
    PERCIS_TRY(cp(r, ctx->r, sizeof(double) * (n + 2)));
    PERCIS_TRY(cp(Cv, ctx->Cv, sizeof(double) * n));
    PERCIS_TRY(cp(lambda, ctx->lam, sizeof(double) * n));
    if (c) *c = ctx->c_host;
    if (dhat) *dhat = ctx->dhat_host;
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PERCIS_OK;
}

percis_status percis_sample_pairs(percis_ctx *ctx, uint64_t seed, uint32_t tag, int64_t i0, int64_t count, int32_t *s,
                                  int32_t *t) {
    PERCIS_TRY(need_states(ctx));
    if (count < 0 || i0 < 0 || (count > 0 && (!s || !t))) return set_err(ctx, PERCIS_E_INVALID, "bad arguments");
    DeviceGuard g(ctx->device);
    PERCIS_TRY(sample_pairs(ctx, seed, tag, i0, count, s, t, nullptr));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PERCIS_OK;
}

percis_status percis_bfs(percis_ctx *ctx, int32_t source, int32_t target, int32_t *dist, double *sigma,
                         int32_t *sigma_overflow) {
    if (sigma_overflow) *sigma_overflow = 0;
    PERCIS_TRY(need_graph(ctx));
    if (source < 0 || source >= ctx->n || target >= ctx->n) return set_err(ctx, PERCIS_E_INVALID, "bad vertex");
    DeviceGuard g(ctx->device);
    PERCIS_TRY(wait_graph(ctx));
    clear_status(ctx);
    PERCIS_TRY(plain_bfs(ctx, nullptr, nullptr, 0, source, target < 0 ? -1 : target));
    PERCIS_TRY(plain_dist_sigma(ctx, dist, sigma));
    const uint32_t st = read_status(ctx);
    if (st & DEV_TIMEOUT) return set_err(ctx, PERCIS_E_TIMEOUT, "device wait exceeded its budget");
    PERCIS_CUDA(ctx, cudaGetLastError());
    if (sigma_overflow) *sigma_overflow = (st & DEV_SIGMA_OVERFLOW) ? 1 : 0;
    return PERCIS_OK;
}

percis_status percis_msbfs(percis_ctx *ctx, int32_t nsrc, const int32_t *sources, int32_t *dist, double *sigma) {
    PERCIS_TRY(need_graph(ctx));
    if (nsrc < 1 || nsrc > 512 || !sources) return set_err(ctx, PERCIS_E_INVALID, "need 1..512 sources");
    DeviceGuard g(ctx->device);
    PERCIS_TRY(wait_graph(ctx));
    {
        int32_t hsrc[512];
        PERCIS_CUDA(ctx, cudaMemcpyAsync(hsrc, sources, sizeof(int32_t) * nsrc, cudaMemcpyDeviceToHost, ctx->stream));
        PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        std::sort(hsrc, hsrc + nsrc);
        for (int i = 0; i < nsrc; ++i)
            if (hsrc[i] < 0 || hsrc[i] >= ctx->n || (i > 0 && hsrc[i] == hsrc[i - 1]))
                return set_err(ctx, PERCIS_E_INVALID, "sources must be distinct vertex ids");
    }
    clear_status(ctx);
    PERCIS_TRY(msbfs_full(ctx, nsrc, sources, dist, sigma));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const uint32_t st = read_status(ctx);
    if (st & DEV_TIMEOUT) return set_err(ctx, PERCIS_E_TIMEOUT, "device wait exceeded its budget");
    return PERCIS_OK;
}

percis_status percis_run_phase(percis_ctx *ctx, uint64_t seed, int phase, int64_t count, int32_t *s, int32_t *t,
                               int32_t *kind, int32_t *ilen, int64_t *cnt) {
    PERCIS_TRY(need_states(ctx));
    if ((phase != 0 && phase != 1) || count < 1) return set_err(ctx, PERCIS_E_INVALID, "phase 0/1, count >= 1");
    DeviceGuard g(ctx->device);
    PhaseOut po;
    PERCIS_TRY(run_phase(ctx, seed, phase, count, &po));
    ctx->last_ell = count;
    auto cp = [&](void *dst, const DevBuf &b, size_t bytes) -> percis_status {
        if (!dst) return PERCIS_OK;
        PERCIS_CUDA(ctx, cudaMemcpyAsync(dst, b.p, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        return PERCIS_OK;
    };
    PERCIS_TRY(cp(s, ctx->pair_s, sizeof(int32_t) * count));
    PERCIS_TRY(cp(t, ctx->pair_t, sizeof(int32_t) * count));
    PERCIS_TRY(cp(kind, ctx->kind, sizeof(int32_t) * count));
    PERCIS_TRY(cp(ilen, ctx->ilen, sizeof(int32_t) * count));
    if (cnt) {
        k_u64_to_i64<<<grid_for(ctx, ctx->n, 256), 256, 0, ctx->stream>>>(ctx->cnt.as<unsigned long long>(), ctx->n,
                                                                         (long long *)cnt);
        PERCIS_CHECK_LAUNCH(ctx, "cnt copy");
    }
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PERCIS_OK;
}

// Autotuner: coordinate descent over the options that change speed but not
// results (lane order, lane width, direction rule), each candidate timed with
// CUDA events on a probe phase of the current graph and states.
percis_status percis_autotune(percis_ctx *ctx, int64_t probe_samples, uint64_t seed, percis_options *chosen) {
    PERCIS_TRY(need_states(ctx));
    if (probe_samples < 1) return set_err(ctx, PERCIS_E_INVALID, "probe_samples >= 1");
    if (ctx->opt.form == PERCIS_FORM_PLAIN)
        return set_err(ctx, PERCIS_E_INVALID, "the autotuner tunes the batched and bidirectional forms");
    DeviceGuard g(ctx->device);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PERCIS_CUDA(ctx, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_err(ctx, cudaGetLastError(), "event");
    }
    percis_options best = ctx->opt;
    const percis_options saved = ctx->opt;
    percis_status st = PERCIS_OK;
    auto time_opt = [&](const percis_options &o, float *ms) -> percis_status {
        ctx->opt = o;
        float bestms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            PhaseOut po;
            PERCIS_CUDA(ctx, cudaEventRecord(e0, ctx->stream));
            PERCIS_TRY(run_phase(ctx, seed + (uint64_t)rep, 0, probe_samples, &po));
            PERCIS_CUDA(ctx, cudaEventRecord(e1, ctx->stream));
            PERCIS_CUDA(ctx, cudaEventSynchronize(e1));
            float t = 0.f;
            PERCIS_CUDA(ctx, cudaEventElapsedTime(&t, e0, e1));
            bestms = std::min(bestms, t);
        }
        *ms = bestms;
        return PERCIS_OK;
    };
    // coordinate descent over one form's options, from o0; *o_best / *ms_best the winner
    auto tune_form = [&](percis_options o0, percis_options *o_best, float *ms_best) -> percis_status {
        percis_options b = o0;
        float bms = 0.f;
        PERCIS_TRY(time_opt(b, &bms));
        auto try_opt = [&](const percis_options &o) -> percis_status {
            float ms = 0.f;
            PERCIS_TRY(time_opt(o, &ms));
            if (ms < bms) bms = ms, b = o;
            return PERCIS_OK;
        };
        if (o0.form == PERCIS_FORM_BIDIR) {
            // 1. heavy-level threshold
            const int64_t heavy[6] = {2048, 4096, 8192, 16384, 65536, -1};
            for (int k = 0; k < 6; ++k) {
                percis_options o = b;
                o.bi_heavy_edges = heavy[k];
                PERCIS_TRY(try_opt(o));
            }
            // 2. the first pass's store: the default, or hashed tables of 2^16 or 2^18
            const int tl[2] = {16, 18};
            for (int k = 0; k < 2; ++k) {
                percis_options o = b;
                o.bi_table_log = o.bi_table_max_log = tl[k];
                PERCIS_TRY(try_opt(o));
            }
            // 3. resident blocks per SM
            for (int bp = 2; bp <= 4; ++bp) {
                percis_options o = b;
                o.bi_blocks_per_sm = bp;
                PERCIS_TRY(try_opt(o));
            }
        } else {
            // 1. lane order
            for (int lo = 0; lo <= 1; ++lo) {
                percis_options o = b;
                o.lane_order = lo;
                PERCIS_TRY(try_opt(o));
            }
            // 2. lane width
            const int widths[4] = {64, 128, 256, 512};
            for (int k = 0; k < 4; ++k) {
                percis_options o = b;
                o.lanes = widths[k];
                PERCIS_TRY(try_opt(o));
            }
            // 3. direction: pull, push, or by work estimate with the push threshold
            const double alphas[4] = {0.25, 0.5, 1.0, 2.0};
            for (int k = 0; k < 6; ++k) {
                percis_options o = b;
                o.direction = k < 2 ? k : 2;
                if (k >= 2) o.push_alpha = alphas[k - 2];
                PERCIS_TRY(try_opt(o));
            }
        }
        *o_best = b;
        *ms_best = bms;
        return PERCIS_OK;
    };
    float best_ms = 0.f;
    st = tune_form(saved, &best, &best_ms);
    if (st == PERCIS_OK && saved.tune_form) {
        percis_options other = saved;
        other.form = saved.form == PERCIS_FORM_BIDIR ? PERCIS_FORM_BATCHED : PERCIS_FORM_BIDIR;
        percis_options ob;
        float oms = 0.f;
        st = tune_form(other, &ob, &oms);
        if (st == PERCIS_OK && oms < best_ms) best = ob, best_ms = oms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->have_paths = false;  // the probe phases replaced the last sample
    if (st != PERCIS_OK) {
        ctx->opt = saved;
        return st;
    }
    // only the speed options (and, when allowed, the form) change; everything else
    // stays as the caller set it
    ctx->opt = saved;
    ctx->opt.form = best.form;
    ctx->opt.lane_order = best.lane_order;
    ctx->opt.lanes = best.lanes;
    ctx->opt.direction = best.direction;
    ctx->opt.push_alpha = best.push_alpha;
    ctx->opt.bi_heavy_edges = best.bi_heavy_edges;
    ctx->opt.bi_table_log = best.bi_table_log;
    ctx->opt.bi_table_max_log = best.bi_table_max_log;
    ctx->opt.bi_blocks_per_sm = best.bi_blocks_per_sm;
    if (chosen) *chosen = ctx->opt;
    return PERCIS_OK;
}

int64_t percis_last_levels(percis_ctx *ctx, int64_t *out, int64_t cap) {
    if (!ctx || !ctx->ms_ctl.p || !out) return 0;
    DeviceGuard g(ctx->device);
    MsCtl hc;
    if (cudaMemcpyAsync(&hc, ctx->ms_ctl.p, sizeof(hc), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int64_t lv = std::min<int64_t>(std::min<int64_t>(hc.level, 32), cap);
    for (int64_t L = 0; L < lv; ++L)
        for (int k = 0; k < 6; ++k) out[6 * L + k] = (int64_t)hc.lvl_rec[L][k];
    return lv;
}

int64_t percis_sample_trace(percis_ctx *ctx, int64_t *out, int64_t cap) {
    if (!ctx || !ctx->bi_trace.p || !out || cap < 0) return 0;
    DeviceGuard g(ctx->device);
    const int64_t k = std::min<int64_t>(ctx->bi_trace_n, cap);
    if (k > 0 && (cudaMemcpyAsync(out, ctx->bi_trace.p, sizeof(int64_t) * 8 * k, cudaMemcpyDeviceToHost,
                                  ctx->stream) != cudaSuccess ||
                  cudaStreamSynchronize(ctx->stream) != cudaSuccess)) {
        cudaGetLastError();
        return 0;
    }
    return k;
}

percis_status percis_get_paths(percis_ctx *ctx, int64_t *path_ptr, int32_t *path_nodes, int64_t *total) {
    PERCIS_TRY(need_states(ctx));
    if (!ctx->have_paths) return set_err(ctx, PERCIS_E_NO_SAMPLE, "no sampling phase yet");
    DeviceGuard g(ctx->device);
    const int64_t count = ctx->phase_count;
    PERCIS_TRY(ensure(ctx, ctx->grad_tmp, sizeof(long long) * (2 * count + 2), "path ptr"));
    long long *len64 = ctx->grad_tmp.as<long long>();
    long long *ptr = len64 + count + 1;
    k_ilen_i64<<<grid_for(ctx, count, 256), 256, 0, ctx->stream>>>(ctx->ilen.as<int32_t>(), count, len64);
    PERCIS_CHECK_LAUNCH(ctx, "ilen");
    PERCIS_TRY(scan_exclusive_i64(ctx, (const int64_t *)len64, (int64_t *)ptr, count));
    long long tot = 0;
    PERCIS_CUDA(ctx, cudaMemcpyAsync(&tot, ptr + count, sizeof(tot), cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (total) *total = tot;
    if (path_ptr)
        PERCIS_CUDA(ctx, cudaMemcpyAsync(path_ptr, ptr, sizeof(long long) * (count + 1), cudaMemcpyDeviceToDevice,
                                         ctx->stream));
    if (path_nodes) {
        k_gather_paths<<<grid_for(ctx, count, 256), 256, 0, ctx->stream>>>(
            ctx->ilen.as<int32_t>(), ctx->path_off.as<long long>(), ctx->arena.as<int32_t>(), ptr, count, path_nodes);
        PERCIS_CHECK_LAUNCH(ctx, "gather paths");
    }
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return PERCIS_OK;
}

}  // extern "C"
