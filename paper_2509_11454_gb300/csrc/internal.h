// Internal declarations shared by the translation units of libpercis.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/percis.h"

namespace percis {

struct MultiGraph;  // many independent graphs in one context (multi.cu)

// Grow-only device buffer.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    template <class T>
    T *as() const {
        return static_cast<T *>(p);
    }
};

// Control block of the persistent kernels (device memory, zeroed per launch).
struct alignas(16) MsCtl {
    uint32_t bar_count, bar_gen;  // GridBarrier
    uint32_t status;
    uint32_t ticket;
    int32_t level;                // last level reached
    int32_t push_next;            // direction of the next level (1 = push)
    int32_t qn[2];                // frontier queue sizes (ping-pong by level parity): light vertices from the front
    int32_t qh[2];                // and vertices of in-degree > 32 from the back of the same array
    unsigned long long active[8];    // lanes still running (K <= 8 words)
    unsigned long long nonempty[2][8];  // per-level OR of discovered bits (ping-pong)
    unsigned long long fedges[2];    // push work of the next level: frontier out-edges x words (ping-pong)
    unsigned long long uedges[2];    // pull work of the next level: unvisited in-edges x words (ping-pong)
    unsigned long long t_start;      // globaltimer at the first level
    unsigned long long lvl_rec[32][6];  // per level: end time, direction, queue size, out-edges,
                                        // time after phase A, time after the queue build
};

struct PlainCtl {
    uint32_t bar_count, bar_gen;
    uint32_t status;
    int32_t qsize[3];  // queue sizes, level L in slot L % 3
    int32_t level;
    int32_t found;
};

}  // namespace percis

struct percis_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;
    percis_options opt{};
    int num_sms = 0;
    int64_t launches = 0;

    // graph
    bool have_graph = false;
    int64_t n = 0, nnz = 0;
    int directed = 0;
    percis::DevBuf rp, col, irp, icol;  // irp/icol used only when directed
    int64_t vertex_diam = -1;
    bool rows_sorted = false;  // every CSR row strictly increasing (no duplicate edges)
    percis::DevBuf vorder;  // vertices sorted by (highest-degree neighbour, id): lane order of sources
    bool vorder_ready = false;

    // states and preprocessing
    bool have_states = false;
    percis::DevBuf x, xs, perm, w, ci, r, Cv, lam, grp_lo, grp_hi;
    double c_host = 0.0, dhat_host = 0.0;
    percis::DevBuf dscal;  // device scalars: [0] = c, [1] = dhat

    // plain BFS state
    percis::DevBuf ep, lvl, sigma1, qa, qb, plain_ctl;
    int32_t epoch = 0;
    int plain_grid = 0;  // cooperative grid of the plain BFS on this device (0 = not yet queried)
    int bi_per_sm = 0;   // resident blocks per SM of the bidirectional kernel (0 = not yet queried)

    // batched BFS state
    percis::DevBuf vis, fhist, sigmaW, ms_ctl, remaining, found;
    int32_t lanes_alloc = 0;
    int32_t levels_alloc = 0;
    int sigma_mode = 0;  // batched sigma storage: 0 = 32-bit, 1 = 64-bit integers, 2 = FP64
    percis::DevBuf fq0, fq1;  // frontier queues
    percis::DevBuf acc_ap, ap_tau, ap_stamp, ap_list;  // all-paths estimator
    percis::DevBuf plan_dev;                           // lane batches of a many-graph phase
    percis::DevBuf bi_info, bi_queue;                  // bidirectional form, direct store: per-slot scratch
    int64_t bi_slots = 0, bi_n = 0, bi_epoch = 0;
    percis::DevBuf bi_hent, bi_hq, bi_hep, bi_defer;   // bidirectional form, hashed store: tables, queues,
                                                       // slot epochs, samples handed to the direct store
    int64_t bi_hregion = 0, bi_hslots = 0;
    int bi_h0 = 0, bi_hash_per_sm = 0, bi_heavy_per_sm = 0;
    bool groups_ready = false;  // grp_lo / grp_hi hold the current states' tie groups
    int bi_launches = 1;         // launches of the last bidirectional phase (first pass, heavy pass)
    int64_t max_degree_host = -1;  // largest degree of the loaded graph(s), read on first use (-1: not yet)
    int64_t phase_span = 0;  // samples of the running phase (direct-store epochs are indexed by sample)
    percis::DevBuf bi_trace;  // per-sample trace of the last bidirectional phase (instrument = 2)
    int64_t bi_trace_n = 0;
    int64_t ap_warps = 0, ap_n = 0;
    int32_t ap_epoch = 0;

    // samples of the last phase
    percis::DevBuf pair_s, pair_t, kind, ilen, path_off, arena, cnt, arena_top;
    percis::DevBuf src_count, src_fill, src_off, lane_of_v, sorted_samples, samp_lane, samp_t, lane_src, lane_off;
    int64_t phase_count = 0;
    int64_t arena_cap = 0;
    bool have_paths = false;
    int last_phase = -1;
    uint64_t last_seed = 0;
    int64_t last_ell = 0;

    // measurement: event pairs around each sigma-BFS launch of a phase; work counters
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_next = 0;
    percis::DevBuf counters, levdeg;

    // scratch for reductions/scans
    percis::DevBuf scratch, red, status;
    percis::DevBuf radix_counts, sort_a, sort_b;  // radix sort: per-tile digit counts, transpose scratch
    // The in-adjacency of a directed graph is built on `aux` while the states are
    // prepared on the context stream; every use of it first makes the context
    // stream wait for graph_ready (wait_graph).  tr_counts / tr_scratch are the
    // transpose's own radix counts and scan partials.
    cudaStream_t aux = nullptr;
    cudaEvent_t aux_go = nullptr, graph_ready = nullptr;
    bool graph_pending = false;
    percis::DevBuf tr_counts, tr_scratch, graph_info;  // graph_info[0]: largest out- or in-degree (u64)
    uint32_t *tr_sorted_keys = nullptr;  // the sorted targets between transpose_sort and transpose_finish
    void *hmirror = nullptr;  // pinned host words: status and phase statistics read back together
    percis::DevBuf table_ctl;                      // cooperative table scan: barrier, window state, block runs
    int table_grid = 0;                            // co-resident blocks of the table scan (0 = not yet queried)
    percis::DevBuf pc_tmp, grad_tmp, host_pinned;

    // many graphs: one sub-context per graph for everything but the batched BFS
    percis::MultiGraph *multi = nullptr;
    bool skip_diam = false;  // the union of many graphs takes the per-graph bounds
};

namespace percis {
// The launches of a scope go to ctx->aux, with the transpose's own radix counts
// and scan partials; the context's stream and buffers are restored at exit.
struct AuxScope {
    percis_ctx *c;
    explicit AuxScope(percis_ctx *ctx) : c(ctx) { swap(); }
    ~AuxScope() { swap(); }
    AuxScope(const AuxScope &) = delete;
    AuxScope &operator=(const AuxScope &) = delete;
    void swap() {
        std::swap(c->stream, c->aux);
        std::swap(c->radix_counts, c->tr_counts);
        std::swap(c->scratch, c->tr_scratch);
    }
};
}  // namespace percis

namespace percis {

// error helpers (api.cu)
percis_status set_err(percis_ctx *ctx, percis_status st, const std::string &msg);
percis_status cuda_err(percis_ctx *ctx, cudaError_t e, const char *where);
percis_status ensure(percis_ctx *ctx, DevBuf &b, size_t bytes, const char *what);

#define PERCIS_CHECK_LAUNCH(ctx, where)                         \
    do {                                                        \
        (ctx)->launches++;                                      \
        cudaError_t e__ = cudaGetLastError();                   \
        if (e__ != cudaSuccess) return cuda_err((ctx), e__, (where)); \
    } while (0)

#define PERCIS_CUDA(ctx, call)                                  \
    do {                                                        \
        cudaError_t e__ = (call);                               \
        if (e__ != cudaSuccess) return cuda_err((ctx), e__, #call); \
    } while (0)

#define PERCIS_TRY(call)                       \
    do {                                       \
        percis_status s__ = (call);            \
        if (s__ != PERCIS_OK) return s__;      \
    } while (0)

// Next event of the context's pool (created on demand; nullptr if creation fails).
cudaEvent_t next_event(percis_ctx *ctx);
// Summed elapsed time of the event pairs recorded since ev_next was reset (stream synchronised).
double events_elapsed_ms(percis_ctx *ctx);

// util.cu: scans and simple fills
percis_status scan_exclusive_i64(percis_ctx *ctx, const int64_t *in, int64_t *out, int64_t n);
percis_status scan_exclusive_f64(percis_ctx *ctx, const double *in, double *out, int64_t n);
int grid_for(percis_ctx *ctx, int64_t work, int block);

// radix.cu: stable LSD radix sort of (key, value) pairs by key bits [lo_bit, lo_bit + bits),
// 8 bits per pass, in place (tk/tv: scratch of n keys and n values); the in-adjacency
// (irp, icol) of the loaded directed CSR, every in-list ordered by source
percis_status radix_sort_u64(percis_ctx *ctx, uint64_t *keys, int32_t *vals, uint64_t *tk, int32_t *tv, int64_t n,
                             int lo_bit, int bits);
percis_status transpose_sort(percis_ctx *ctx);    // in-adjacency: edges sorted by target (valid row_ptr)
percis_status transpose_finish(percis_ctx *ctx);  // in-adjacency: offsets (valid columns)

// prep.cu
percis_status prep_graph(percis_ctx *ctx);  // transpose (directed), validation, VertexDiamUB
percis_status prep_states(percis_ctx *ctx);  // sort, tables, C_v, lambda, d^
percis_status prep_groups(percis_ctx *ctx);
percis_status wait_graph(percis_ctx *ctx);  // the context stream waits for the in-adjacency  // tie groups of the sorted states (backward, on first use)
percis_status prep_vorder(percis_ctx *ctx);  // lane order of the batched form (on first use)

// sampler.cu
percis_status sample_pairs(percis_ctx *ctx, uint64_t seed, uint32_t tag, int64_t i0, int64_t count, int32_t *s,
                           int32_t *t, int32_t *kind, const uint64_t *seed_dev = nullptr,
                           cudaStream_t stream = nullptr);
percis_status group_by_source(percis_ctx *ctx, int64_t count, int64_t *n_sources, int64_t *n_valid);

// bfs_plain.cu
percis_status plain_bfs(percis_ctx *ctx, const int32_t *s_dev, const int32_t *t_dev, int64_t idx, int32_t s_host,
                        int32_t t_host, bool levels_only = false);
percis_status plain_backtrack(percis_ctx *ctx, uint64_t seed, uint32_t tag, int64_t idx);
percis_status plain_phase(percis_ctx *ctx, uint64_t seed, uint32_t tag_path, int64_t count);
percis_status plain_dist_sigma(percis_ctx *ctx, int32_t *dist, double *sigma);
percis_status vertex_diam_ub(percis_ctx *ctx, int64_t *D);

// bibfs.cu
percis_status bidir_phase(percis_ctx *ctx, uint64_t seed, uint32_t tag_path, int64_t count);

// msbfs.cu
percis_status batched_phase(percis_ctx *ctx, uint64_t seed, uint32_t tag_path, int64_t count, int64_t n_sources,
                            int64_t *batches);
percis_status msbfs_full(percis_ctx *ctx, int32_t nsrc, const int32_t *sources, int32_t *dist, double *sigma);
int choose_lanes(percis_ctx *ctx, int64_t n_sources);

// backward.cu
percis_status backward_fixed(percis_ctx *ctx, const double *g, double *grad);

// exact.cu
percis_status exact_pc(percis_ctx *ctx, double *pc);

// api.cu: one sampling phase (pair tag = phase, path tag = 2 + phase)
struct PhaseOut {
    int64_t sources = 0, batches = 0;
    int32_t overflow = 0;
    double bfs_ms = 0.0;
    int64_t bfs_launches = 0;
    int64_t work[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    // asked for by setting want_stats (read back with the phase's status):
    // sum |I|, sum |I|^2, zero-weight and unreachable samples, and with
    // stats_pmax max_v lambda_v cnt_v / count
    bool want_stats = false, stats_pmax = false;
    int64_t s1 = 0, s2 = 0, zero_w = 0, unreach = 0;
    double pmax = 0.0;
};
percis_status run_phase(percis_ctx *ctx, uint64_t seed, int phase, int64_t count, PhaseOut *po);

// multi.cu
void multi_free(percis_ctx *ctx);
void multi_set_options(percis_ctx *ctx);  // the graphs' contexts follow the union's options
percis_status percis_multi_set_states(percis_ctx *ctx, const double *x, int on_device);
percis_status percis_multi_backward(percis_ctx *ctx, const double *grad_pc, double *grad_x, int on_device);
// pairs of a phase of a many-graph context: graph g draws its counts[g]
// samples with indices off_g.. from its own tables, as global vertex ids
percis_status multi_sample_pairs(percis_ctx *ctx, uint64_t seed, uint32_t tag);
// consecutive lanes from graphs whose vertex ranges fit the batch buffers
struct LaneBatch {
    int32_t lane_base, nlanes, vlo;
    int64_t nr;
};
percis_status multi_plan_batches(percis_ctx *ctx, int64_t n_sources, int W, std::vector<LaneBatch> *out);
int64_t multi_range(percis_ctx *ctx);  // vertex range of the batch buffers
// for the bidirectional form: graph of every vertex, first id of every graph, largest graph
void multi_graph_view(percis_ctx *ctx, const int32_t **gid, const int64_t **vbase, int64_t *largest);

// bounds.cpp
struct Bounds {
    double rho_tilde, Lambda, rho_hat, v_hat, x_hat;
    int64_t ell;
};
Bounds compute_bounds(double eps, double delta, double dhat, int64_t D, int64_t ell1, int64_t sum_ilen,
                      int64_t sum_ilen2, double p1_max, int data_independent);
int64_t ell1_default(double eps, double delta);

}  // namespace percis
