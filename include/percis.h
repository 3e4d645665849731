/*
 * percis.h -- C ABI of the GB300 (sm_103a) PercIS library.
 *
 * PercIS approximates the percolation centrality p(v) of every vertex
 * (Definition 1: p(v) = sum over s != v != t of sigma_st(v)/sigma_st *
 * kappa(s,t,v), kappa(s,t,v) = R(x_s - x_t) / sum_{u != v != w} R(x_u - x_w),
 * R(x) = max(0, x)) by importance sampling (Section III): pairs (s,t) are
 * drawn with probability kappa~(s,t) = R(x_s - x_t)/C, one shortest s-t path
 * is drawn uniformly from Gamma_st, and p~(v) = (1/l) sum_i
 * kappa(s_i,t_i,v)/kappa~(s_i,t_i) 1[v internal to path i].  Algorithm 1 sets
 * l in two phases (Theorem 1, Propositions 2-3).
 *
 * Conventions for every call:
 *  - All device work is ordered on the context's CUDA stream.
 *  - Inputs are copied; the caller keeps ownership of every buffer it passes.
 *  - Output buffers are caller-owned.  "device" pointers must be device (or
 *    managed) memory of the context's device; "host" pointers plain host
 *    memory.  Calls that take an `on_device` flag accept either.
 *  - Node ids are 0-based int32; CSR row offsets are int64.
 *  - No C++ exception crosses this boundary.  Every call returns a
 *    percis_status; percis_last_error() gives a one-line reason.
 *  - The library allocates its scratch memory with cudaMalloc (grow-only,
 *    reused across calls) and frees it in percis_destroy().
 *  - A context is not thread-safe; use one context per host thread/stream.
 */
#ifndef PERCIS_H
#define PERCIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct percis_ctx percis_ctx;

typedef enum {
    PERCIS_OK = 0,
    PERCIS_E_INVALID = 1,     /* bad argument, malformed CSR, x outside [0,1] or NaN */
    PERCIS_E_DEGENERATE = 2,  /* some C_v <= 0: p(v) undefined (Section II-A) */
    PERCIS_E_OOM = 3,         /* cudaMalloc failed */
    PERCIS_E_CUDA = 4,        /* any other CUDA error (see percis_last_error) */
    PERCIS_E_TIMEOUT = 5,     /* a device-side wait exceeded its budget; context still usable */
    PERCIS_E_TOO_LARGE = 6,   /* request above a documented size cap */
    PERCIS_E_NO_SAMPLE = 7,   /* backward/inspection before a sampling phase */
    PERCIS_E_STATE = 8        /* call order: graph or states not loaded yet */
} percis_status;

/* How sampled paths are produced:
 *  BATCHED: samples are grouped by source; up to `lanes` distinct sources
 *           share one persistent multi-source sigma-BFS (bitset frontiers,
 *           one bit per source per vertex), followed in the same launch by
 *           the per-sample backtrack from t.
 *  PLAIN:   one single-source sigma-BFS launch plus one backtrack launch per
 *           sampled pair (the baseline form).  Same paths as BATCHED.
 *  BIDIR:   RandomSP by a balanced bidirectional BFS (Section III-B), one
 *           block per sample: the side with the smaller frontier degree sum
 *           expands until the sides meet; the meeting vertex is drawn with
 *           probability sigma_s(v) sigma_t(v) / sigma_st (first in vertex-id
 *           order whose running sum reaches u_0 sigma_st) and both sides are
 *           backtracked from it.  Same pairs and the same path distribution,
 *           other paths than BATCHED (each path uniform over the shortest
 *           paths); paths list the meeting vertex, then the s side, then the
 *           t side.  No all-paths estimator.  Scratch per block: a hashed
 *           table of the vertices the sample reaches (32 bytes per entry, at
 *           most half full; 2,048 entries to start, up to 131,072), plus, for
 *           samples that outgrow it, a second pass with 48 bytes per vertex of
 *           the graph (of the largest graph in a many-graph context) and
 *           block. */
enum { PERCIS_FORM_BATCHED = 0, PERCIS_FORM_PLAIN = 1, PERCIS_FORM_BIDIR = 2 };

typedef struct {
    int32_t form;             /* PERCIS_FORM_*; default BATCHED */
    int32_t lanes;            /* batched lane width: 0 = auto, else 64, 128, 256 or 512 */
    int64_t ell1;             /* 0 = Algorithm 1 default max{1000, ceil(ln(1/delta)/eps)} */
    int64_t ell;              /* 0 = Theorem 1 bound; > 0 forces the phase-2 sample size */
    int64_t vertex_diam;      /* < 0 = VertexDiamUB of the loaded graph; >= 0 overrides D */
    int32_t keep_paths;       /* 1 (default): keep phase-2 paths for percis_backward */
    int32_t data_independent; /* 1: PercIS-DI (rho^ = D, v^ = d^2/4, no phase 1; Section IV-B) */
    double timeout_s;         /* budget of every device-side wait (default 10 s) */
    int32_t instrument;       /* 1: sampling launches also count their work into percis_info.work;
                                 2: the bidirectional form also records a per-sample trace
                                 (percis_sample_trace).  Slower; for measurement runs only. */
    int32_t lane_order;       /* batched lane assignment: 0 = sources by vertex id, 1 (default) =
                                 sources grouped by their highest-degree neighbour, so that lanes
                                 with similar BFS levels share 64-bit words and sigma sectors */
    int32_t direction;        /* batched levels: 0 = pull (each unvisited vertex sums over its
                                 in-neighbours), 1 = push (each frontier vertex adds its counts to
                                 its out-neighbours), 2 (default) = per level, push while
                                 push_alpha * (frontier out-edges x words) < (in-edges x words
                                 of vertices with an unvisited active lane) */
    int32_t estimator;        /* 0 (default) = one uniform path per sample (Section III-A);
                                 1 = all paths: every internal v of every shortest s-t path
                                 gets sigma_sv sigma_vt / sigma_st (same expectation; the
                                 Rao-Blackwellised form; batched form only; no backward) */
    double push_alpha;        /* direction 2 threshold; 0 = default (0.5) */
    int32_t cuda_graphs;      /* 1: a many-graph context records the per-graph pair-sampling
                                 launches of a phase once in a CUDA graph and replays it while
                                 the per-graph sample counts repeat (phase 1 always does);
                                 the seed is read from device memory, results are unchanged */
    int32_t bi_table_log;     /* bidirectional form, store of the first pass: 0 (default) = the
                                 direct store (an entry per vertex of the graph and block) when
                                 it fits bi_scratch_gib with every resident block, else one
                                 hashed table per block of the smallest 2^k >= 2n + 1024
                                 entries, k <= 18; k in [10, 20] = hashed, starting at 2^k and
                                 moving to tables 4x larger as a sample grows; < 0 = the
                                 direct store.  Results do not depend on it. */
    int32_t bi_table_max_log; /* largest hashed table when bi_table_log > 0: 0 = the smallest
                                 size 4^j times the first that holds every vertex of the
                                 (largest) graph at most half full, at most 2^20 entries; k =
                                 at most 2^k.  Samples that would fill more than 3/4 of it, or
                                 pass 4,095 levels on a side, are handed to the heavy pass. */
    int32_t bi_scratch_gib;   /* direct store: device memory its blocks may use, GiB (0 = 48);
                                 it holds 56 bytes per vertex and block, so it caps the blocks
                                 (the heavy pass wants one block per SM: 152 x 56 x n bytes) */
    int32_t bi_blocks_per_sm; /* bidirectional first pass: resident blocks per SM, 0 (default) = as
                                 many as fit (4); fewer leave more memory bandwidth to each */
    int32_t tune_form;        /* 1: percis_autotune may also switch between the batched and the
                                 bidirectional form (results then change with the form: both
                                 draw a uniform shortest path, by different procedures) */
    int64_t bi_heavy_edges;   /* a sample whose next level would scan more than this many edges
                                 stops untouched and runs again after the first pass, alone in
                                 a block of 1,024 threads in the direct store (the heavy pass);
                                 0 = default: 16,384 on graphs with a vertex of degree >= 16,384
                                 (hubs make single levels huge), else never; < 0 = never.
                                 Samples the first pass takes in the last two rounds of its
                                 queue (a sample per block) hand over above min(this, 2,048),
                                 so that its blocks end together.  Results do not depend on it. */
    int64_t reserved;         /* must be 0 */
} percis_options;

typedef struct {
    int64_t n, nnz;
    int64_t ell1, ell;            /* phase sizes actually used */
    int64_t vertex_diam;          /* D used in rho^ */
    double C, dhat;               /* C = sum_{u,w} R(x_u - x_w); d^ = max_v C/C_v */
    double rho_tilde, Lambda;     /* Proposition 2 statistics of phase 1 */
    double rho_hat, v_hat, x_hat; /* Algorithm 1 */
    double p1_max;                /* max_v phase-1 p~(v) */
    int64_t zero_weight[2];       /* samples with R(x_s - x_t) = 0, per phase */
    int64_t unreachable[2];       /* samples with Gamma_st empty, per phase */
    int64_t sum_internal[2];      /* sum_i |I(tau_i)|, per phase */
    int64_t sources[2];           /* distinct BFS sources (batched form), per phase */
    int64_t batches[2];           /* persistent launches (batched form), per phase */
    int32_t sigma_overflow;       /* 1 if some sigma reached 2^53 (paths no longer exact) */
    int32_t lanes;                /* lane width used */
    int64_t kernel_launches;      /* kernels this call launched */
    double bfs_ms[2];             /* summed device time of the sigma-BFS launches, per phase
                                     (CUDA events on the context stream) */
    int64_t bfs_launches[2];      /* number of those launches, per phase */
    /* Work counters, filled when options.instrument = 1 (batched form), per phase:
     * work[p][0] sigma reads over shortest-path DAG edges (lane-edge pairs)
     * work[p][1] sigma writes (lane-vertex discoveries)
     * work[p][2] union-frontier vertices summed over levels (adjacency rows needed)
     * work[p][3] out-degree sum of those vertices (adjacency entries needed)
     * work[p][4] sum over samples of the edges a top-down BFS from s scans to
     *            settle t (whole reachable set when t is unreachable)
     * work[p][5] levels run, summed over launches
     * work[p][6] sampled pairs that reached a BFS (R(x_s - x_t) > 0)
     * work[p][7] reserved
     * Bidirectional form instead: [0] edges scanned by both sides, [1] count
     * additions (edges into a new level), [2] vertices reached by both
     * sides, [3] samples traversed (plus 2^32 per meeting layer above 256
     * members), [4] samples handed over to the heavy pass (a level above
     * bi_heavy_edges, a full table or a side past 4,095 levels), [5] moves to
     * a larger table; the rest 0.  bfs_launches is then the number of
     * bidirectional passes (one per phase, two when the heavy pass ran). */
    int64_t work[2][8];
} percis_info;

/* ------------------------------------------------------------ lifecycle */

/* Create a context on `device`.  `stream` is a cudaStream_t (NULL = a new
 * non-blocking stream owned by the context). */
percis_status percis_create(percis_ctx **out, int device, void *stream);
/* Free every buffer the context owns.  NULL is ignored. */
void percis_destroy(percis_ctx *ctx);
/* Switch the stream later calls are ordered on (not owned). */
percis_status percis_set_stream(percis_ctx *ctx, void *stream);
/* Last error message of this context ("" when none).  Owned by the context. */
const char *percis_last_error(const percis_ctx *ctx);
/* Number of kernels this context has launched since it was created
 * (measurement aid; -1 for a NULL context). */
int64_t percis_launch_count(const percis_ctx *ctx);
/* Fill `opt` with the defaults listed in percis_options. */
void percis_default_options(percis_options *opt);
percis_status percis_set_options(percis_ctx *ctx, const percis_options *opt);

/* ---------------------------------------------------------------- inputs */

/* Load a graph G = (V, E) (Section II-A; directed or undirected,
 * unweighted) in CSR form: row_ptr int64[n+1] (row_ptr[0] = 0,
 * non-decreasing, row_ptr[n] = nnz), col int32[nnz] in [0, n).  For an
 * undirected graph every edge must appear in both rows.  Self-loops are
 * allowed and never lie on a shortest path.  Also computes VertexDiamUB
 * (Algorithm 1): for undirected graphs one BFS from the largest-degree vertex
 * of every component, D = 2*ecc - 1; for directed graphs D = n - 2.
 * on_device: 1 if row_ptr/col are device pointers.  Errors: INVALID (bad
 * sizes or indices), OOM, CUDA.  Synchronises the stream once the CSR is
 * validated.  A directed graph's in-adjacency (the stable transpose) is then
 * built on a second stream of the context, so that percis_set_states can run
 * meanwhile; every later call that reads it first makes the context's stream
 * wait for it (no host synchronisation). */
percis_status percis_load_csr(percis_ctx *ctx, int64_t n, int64_t nnz, const int64_t *row_ptr, const int32_t *col,
                              int directed, int on_device);

/* Set the percolation states x_v in [0,1] (Section II-A), double[n] in node
 * order.  Sorts them non-increasingly (ties by node id), builds Algorithm 2's
 * tables w_i, c_i, r_i, c (appendix, preprocessing loop), C_v = C - sum_u
 * |x_v - x_u| and lambda_v = C/C_v = kappa/kappa~ (closed form of d_v in the
 * proof of Proposition 5).  Errors: STATE (no graph), INVALID (NaN or outside
 * [0,1]), DEGENERATE (some C_v <= 0, Section II-A).  Synchronises. */
percis_status percis_set_states(percis_ctx *ctx, const double *x, int on_device);

/* ------------------------------------------------------------ estimation */

/* Algorithm 1 (PercIS): D, l1 phase-1 samples, rho^ (Proposition 2), v^
 * (Proposition 3), x^, l = sup_{x in (0, x^]} d^2 ln(4 d^ rho^/(x delta)) /
 * (g(x) h(eps d^/g(x))) (Theorem 1), l fresh phase-2 samples, and
 * pc_out[v] = p~(v) = lambda_v cnt_v / l.  Samples are addressed by
 * (seed, phase, index) through Philox4x32-10, so results do not depend on
 * the form or the lane width.  eps, delta in (0,1).  pc_out: double[n],
 * device memory if pc_on_device else host.  info: host, may be NULL.
 * Errors: STATE, INVALID, TIMEOUT, CUDA, OOM.  Synchronises once after phase 1
 * (the bound needs four scalars) and at the end. */
percis_status percis_estimate(percis_ctx *ctx, double eps, double delta, uint64_t seed, double *pc_out,
                              int pc_on_device, percis_info *info);

/* Exact percolation centrality (Definition 1) by all-sources sigma-BFS and a
 * dependency accumulation with target weights R(x_s - x_w) (the extended
 * Brandes method used for exact values, Section IV-A).  pc_out: double[n].
 * Errors: TOO_LARGE when n * nnz > 2^40; STATE; CUDA.  Synchronises. */
percis_status percis_exact_small(percis_ctx *ctx, double *pc_out, int pc_on_device);

/* Vector-Jacobian product of the last estimate with respect to the states:
 * grad_x[u] = sum_v grad_pc[v] dF_v/dx_u at the current x, where
 * F_v(x) = (C/l) sum_i a_i(v) R(x_{s_i} - x_{t_i}) / (R_i C_v(x)) is the
 * Section III-A estimator with the phase-2 sample (pairs, paths a_i, and the
 * sampling weights R_i, C) held fixed, so F = p~ at the current x and E[dF]
 * = dp (not in the paper: importance-sampling gradient).  The ramp's
 * derivative at 0 is 0.  grad_pc, grad_x: double[n], device if on_device.
 * Errors: NO_SAMPLE (no estimate with keep_paths), STATE, CUDA. */
percis_status percis_backward(percis_ctx *ctx, const double *grad_pc, double *grad_x, int on_device);

/* ------------------------------------------ stage entry points (parity) */

/* Sorted states and Algorithm 2 tables.  Any output may be NULL.  Device
 * outputs: perm int32[n] (sorted position i-1 -> node id), xs double[n],
 * w/ci/r double[n+2] (1-based, index n+1 = 0), Cv/lambda double[n] (node
 * order).  Host outputs: c, dhat (double; 0 before states are set),
 * vertex_diam (int64).  Device outputs need states (else STATE). */
percis_status percis_get_prep(percis_ctx *ctx, int32_t *perm, double *xs, double *w, double *ci, double *r, double *Cv,
                              double *lambda, double *c, double *dhat, int64_t *vertex_diam);

/* Algorithm 2 sampling of pairs i0 .. i0+count-1 with Philox tag `tag`
 * (0 = phase 1, 1 = phase 2).  Device outputs s, t: int32[count] node ids. */
percis_status percis_sample_pairs(percis_ctx *ctx, uint64_t seed, uint32_t tag, int64_t i0, int64_t count, int32_t *s,
                                  int32_t *t);

/* Single-source sigma-counting BFS with the plain kernel (Section III-B:
 * the BFS from s that RandomSP backtracks).  target < 0: full traversal;
 * target == source: level 0 only; else truncated once target's level is
 * discovered (that level's counts complete).  Device outputs dist int32[n]
 * (-1 = not reached), sigma double[n] (0 = not reached); either may be NULL.
 * sigma_overflow (host, optional): set to 1 when some path count reached 2^53
 * (its FP64 value is then rounded), else 0. */
percis_status percis_bfs(percis_ctx *ctx, int32_t source, int32_t target, int32_t *dist, double *sigma,
                         int32_t *sigma_overflow);

/* Multi-source sigma-counting BFS with the batched kernel, full traversal
 * from nsrc distinct sources (nsrc <= 512).  Device outputs, source-major:
 * dist int32[nsrc*n], sigma double[nsrc*n]. */
percis_status percis_msbfs(percis_ctx *ctx, int32_t nsrc, const int32_t *sources, int32_t *dist, double *sigma);

/* One sampling phase (phase 0: pair tag 0, path tag 2; phase 1: pair tag 1,
 * path tag 3) of `count` samples with the configured form.  Device outputs
 * (any may be NULL): s, t int32[count]; kind int32[count] (0 = path sampled,
 * 1 = R(x_s - x_t) = 0, 2 = t unreachable); ilen int32[count] = |I(tau)|;
 * cnt int64[n] = number of sampled paths with v internal.  The paths stay
 * in the context for percis_get_paths / percis_backward. */
percis_status percis_run_phase(percis_ctx *ctx, uint64_t seed, int phase, int64_t count, int32_t *s, int32_t *t,
                               int32_t *kind, int32_t *ilen, int64_t *cnt);

/* ---- Many graphs in one context ----
 * A batch of num_graphs independent graphs, each its own instance of the
 * problem of Section II (own C, lambda_v, d^, vertex-diameter bound D, l1
 * and l), as one block-diagonal CSR: graph g owns the vertices
 * graph_vptr[g] .. graph_vptr[g+1]-1 (ids of the whole batch) and each of
 * its edges stays inside that range.  Every graph runs its own state
 * preprocessing, Algorithm 2 sampler and Algorithm 1 bounds; the
 * sigma-counting BFS of all graphs shares the batched launches (lanes of
 * several graphs in one launch over the vertex range of those graphs).
 * (Not in the paper, whose method is per graph.)
 * Sample numbering: in each phase, graph g's samples carry the indices
 * off_g .. off_g + l_g - 1 (off_g = the sum of the sample counts of graphs
 * 0 .. g-1) in the Philox counters of the pair and path draws; graph g's
 * estimate equals a single-graph run whose samples start at off_g.
 * All arrays are host memory (copied).  Errors: INVALID for a malformed
 * batch (graph_vptr not running from 0 to n, a graph of fewer than two
 * vertices, row_ptr not monotone, an edge leaving its graph).
 * After this call, percis_set_states(ctx, x[n], ...) sets every graph's
 * states (DEGENERATE names the graph), percis_estimate_graphs estimates, and
 * percis_backward(ctx, grad_pc[n], grad_x[n], ...) differentiates every
 * graph's estimate with its own frozen sample; percis_estimate refuses. */
percis_status percis_load_graphs(percis_ctx *ctx, int32_t num_graphs, const int64_t *graph_vptr, int64_t n,
                                 int64_t nnz, const int64_t *row_ptr, const int32_t *col, int directed);
int32_t percis_num_graphs(percis_ctx *ctx);  /* 0 for a single-graph context */

/* Algorithm 1 for every graph of a percis_load_graphs context at the same
 * (eps, delta, seed).  pc_out[n]: estimates of all vertices (device or host
 * memory per pc_on_device).  info: NULL or num_graphs entries, entry g for
 * graph g; the launch counts, sources, batches and BFS times are shared by
 * all graphs and every entry reports the totals.  Errors as percis_estimate;
 * INVALID for the plain form. */
percis_status percis_estimate_graphs(percis_ctx *ctx, double eps, double delta, uint64_t seed, double *pc_out,
                                     int pc_on_device, percis_info *info);

/* Autotuner (speed options only; not in the paper, whose results these options
 * do not change).  Coordinate descent, each candidate timed (CUDA events, best
 * of two) on probe phases of probe_samples pairs drawn with `seed` from the
 * loaded graph and states:
 *  - batched form: lane order {0, 1}, then lanes {64, 128, 256, 512}, then
 *    direction {pull, push, work estimate with push_alpha 0.25, 0.5, 1, 2};
 *  - bidirectional form: bi_heavy_edges {2048, 4096, 8192, 16384, 65536,
 *    never}, then the first pass's store {default, hashed 2^16, hashed 2^18},
 *    then bi_blocks_per_sm {2, 3, 4}.
 * With options.tune_form = 1 both forms are tuned and the faster one is kept
 * (its options as tuned).  The winner is stored in the context's options
 * (other fields unchanged) and copied to *chosen when chosen is not NULL.  The
 * probe replaces the last sample, so percis_backward needs a new
 * percis_estimate first.
 * Errors: STATE before percis_set_states; INVALID for probe_samples < 1 or the
 * plain form; any error of the probe phases (options are then left as they
 * were). */
percis_status percis_autotune(percis_ctx *ctx, int64_t probe_samples, uint64_t seed, percis_options *chosen);

/* Per-level profile of the last batched launch (measurement aid).  For each
 * level L < min(cap, 32) writes six int64 to out[6L..6L+5]: device time from
 * the launch's start to the end of level L (ns); direction in bit 0 (1 = push)
 * and the pull-work estimate that chose it in the bits above; frontier queue
 * size; push-work estimate (frontier out-edges x words); time at the end of
 * the level's first pass; time after the new frontier was collected.
 * Returns the number of levels. */
int64_t percis_last_levels(percis_ctx *ctx, int64_t *out, int64_t cap);

/* Per-sample trace of the last bidirectional phase (measurement aid), recorded
 * when options.instrument = 2: for sample i, out[8i..8i+7] = device time (ns)
 * when a block took it and when it finished; edges its levels scanned;
 * levels | store << 32 | block << 33 | heavy << 63 (store 0 = hashed tables,
 * 1 = direct; heavy = 1 for the 1,024-thread pass, whose run a handed-over
 * sample shows); the times the levels ended and the meeting vertex was
 * chosen; and two words that are 0 unless the path walk failed (a
 * BAD_PATH status): the step, side and list length, and the vertex and level
 * it stopped at.  Returns the number of samples written (at most cap). */
int64_t percis_sample_trace(percis_ctx *ctx, int64_t *out, int64_t cap);

/* Internal nodes of the paths of the last sampling phase, t-side first.
 * Device outputs: path_ptr int64[count+1], path_nodes int32[path_ptr[count]]
 * (pass path_nodes = NULL to size it first; *total receives the total). */
percis_status percis_get_paths(percis_ctx *ctx, int64_t *path_ptr, int32_t *path_nodes, int64_t *total);

/* ------------------------------------------------ allocation-free call */

/* Largest graph (vertices) percis_bfs_noalloc accepts; its scratch is two
 * int32 frontier queues of this length plus a 256-byte control block, 8 MiB
 * in a static device array that every GPU using the library keeps until the
 * process exits. */
#define PERCIS_NOALLOC_MAX_N 1048576

/* The single-source sigma-counting BFS of percis_bfs for callers that cannot
 * allocate device memory: for instance a process that hands all of the GPU's
 * memory to its own pool at start-up, or a latency-critical path that cannot
 * take cudaMalloc's implicit device synchronisation.  It needs no context and
 * calls no cudaMalloc, cudaFree or allocating library routine.  (The paper has
 * no counterpart; this is a calling convention of this library.)
 *
 * Runs on the calling thread's current CUDA device and on `stream`
 * (a cudaStream_t; NULL = the legacy default stream), and synchronises that
 * stream before returning.  All pointers are device pointers of that device:
 * row_ptr int64[n+1] / col int32[nnz] the CSR (valid as percis_load_csr
 * requires; column indices outside [0, n) make the call return INVALID);
 * in_row_ptr / in_col the in-adjacency of a directed graph, or both NULL for
 * an undirected graph (in-lists = CSR rows).  The row offsets are NOT
 * validated (there is no context that could have checked them): they must
 * start at 0, never decrease and stay within the column array, or the kernel
 * reads outside the caller's buffers.  target < 0: full traversal;
 * target == source: level 0 only; else the traversal stops once target's
 * level is discovered.  Outputs dist int32[n] (-1 = not reached) and sigma
 * double[n] (0 = not reached), written in full.  Results equal percis_bfs's.
 * timeout_s: budget of each device-side wait (<= 0: 10 s); a wait that runs
 * out makes the call return TIMEOUT and leaves the scratch usable by the next
 * call.  sigma_overflow (host, optional): set to 1 when some path count
 * reached 2^53 (its FP64 value is then rounded), else 0.
 *
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress) and the launch size.  Every call enqueues a
 * memset, a cooperative launch and a copy, then synchronises the stream, so
 * it must never be called on a stream that is being captured: such a call
 * returns INVALID without issuing any work.  Every call uses the same
 * scratch array and clears what must start at zero; calls that overlap on
 * the GPU race on it, so serialise them.  Errors: INVALID (n outside [1,
 * PERCIS_NOALLOC_MAX_N], NULL pointer, vertex out of range, a column index
 * outside [0, n) -- that entry is skipped and the outputs hold the traversal
 * without it --, a capturing stream), TIMEOUT, CUDA. */
percis_status percis_bfs_noalloc(int64_t n, const int64_t *row_ptr, const int32_t *col, const int64_t *in_row_ptr,
                                 const int32_t *in_col, int32_t source, int32_t target, int32_t *dist, double *sigma,
                                 void *stream, double timeout_s, int32_t *sigma_overflow);

#ifdef __cplusplus
}
#endif

#endif /* PERCIS_H */
