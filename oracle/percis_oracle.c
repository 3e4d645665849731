/*
 * percis_oracle.c -- plain CPU oracle for PercIS (Cruciani & Pellegrina,
 * "Fast Percolation Centrality Approximation with Importance Sampling").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The CUDA library never
 * links, loads or calls it, and the two share no code.
 *
 * Everything here is deliberately plain: FP64, one thread, no blocking or
 * fusion, compiled with -ffp-contract=off so that a*b-c is never fused.
 * Each function cites the passage of the paper it follows.
 *
 * Conventions (readings of passages the paper leaves open; each is also
 * listed in the design notes):
 *  - Node ids are 0-based.  Sorted positions follow the paper's 1-based
 *    notation: position i holds the i-th largest state, ties broken by
 *    ascending node id (Section II-A assumes x_1 >= ... >= x_n).
 *  - Uniform draws U(0,1) of Algorithm 2 are taken in (0,1]:
 *    u = ((w >> 11) + 1) * 2^-53 with w a 64-bit Philox4x32-10 output.
 *  - Algorithm 2's c_i is clamped at 0 when rounding makes it negative.
 *  - A sampled pair with R(x_s - x_t) = 0 (a tie, or s = t through
 *    rounding) has kappa(s,t,v) = 0 and contributes nothing; an unreachable
 *    target (Gamma_st empty) contributes nothing.  Both still count in l.
 *  - Predecessors are visited in in-adjacency order: the CSR row itself for
 *    undirected graphs, and for directed graphs the transpose built by a
 *    stable counting sort (sources ascending).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ Philox */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with
 * multipliers 0xD2511F53 and 0xCD9E8D57, key bumped by the Weyl constants
 * 0x9E3779B9 and 0xBB67AE85 between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t y0 = (uint32_t)(p1 >> 32) ^ x1 ^ k0;
        uint32_t y1 = (uint32_t)p1;
        uint32_t y2 = (uint32_t)(p0 >> 32) ^ x3 ^ k1;
        uint32_t y3 = (uint32_t)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Two uniforms in (0,1] from counter (i_lo, i_hi, tag, j) and key = seed. */
void orc_uniforms(uint64_t seed, uint64_t i, uint32_t tag, uint32_t j, double out[2]) {
    uint32_t ctr[4] = {(uint32_t)i, (uint32_t)(i >> 32), tag, j};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    uint64_t wa = ((uint64_t)o[1] << 32) | o[0];
    uint64_t wb = ((uint64_t)o[3] << 32) | o[2];
    out[0] = (double)((wa >> 11) + 1) * 0x1p-53;
    out[1] = (double)((wb >> 11) + 1) * 0x1p-53;
}

/* ------------------------------------------------------------ sorted states */

static const double *g_sort_x;
static int cmp_desc(const void *pa, const void *pb) {
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    double xa = g_sort_x[a], xb = g_sort_x[b];
    if (xa > xb) return -1;
    if (xa < xb) return 1;
    return (a > b) - (a < b);
}

/* Section II-A: relabel nodes so that x_1 >= x_2 >= ... >= x_n.
 * perm[i-1] = node id at sorted position i; xs[i-1] = its state. */
void orc_sort_states(int64_t n, const double *x, int32_t *perm, double *xs) {
    for (int64_t v = 0; v < n; v++) perm[v] = (int32_t)v;
    g_sort_x = x;
    qsort(perm, (size_t)n, sizeof(int32_t), cmp_desc);
    for (int64_t i = 0; i < n; i++) xs[i] = x[perm[i]];
}

/* Algorithm 2, preprocessing loop (appendix): arrays are 1-based with
 * length n+2; w[n+1] = r[n+1] = 0.  Returns c. */
double orc_tables(int64_t n, const double *xs, double *w, double *ci, double *r) {
    w[n + 1] = 0.0;
    r[n + 1] = 0.0;
    ci[n + 1] = 0.0;
    w[0] = r[0] = ci[0] = 0.0;
    double c = 0.0;
    for (int64_t i = n; i >= 1; i--) {
        w[i] = w[i + 1] + xs[i - 1];
        double cv = (double)(n - i + 1) * xs[i - 1] - w[i];
        if (cv < 0.0) cv = 0.0;
        ci[i] = cv;
        r[i] = r[i + 1] + ci[i];
        c = c + ci[i];
    }
    return c;
}

/* Algorithm 2, first binary search: s = argmin_x {(c - r_{x+1})/c >= u}. */
int64_t orc_search_s(int64_t n, const double *r, double c, double u) {
    int64_t a = 1, b = n, d = (a + b) / 2;
    while (a <= b) {
        double k = (c - r[d + 1]) / c;
        if (u <= k) b = d - 1;
        else a = d + 1;
        d = (a + b) / 2;
    }
    return b + 1;
}

/* Algorithm 2, second binary search over t in [s, n]. */
int64_t orc_search_t(int64_t n, int64_t s, const double *xs, const double *w, const double *ci, double u) {
    int64_t a = s, b = n, d = (a + b) / 2;
    while (a <= b) {
        double num = (double)(d - s + 1) * xs[s - 1] - w[s] + w[d + 1];
        double k = num / ci[s];
        if (u <= k) b = d - 1;
        else a = d + 1;
        d = (a + b) / 2;
    }
    return b + 1;
}

/* Draw `count` pairs with sample indices i0 .. i0+count-1 (Algorithm 2).
 * Outputs node ids and sorted positions (1-based). */
void orc_sample_pairs(int64_t n, const double *xs, const int32_t *perm, const double *w, const double *ci,
                      const double *r, double c, uint64_t seed, uint32_t tag, int64_t i0, int64_t count,
                      int32_t *s_node, int32_t *t_node, int64_t *s_pos, int64_t *t_pos) {
    for (int64_t k = 0; k < count; k++) {
        double u[2];
        orc_uniforms(seed, (uint64_t)(i0 + k), tag, 0u, u);
        int64_t s = orc_search_s(n, r, c, u[0]);
        int64_t t = orc_search_t(n, s, xs, w, ci, u[1]);
        if (s_pos) s_pos[k] = s;
        if (t_pos) t_pos[k] = t;
        s_node[k] = perm[s - 1];
        t_node[k] = perm[t - 1];
    }
}

/* --------------------------------------------------------------- graphs */

/* In-adjacency for directed graphs: stable counting sort of the edge list by
 * target, visiting sources in ascending order.  irp: n+1, icol: nnz. */
void orc_transpose(int64_t n, const int64_t *rp, const int32_t *col, int64_t *irp, int32_t *icol) {
    for (int64_t v = 0; v <= n; v++) irp[v] = 0;
    for (int64_t e = 0; e < rp[n]; e++) irp[col[e] + 1]++;
    for (int64_t v = 0; v < n; v++) irp[v + 1] += irp[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    for (int64_t v = 0; v <= n; v++) fill[v] = irp[v];
    for (int64_t u = 0; u < n; u++)
        for (int64_t e = rp[u]; e < rp[u + 1]; e++) icol[fill[col[e]]++] = (int32_t)u;
    free(fill);
}

/* sigma-counting BFS from s (Section III-B, RandomSP via a BFS "initialized
 * from s and expanded until t is found").  With t >= 0 the traversal stops
 * once the level holding t is discovered (every level before it has been
 * fully expanded, so sigma of t is complete); with t < 0 it runs to the end.
 * sigma_w = sum of sigma_u over in-neighbours u with dist(u) = dist(w)-1.
 * dist = -1 / sigma = 0 for undiscovered vertices.  Returns dist(s,t)
 * (-1 if unreachable) or, for t < 0, the eccentricity of s.
 * edges: out-edges scanned by expanding the levels before the last one.
 * order: discovery order (size n); *norder receives its length.
 * *overflow is set when a sigma reaches 2^53. */
int64_t orc_bfs(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *irp, const int32_t *icol,
                int32_t s, int32_t t, int32_t *dist, double *sigma, int32_t *order, int64_t *norder,
                int64_t *edges, int32_t *overflow) {
    for (int64_t v = 0; v < n; v++) {
        dist[v] = -1;
        sigma[v] = 0.0;
    }
    int64_t no = 0, lstart = 0, level = 0, e_scanned = 0;
    dist[s] = 0;
    sigma[s] = 1.0;
    order[no++] = s;
    while (lstart < no) {
        if (t >= 0 && dist[t] >= 0) break;
        int64_t lend = no;
        for (int64_t k = lstart; k < lend; k++) {
            int32_t u = order[k];
            e_scanned += rp[u + 1] - rp[u];
            for (int64_t e = rp[u]; e < rp[u + 1]; e++) {
                int32_t v = col[e];
                if (dist[v] < 0) {
                    dist[v] = (int32_t)(level + 1);
                    order[no++] = v;
                }
            }
        }
        for (int64_t k = lend; k < no; k++) {
            int32_t w = order[k];
            double sum = 0.0;
            for (int64_t e = irp[w]; e < irp[w + 1]; e++) {
                int32_t u = icol[e];
                if (dist[u] == level) sum += sigma[u];
            }
            sigma[w] = sum;
            if (sum >= 0x1p53 && overflow) *overflow = 1;
        }
        lstart = lend;
        if (lend == no) break;
        level++;
    }
    if (norder) *norder = no;
    if (edges) *edges = e_scanned;
    if (t >= 0) return dist[t];
    int64_t ecc = 0;
    for (int64_t k = 0; k < no; k++)
        if (dist[order[k]] > ecc) ecc = dist[order[k]];
    return ecc;
}

/* RandomSP backtrack (Section III-B; a uniform path of Gamma_st, as in the
 * importance distribution q of Section III-A): from w = t, step r draws
 * u_r in (0,1] (Philox counter (i, tag, r/2), component r%2) and moves to the
 * first predecessor, in in-adjacency order, whose running sigma sum reaches
 * u_r * sigma_w.  Writes the internal nodes (t-side first) and returns
 * their number, or -1 when t was not reached. */
int32_t orc_backtrack(const int64_t *irp, const int32_t *icol, const int32_t *dist, const double *sigma, int32_t s,
                      int32_t t, uint64_t seed, uint32_t tag, uint64_t i, int32_t *path) {
    if (dist[t] < 0) return -1;
    int32_t w = t, k = 0;
    uint32_t r = 0;
    while (w != s) {
        double u[2];
        orc_uniforms(seed, i, tag, r >> 1, u);
        double target = u[r & 1] * sigma[w];
        double cum = 0.0;
        int32_t pick = -1;
        for (int64_t e = irp[w]; e < irp[w + 1]; e++) {
            int32_t p = icol[e];
            if (dist[p] == dist[w] - 1) {
                cum += sigma[p];
                if (cum >= target) {
                    pick = p;
                    break;
                }
            }
        }
        if (pick < 0) return -2; /* cannot happen for exact sigma */
        if (pick != s) path[k++] = pick;
        w = pick;
        r++;
    }
    return k;
}

/* RandomSP by a balanced bidirectional BFS (Section III-B).  The paper names
 * the traversal but not its details; this follows the reading stated here.
 * Forward side from s over out-edges, backward side from t over in-edges,
 * each with its own distance and path counts (sigma_s, sigma_t).  While both
 * frontiers are non-empty, expand one level of the side whose frontier has
 * the smaller sum of degrees in its direction (the forward side on a tie).
 * The first level L_a of a side that contains vertices the other side has
 * reached ends the search: with a the expanded side's new level and b the
 * other side's last level, every such vertex lies at distance b from the
 * other end, d(s,t) = a + b, and every shortest path crosses the layer
 * M = {v : d(s,v) = a_F} exactly once, so sigma_st = sum over M of
 * sigma_s(v) sigma_t(v).  The path: v in M with probability
 * sigma_s(v) sigma_t(v) / sigma_st (first v in vertex-id order whose running
 * sum reaches u_0 sigma_st), then the forward side backtracked from v to s and
 * the backward side from v to t, each step choosing among the next vertices
 * towards the end (in-CSR order towards s, out-CSR order towards t) the first
 * whose running count reaches u sigma(w) (uniform steps 1, 2, ...).
 * Internal nodes are written v first (unless v is s or t), then the s side
 * from v, then the t side from v.  Returns d(s,t), or -1 when a frontier
 * empties first (t unreachable).  *sst = sigma_st; *edges_out = edges scanned
 * by both sides. */
int32_t orc_bibfs(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *irp, const int32_t *icol,
                  int32_t s, int32_t t, uint64_t seed, uint32_t tag, uint64_t i, int32_t *path, int32_t *plen,
                  double *sst, int64_t *edges_out, int32_t *overflow) {
    int32_t *dist[2];
    double *sig[2];
    int32_t *queue[2];
    for (int x = 0; x < 2; x++) {
        dist[x] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        sig[x] = (double *)calloc((size_t)n, sizeof(double));
        queue[x] = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        for (int64_t v = 0; v < n; v++) dist[x][v] = -1;
    }
    const int64_t *ptr[2] = {rp, irp};  /* forward: out-edges; backward: in-edges */
    const int32_t *adj[2] = {col, icol};
    int32_t end[2] = {s, t};
    int64_t lo[2] = {0, 0}, hi[2] = {1, 1}; /* current frontier = queue[x][lo..hi) */
    int32_t lev[2] = {0, 0};
    int64_t cost[2];
    int64_t edges = 0;
    int32_t d = -1;
    *plen = 0;
    *sst = 0.0;
    for (int x = 0; x < 2; x++) {
        dist[x][end[x]] = 0;
        sig[x][end[x]] = 1.0;
        queue[x][0] = end[x];
        cost[x] = ptr[x][end[x] + 1] - ptr[x][end[x]];
    }
    int32_t *meet = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t nm = 0;
    if (s != t) {
        while (hi[0] > lo[0] && hi[1] > lo[1]) {
            const int x = cost[0] <= cost[1] ? 0 : 1, y = 1 - x;
            int64_t top = hi[x];
            /* discover level lev+1 */
            for (int64_t q = lo[x]; q < hi[x]; q++) {
                const int32_t u = queue[x][q];
                for (int64_t e = ptr[x][u]; e < ptr[x][u + 1]; e++) {
                    const int32_t v = adj[x][e];
                    edges++;
                    if (dist[x][v] < 0) {
                        dist[x][v] = lev[x] + 1;
                        queue[x][top++] = v;
                    }
                    if (dist[x][v] == lev[x] + 1) sig[x][v] += sig[x][u];
                }
            }
            lo[x] = hi[x];
            hi[x] = top;
            lev[x]++;
            cost[x] = 0;
            for (int64_t q = lo[x]; q < hi[x]; q++) {
                const int32_t v = queue[x][q];
                cost[x] += ptr[x][v + 1] - ptr[x][v];
                if (sig[x][v] >= 9007199254740992.0) *overflow = 1;
                if (dist[y][v] >= 0) meet[nm++] = v;
            }
            if (nm > 0) {
                d = lev[x] + dist[y][meet[0]];
                break;
            }
        }
    }
    if (d >= 0) {
        /* the meeting layer in vertex-id order (insertion sort of a small set) */
        for (int64_t a = 1; a < nm; a++) {
            const int32_t key = meet[a];
            int64_t b = a - 1;
            while (b >= 0 && meet[b] > key) {
                meet[b + 1] = meet[b];
                b--;
            }
            meet[b + 1] = key;
        }
        double total = 0.0;
        for (int64_t a = 0; a < nm; a++) total += sig[0][meet[a]] * sig[1][meet[a]];
        /* sigma_st (and each term sigma_s(v) sigma_t(v)) is a path count too: past
         * 2^53 the FP64 values are no longer exact */
        if (total >= 9007199254740992.0) *overflow = 1;
        *sst = total;
        double u[2];
        orc_uniforms(seed, i, tag, 0, u);
        const double target = u[0] * total;
        double cum = 0.0;
        int32_t v = meet[nm - 1];
        for (int64_t a = 0; a < nm; a++) {
            cum += sig[0][meet[a]] * sig[1][meet[a]];
            if (cum >= target) {
                v = meet[a];
                break;
            }
        }
        int32_t k = 0;
        if (v != s && v != t) path[k++] = v;
        uint32_t step = 1;
        for (int x = 0; x < 2; x++) {
            /* towards s: predecessors over in-edges; towards t: successors over out-edges */
            const int64_t *bp = x == 0 ? irp : rp;
            const int32_t *bc = x == 0 ? icol : col;
            int32_t w = v;
            while (w != end[x]) {
                orc_uniforms(seed, i, tag, step >> 1, u);
                const double tg = u[step & 1] * sig[x][w];
                double c2 = 0.0;
                int32_t pick = -1;
                for (int64_t e = bp[w]; e < bp[w + 1]; e++) {
                    const int32_t p2 = bc[e];
                    if (dist[x][p2] >= 0 && dist[x][p2] == dist[x][w] - 1) {
                        c2 += sig[x][p2];
                        if (c2 >= tg) {
                            pick = p2;
                            break;
                        }
                    }
                }
                if (pick < 0) {
                    d = -2;
                    break;
                }
                if (pick != end[x]) path[k++] = pick;
                w = pick;
                step++;
            }
            if (d < 0) break;
        }
        *plen = k;
    }
    *edges_out = edges;
    for (int x = 0; x < 2; x++) {
        free(dist[x]);
        free(sig[x]);
        free(queue[x]);
    }
    free(meet);
    return d;
}

/* All shortest paths at once (the Rao-Blackwellised form of the Section III-A
 * estimator: E over the uniform path of 1[v in I] is sigma_st(v)/sigma_st).
 * After the truncated BFS from s to t, tau_w = number of shortest w-t paths by
 * a reverse sweep from t over the shortest-path DAG (tau_t = 1,
 * tau_u = sum of tau_w over w with u in pred(w)), and every internal v gets
 * f(v) = sigma_sv * tau_v / sigma_st.  Writes the internal nodes and their f
 * (t-side levels first, each level in discovery order) and returns their
 * number, or -1 when t was not reached. */
int32_t orc_allpaths(int64_t n, const int64_t *irp, const int32_t *icol, const int32_t *dist, const double *sigma,
                     int32_t s, int32_t t, int32_t *nodes, double *frac) {
    if (dist[t] < 0) return -1;
    const int32_t d = dist[t];
    double *tau = (double *)calloc((size_t)n, sizeof(double));
    char *in = (char *)calloc((size_t)n, 1);
    int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t nc = 1, k = 0;
    cur[0] = t;
    tau[t] = 1.0;
    for (int32_t L = d - 1; L >= 1; L--) {
        int64_t nn = 0;
        for (int64_t q = 0; q < nc; q++) {
            const int32_t w = cur[q];
            for (int64_t e = irp[w]; e < irp[w + 1]; e++) {
                const int32_t p = icol[e];
                if (dist[p] != L) continue;
                if (!in[p]) {
                    in[p] = 1;
                    nxt[nn++] = p;
                }
                tau[p] += tau[w];
            }
        }
        for (int64_t q = 0; q < nn; q++) {
            const int32_t v = nxt[q];
            nodes[k] = v;
            frac[k] = sigma[v] * tau[v] / sigma[t];
            k++;
        }
        int32_t *tmp = cur;
        cur = nxt;
        nxt = tmp;
        nc = nn;
    }
    (void)s;
    free(tau);
    free(in);
    free(cur);
    free(nxt);
    return (int32_t)k;
}

/* One sampling phase of Algorithm 1 (Algorithm 2 + RandomSP + estimator).
 * Samples i0 .. i0+count-1: pair tag `tag_pair`, path tag `tag_path`.
 * kind[k]: 0 = path sampled, 1 = zero weight (R(x_s-x_t) = 0), 2 = t not
 *          reachable from s.
 * ilen[k]: |I(tau)| (0 unless kind = 0).
 * cnt[v] += 1 for every internal node (exact integer counts).
 * acc (optional): acc[v] += kappa(s,t,v)/kappa~(s,t) for every internal v,
 *   evaluated literally as (R/Cv[v]) / (R/C)  (Section III-A estimator).
 * path_ptr/path_nodes (optional): internal nodes of each sample.
 * edges (optional): out-edges a top-down truncated BFS from s scans
 *   before settling t (the whole reachable set when t is unreachable).
 * Returns 0, or -1 if path storage overflowed, -2 on an internal error. */
int orc_run_samples(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *irp, const int32_t *icol,
                    const double *x, const double *xs, const int32_t *perm, const double *w, const double *ci,
                    const double *r, double c, const double *Cv, uint64_t seed, uint32_t tag_pair, uint32_t tag_path,
                    int64_t i0, int64_t count, int32_t *s_out, int32_t *t_out, int32_t *kind, int32_t *ilen,
                    int64_t *cnt, double *acc, int64_t *path_ptr, int32_t *path_nodes, int64_t path_cap,
                    int64_t *edges, int32_t *overflow, double *acc_all, int bidir) {
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *sigma = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *apn = acc_all ? (int32_t *)malloc(sizeof(int32_t) * (size_t)n) : NULL;
    double *apf = acc_all ? (double *)malloc(sizeof(double) * (size_t)n) : NULL;
    int rc = 0;
    int64_t pp = 0;
    if (path_ptr) path_ptr[0] = 0;
    for (int64_t k = 0; k < count; k++) {
        uint64_t i = (uint64_t)(i0 + k);
        int32_t s, t;
        orc_sample_pairs(n, xs, perm, w, ci, r, c, seed, tag_pair, (int64_t)i, 1, &s, &t, NULL, NULL);
        s_out[k] = s;
        t_out[k] = t;
        double R = x[s] - x[t];
        int32_t len = 0;
        int64_t e_scanned = 0;
        if (!(R > 0.0)) {
            kind[k] = 1;
        } else {
            int64_t no;
            int64_t d;
            int32_t got = 0;
            if (bidir) {
                double sst;
                d = orc_bibfs(n, rp, col, irp, icol, s, t, seed, tag_path, i, path, &got, &sst, &e_scanned,
                              overflow);
                if (d == -2) {
                    rc = -2;
                    d = -1;
                }
            } else {
                d = orc_bfs(n, rp, col, irp, icol, s, t, dist, sigma, order, &no, &e_scanned, overflow);
            }
            if (d < 0) {
                kind[k] = 2;
            } else {
                if (!bidir) got = orc_backtrack(irp, icol, dist, sigma, s, t, seed, tag_path, i, path);
                if (got < 0) {
                    rc = -2;
                    got = 0;
                }
                kind[k] = 0;
                len = got;
                if (acc_all) {
                    /* all-paths form: kappa/kappa~ weighted fractions */
                    const int32_t na = orc_allpaths(n, irp, icol, dist, sigma, s, t, apn, apf);
                    for (int32_t q = 0; q < na; q++) acc_all[apn[q]] += (R / Cv[apn[q]]) / (R / c) * apf[q];
                }
                for (int32_t q = 0; q < got; q++) {
                    int32_t v = path[q];
                    cnt[v] += 1;
                    if (acc) acc[v] += (R / Cv[v]) / (R / c);
                }
                if (path_nodes) {
                    if (pp + got > path_cap) rc = -1;
                    else
                        for (int32_t q = 0; q < got; q++) path_nodes[pp + q] = path[q];
                }
                pp += got;
            }
        }
        ilen[k] = len;
        if (path_ptr) path_ptr[k + 1] = pp;
        if (edges) edges[k] = e_scanned;
    }
    free(dist);
    free(sigma);
    free(order);
    free(path);
    free(apn);
    free(apf);
    return rc;
}

/* ------------------------------------------------------- C_v and lambda_v */

/* Definition 1 denominator written out: Cv[v] = sum over (u,w), u != v != w,
 * of R(x_u - x_w).  O(n^3); tiny n only.  Also returns C = sum over all
 * pairs (u,w) of R(x_u - x_w) (Section III-A). */
double orc_cv_literal(int64_t n, const double *x, double *Cv) {
    double C = 0.0;
    for (int64_t u = 0; u < n; u++)
        for (int64_t w = 0; w < n; w++) C += fmax(0.0, x[u] - x[w]);
    for (int64_t v = 0; v < n; v++) {
        double s = 0.0;
        for (int64_t u = 0; u < n; u++) {
            if (u == v) continue;
            for (int64_t w = 0; w < n; w++) {
                if (w == v) continue;
                s += fmax(0.0, x[u] - x[w]);
            }
        }
        Cv[v] = s;
    }
    return C;
}

/* The same quantity in O(n^2): the pairs removed from C when v is excluded
 * are (v,w) and (u,v), whose ramps sum to |x_v - x_u| (proof of
 * Proposition 5).  Cv[v] = C - sum_u |x_v - x_u|. */
double orc_cv_direct(int64_t n, const double *x, double *Cv) {
    double C = 0.0;
    for (int64_t u = 0; u < n; u++)
        for (int64_t w = 0; w < n; w++) C += fmax(0.0, x[u] - x[w]);
    for (int64_t v = 0; v < n; v++) {
        double a = 0.0;
        for (int64_t u = 0; u < n; u++) a += fabs(x[v] - x[u]);
        Cv[v] = C - a;
    }
    return C;
}

/* The same in O(n) from the sorted states and Algorithm 2's suffix sums w:
 * for sorted position i, sum_j |x_i - x_j| = (w_1 - w_i) - (i-1) x_i
 * + (n-i) x_i - w_{i+1}; C is Algorithm 2's c.  Output in node order. */
void orc_cv_sorted(int64_t n, const double *xs, const int32_t *perm, const double *w, double c, double *Cv) {
    for (int64_t i = 1; i <= n; i++) {
        double xi = xs[i - 1];
        double a = (w[1] - w[i]) - (double)(i - 1) * xi + (double)(n - i) * xi - w[i + 1];
        Cv[perm[i - 1]] = c - a;
    }
}

/* ----------------------------------------------------------------- exact */

/* Exact percolation centrality (Definition 1) by a Brandes-style
 * dependency accumulation with target weights R(x_s - x_w), the extension of
 * Brandes' algorithm the paper uses for exact values (Section IV-A):
 *   delta_s(u) = sum over w with u in pred_s(w) of
 *                (sigma_su / sigma_sw) (R(x_s - x_w) + delta_s(w)),
 *   p(v) = sum over s != v of delta_s(v) / Cv[v].
 * pc[v] = NAN when Cv[v] = 0 (p undefined, Section II-A). */
void orc_exact_pc(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *irp, const int32_t *icol,
                  const double *x, const double *Cv, double *pc) {
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *sigma = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *delta = (double *)malloc(sizeof(double) * (size_t)n);
    double *num = (double *)calloc((size_t)n, sizeof(double));
    for (int32_t s = 0; s < n; s++) {
        int64_t no;
        orc_bfs(n, rp, col, irp, icol, s, -1, dist, sigma, order, &no, NULL, NULL);
        for (int64_t k = 0; k < no; k++) delta[order[k]] = 0.0;
        for (int64_t k = no - 1; k >= 1; k--) {
            int32_t wv = order[k];
            double coef = fmax(0.0, x[s] - x[wv]) + delta[wv];
            for (int64_t e = irp[wv]; e < irp[wv + 1]; e++) {
                int32_t u = icol[e];
                if (dist[u] == dist[wv] - 1) delta[u] += sigma[u] / sigma[wv] * coef;
            }
            num[wv] += delta[wv];
        }
    }
    for (int64_t v = 0; v < n; v++) pc[v] = Cv[v] > 0.0 ? num[v] / Cv[v] : NAN;
    free(dist);
    free(sigma);
    free(order);
    free(delta);
    free(num);
}

/* VertexDiamUB (Algorithm 1; Section III-B says one BFS gives a constant
 * factor bound on undirected graphs).  Reading: for every connected
 * component (taken in order of its largest-degree vertex, ties by id) run a
 * BFS from its largest-degree vertex; with eccentricity e every shortest path
 * of the component has at most 2e edges, so at most 2e-1 internal nodes.
 * Directed graphs: n-2 (always valid). */
int64_t orc_vertex_diam_ub(int64_t n, const int64_t *rp, const int32_t *col, int directed) {
    if (directed) return n >= 2 ? n - 2 : 0;
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *sigma = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    char *seen = (char *)calloc((size_t)n, 1);
    int64_t D = 0;
    for (;;) {
        int64_t best = -1, bdeg = 0;
        for (int64_t v = 0; v < n; v++) {
            int64_t dg = rp[v + 1] - rp[v];
            if (!seen[v] && dg > bdeg) {
                best = v;
                bdeg = dg;
            }
        }
        if (best < 0) break;
        int64_t no;
        int64_t ecc = orc_bfs(n, rp, col, rp, col, (int32_t)best, -1, dist, sigma, order, &no, NULL, NULL);
        for (int64_t k = 0; k < no; k++) seen[order[k]] = 1;
        int64_t b = 2 * ecc - 1;
        if (b > D) D = b;
    }
    free(dist);
    free(sigma);
    free(order);
    free(seen);
    return D;
}

/* ------------------------------------------------------------ gradients */

static double sgn(double a) { return (a > 0.0) - (a < 0.0); }

/* Vector-Jacobian product of the fixed-sample estimator
 *   F_v(x) = (Cbar/l) sum_i a_i(v) R(x_{s_i} - x_{t_i}) / (Rbar_i C_v(x))
 * (the Section III-A estimator with the sample and its sampling density held
 * at the states xbar where it was drawn, so F(xbar) = p~), at x = xbar:
 *   grad[u] = (Cbar/l) sum_i (1[u=s_i] - 1[u=t_i]) S_i / Rbar_i
 *             - sum_v gamma_v dC_v/dx_u,
 *   S_i = sum_{v in I_i} g_v / C_v,  gamma_v = g_v F_v / C_v,
 *   dC_v/dx_u = dC/dx_u - dA_v/dx_u, dC/dx_u = sum_w sgn(x_u - x_w),
 *   dA_v/dx_u = sgn(x_u - x_v) (u != v), sum_w sgn(x_v - x_w) (u = v).
 * The ramp's derivative at 0 is taken as 0.  Only the coordinates listed in
 * `us` are computed (each in O(n + sum |I|)); grad is indexed like us. */
void orc_vjp_fixed(int64_t n, const double *x, double C, const double *Cv, int64_t ell, int64_t count,
                   const int32_t *s, const int32_t *t, const int32_t *kind, const int64_t *path_ptr,
                   const int32_t *path_nodes, const double *F, const double *g, int64_t nu, const int64_t *us,
                   double *grad) {
    double *Si = (double *)malloc(sizeof(double) * (size_t)(count > 0 ? count : 1));
    for (int64_t i = 0; i < count; i++) {
        double acc = 0.0;
        for (int64_t q = path_ptr[i]; q < path_ptr[i + 1]; q++) acc += g[path_nodes[q]] / Cv[path_nodes[q]];
        Si[i] = acc;
    }
    for (int64_t k = 0; k < nu; k++) {
        int64_t u = us[k];
        double term1 = 0.0;
        for (int64_t i = 0; i < count; i++) {
            if (kind[i] != 0) continue;
            double Rb = x[s[i]] - x[t[i]];
            double coef = (C / (double)ell) * Si[i] / Rb;
            if (s[i] == u) term1 += coef;
            if (t[i] == u) term1 -= coef;
        }
        double dC = 0.0;
        for (int64_t wv = 0; wv < n; wv++) dC += sgn(x[u] - x[wv]);
        double term2 = 0.0;
        for (int64_t v = 0; v < n; v++) {
            double gam = g[v] * F[v] / Cv[v];
            double dA = (v != u) ? sgn(x[u] - x[v]) : dC;
            term2 += gam * (dC - dA);
        }
        grad[k] = term1 - term2;
    }
    free(Si);
}

/* Vector-Jacobian product of the exact percolation centrality (Definition 1),
 * sum_v g_v dp(v)/dx_u, with p(v) = N_v / C_v and
 * N_v = sum_{s,t} R(x_s - x_t) sigma_st(v)/sigma_st:
 *   dN_v/dx_u = sum_t R'(x_u - x_t) f_ut(v) - sum_s R'(x_s - x_u) f_su(v).
 * With h_v = g_v / C_v the first sum is a dependency accumulation from
 * source u with target weights 1[x_u > x_t]; the second uses the forward
 * path sum T_s(w) = sum_{u in pred(w)} (T_s(u) + h_u sigma_su [u != s]),
 * which equals sum_v h_v sigma_sv sigma_vw over internal v. */
void orc_exact_vjp(int64_t n, const int64_t *rp, const int32_t *col, const int64_t *irp, const int32_t *icol,
                   const double *x, const double *Cv, const double *pc, const double *g, double *grad) {
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *sigma = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *delta = (double *)malloc(sizeof(double) * (size_t)n);
    double *T = (double *)malloc(sizeof(double) * (size_t)n);
    double *h = (double *)malloc(sizeof(double) * (size_t)n);
    double *term1 = (double *)calloc((size_t)n, sizeof(double));
    double *term2 = (double *)calloc((size_t)n, sizeof(double));
    for (int64_t v = 0; v < n; v++) h[v] = g[v] / Cv[v];
    for (int32_t s = 0; s < n; s++) {
        int64_t no;
        orc_bfs(n, rp, col, irp, icol, s, -1, dist, sigma, order, &no, NULL, NULL);
        for (int64_t k = 0; k < no; k++) delta[order[k]] = 0.0;
        for (int64_t k = no - 1; k >= 1; k--) {
            int32_t wv = order[k];
            double coef = (x[s] > x[wv] ? 1.0 : 0.0) + delta[wv];
            for (int64_t e = irp[wv]; e < irp[wv + 1]; e++) {
                int32_t u = icol[e];
                if (dist[u] == dist[wv] - 1) delta[u] += sigma[u] / sigma[wv] * coef;
            }
        }
        double acc = 0.0;
        for (int64_t k = 1; k < no; k++) acc += h[order[k]] * delta[order[k]];
        term1[s] += acc;
        T[s] = 0.0;
        for (int64_t k = 1; k < no; k++) {
            int32_t wv = order[k];
            double tw = 0.0;
            for (int64_t e = irp[wv]; e < irp[wv + 1]; e++) {
                int32_t u = icol[e];
                if (dist[u] == dist[wv] - 1) tw += T[u] + (u != s ? h[u] * sigma[u] : 0.0);
            }
            T[wv] = tw;
            if (x[s] > x[wv]) term2[wv] += tw / sigma[wv];
        }
    }
    for (int64_t u = 0; u < n; u++) {
        double dC = 0.0;
        for (int64_t wv = 0; wv < n; wv++) dC += sgn(x[u] - x[wv]);
        double t3 = 0.0;
        for (int64_t v = 0; v < n; v++) {
            double dA = (v != u) ? sgn(x[u] - x[v]) : dC;
            t3 += g[v] * pc[v] * (dC - dA) / Cv[v];
        }
        grad[u] = term1[u] - term2[u] - t3;
    }
    free(dist);
    free(sigma);
    free(order);
    free(delta);
    free(T);
    free(h);
    free(term1);
    free(term2);
}
