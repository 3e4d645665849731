// Preprocessing kernels: CSR validation and transpose, the stable sort of
// the percolation states, Algorithm 2's tables, C_v, lambda_v and d^.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace percis {

namespace {

// ------------------------------------------------------------- validation

__global__ void k_check_csr(const int64_t *rp, const int32_t *col, int64_t n, int64_t nnz, uint32_t *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (rp[v] > rp[v + 1] || rp[v] < 0 || rp[v + 1] > nnz) atomicOr(status, 1u);
        if (v == 0 && (rp[0] != 0 || rp[n] != nnz)) atomicOr(status, 1u);
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
        const int32_t c = col[e];
        if (c < 0 || (int64_t)c >= n) atomicOr(status, 1u);
    }
}

__global__ void k_check_states(const double *x, int64_t n, uint32_t *status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const double a = x[v];
        if (!(a >= 0.0 && a <= 1.0)) atomicOr(status, DEV_BAD_STATE);
    }
}

// ----------------------------------------------------------- merge sort
// Stable bottom-up merge sort of (key, val) pairs: in a pass of width w an
// element of the left run lands at (its rank in its run) + (number of
// right-run keys < key); an element of the right run at (its rank) +
// (number of left-run keys <= key).  Equal keys keep their input order.

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t *a, int64_t lo, int64_t hi, uint64_t key) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int64_t upper_bound_u64(const uint64_t *a, int64_t lo, int64_t hi, uint64_t key) {
    while (lo < hi) {
        const int64_t mid = lo + ((hi - lo) >> 1);
        if (a[mid] <= key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void k_merge_pass(const uint64_t *kin, const int32_t *vin, uint64_t *kout, int32_t *vout, int64_t n,
                             int64_t w) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t run = i / w;
        const uint64_t key = kin[i];
        int64_t out;
        if ((run & 1) == 0) {
            const int64_t a0 = run * w;
            const int64_t b0 = a0 + w;
            const int64_t b1 = min(b0 + w, n);
            const int64_t rank = b0 < n ? lower_bound_u64(kin, b0, b1, key) - b0 : 0;
            out = a0 + (i - a0) + rank;
        } else {
            const int64_t b0 = run * w;
            const int64_t a0 = b0 - w;
            out = a0 + (i - b0) + (upper_bound_u64(kin, a0, b0, key) - a0);
        }
        kout[out] = key;
        vout[out] = vin[i];
    }
}

// ---------------------------------------------------------- state keys

__global__ void k_state_keys(const double *x, int64_t n, uint64_t *keys, int32_t *vals) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const double a = x[v] + 0.0;  // -0.0 -> +0.0
        // x >= 0: larger value <-> larger bit pattern; complement sorts descending
        keys[v] = ~(uint64_t)__double_as_longlong(a);
        vals[v] = (int32_t)v;
    }
}

__global__ void k_gather_sorted(const double *x, const int32_t *perm, int64_t n, double *xs) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) xs[i] = x[perm[i]] + 0.0;
}

// ------------------------------------------------------- Algorithm 2 scan
// The preprocessing recurrence of Algorithm 2 is evaluated sequentially in
// exactly its order (i = n down to 1) so that w, c_i, r and c are
// bit-identical to any other sequential evaluation: the sampled pairs depend
// on them through exact comparisons.
//
// On this GPU a warp-wide FP64 add occupies its sub-partition's FP64 pipe for
// ~64 cycles, so one thread can retire about one FP64 operation per 64 cycles
// whatever the dependences.  The three sequential parts therefore run on
// different warps (different sub-partitions) and everything parallel runs on
// the rest of the block:
//   warp 0 (one lane):  w_i = w_{i+1} + x_i                 (one add per element)
//   warps 2..7:         c_i = max(0, (n-i+1) x_i - w_i)     (parallel)
//   warp 1 (one lane):  r_i = r_{i+1} + c_i                 (one add per element)
// and c = r_1 (Algorithm 2 accumulates c over the same c_i in the same order
// as r).  Tiles of 512 elements flow through a four-slot ring, one stage per
// tile: stage s loads tile s, adds w over tile s-1, computes c_i of tile s-2,
// adds r over tile s-3 and writes tile s-4 out.
constexpr int kTile = 512;
constexpr int kRing = 4;

struct TableSlots {
    double x[kRing][kTile], t[kRing][kTile], w[kRing][kTile], c[kRing][kTile], r[kRing][kTile];
};

// Number of non-zero sorted states (xs is non-increasing and >= 0, so the
// zeros form a suffix), by bisection, into the int64 word at dscal + 2.
__global__ void k_nonzero_prefix(const double *xs, int64_t n, double *dscal) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int64_t lo = 0, hi = n;  // first zero in [lo, hi]
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (xs[mid] == 0.0) hi = mid;
        else lo = mid + 1;
    }
    *reinterpret_cast<long long *>(dscal + 2) = (long long)lo;
}

__global__ void __launch_bounds__(256) k_tables(const double *xs, int64_t n, double *w, double *ci, double *r,
                                                double *dscal) {
    extern __shared__ __align__(16) unsigned char smem[];
    TableSlots &S = *reinterpret_cast<TableSlots *>(smem);
    // positions past the last non-zero state: x_i = 0 and every sum before them
    // is +0, so w_i = c_i = r_i = 0 exactly; the scans start at the last non-zero one
    const int64_t nz = *reinterpret_cast<const long long *>(dscal + 2);
    for (int64_t i = nz + 1 + threadIdx.x; i <= n; i += blockDim.x) w[i] = ci[i] = r[i] = 0.0;
    const int64_t T = (nz + kTile - 1) / kTile;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wtid = threadIdx.x - 64, wcount = blockDim.x - 64;  // warps 2.. form the worker group
    if (threadIdx.x == 0) {
        w[n + 1] = 0.0;
        r[n + 1] = 0.0;
        ci[n + 1] = 0.0;
        w[0] = r[0] = ci[0] = 0.0;
    }
    double wn = 0.0, rn = 0.0;
    // tile s covers positions i in [hi - cnt + 1, hi], hi = n - s * kTile; local k = i - lo
    for (int64_t st = 0; st < T + 4; ++st) {
        if (warp >= 2) {
            const int64_t so = st - 4;  // write out
            if (so >= 0 && so < T) {
                const int slot = (int)(so % kRing);
                const int64_t hi = nz - so * kTile;
                const int cnt = (int)min((int64_t)kTile, hi);
                const int64_t lo = hi - cnt + 1;
                for (int k = wtid; k < cnt; k += wcount) {
                    w[lo + k] = S.w[slot][k];
                    ci[lo + k] = S.c[slot][k];
                    r[lo + k] = S.r[slot][k];
                }
            }
            if (st < T) {  // load tile st
                const int slot = (int)(st % kRing);
                const int64_t hi = nz - st * kTile;
                const int cnt = (int)min((int64_t)kTile, hi);
                const int64_t lo = hi - cnt + 1;
                for (int k = wtid; k < cnt; k += wcount) {
                    const int64_t i = lo + k;
                    const double xi = xs[i - 1];
                    S.x[slot][k] = xi;
                    S.t[slot][k] = __dmul_rn((double)(n - i + 1), xi);
                }
            }
            const int64_t sc = st - 2;  // c_i of tile st-2
            if (sc >= 0 && sc < T) {
                const int slot = (int)(sc % kRing);
                const int cnt = (int)min((int64_t)kTile, nz - sc * kTile);
                for (int k = wtid; k < cnt; k += wcount) {
                    const double cv = __dsub_rn(S.t[slot][k], S.w[slot][k]);
                    S.c[slot][k] = __double_as_longlong(cv) < 0 ? 0.0 : cv;
                }
            }
        } else if (warp == 0 && lane == 0) {
            const int64_t sw = st - 1;  // w over tile st-1
            if (sw >= 0 && sw < T) {
                const int slot = (int)(sw % kRing);
                const int cnt = (int)min((int64_t)kTile, nz - sw * kTile);
                int k = cnt - 1;
                // x is non-increasing in i, so a tile whose largest state (k = 0)
                // is zero holds only zeros; while w is still zero, each sum is
                // exactly +0 and the dependent adds can be skipped
                if (wn == 0.0 && S.x[slot][0] == 0.0) {
                    for (; k >= 0; --k) S.w[slot][k] = 0.0;
                }
                for (; k >= 7; k -= 8) {  // operands loaded ahead of the dependent adds
                    double v[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = S.x[slot][k - j];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        wn = __dadd_rn(wn, v[j]);
                        S.w[slot][k - j] = wn;
                    }
                }
                for (; k >= 0; --k) {
                    wn = __dadd_rn(wn, S.x[slot][k]);
                    S.w[slot][k] = wn;
                }
            }
        } else if (warp == 1 && lane == 0) {
            const int64_t sr = st - 3;  // r over tile st-3
            if (sr >= 0 && sr < T) {
                const int slot = (int)(sr % kRing);
                const int cnt = (int)min((int64_t)kTile, nz - sr * kTile);
                int k = cnt - 1;
                // an all-zero tile of states has w = 0 and so c = 0 throughout
                if (rn == 0.0 && S.x[slot][0] == 0.0) {
                    for (; k >= 0; --k) S.r[slot][k] = 0.0;
                }
                for (; k >= 7; k -= 8) {
                    double v[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) v[j] = S.c[slot][k - j];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        rn = __dadd_rn(rn, v[j]);
                        S.r[slot][k - j] = rn;
                    }
                }
                for (; k >= 0; --k) {
                    rn = __dadd_rn(rn, S.c[slot][k]);
                    S.r[slot][k] = rn;
                }
            }
        }
        __syncthreads();
    }
    if (warp == 1 && lane == 0) dscal[0] = rn;  // c = r_1
}

// C_v = c - A_v with A_i = (w_1 - w_i) - (i-1) x_i + (n-i) x_i - w_{i+1} for
// sorted position i (the closed form of sum_u |x_i - x_u|), lambda = c / C_v.
__global__ void k_cv_lambda(const double *xs, const int32_t *perm, const double *w, const double *dscal, int64_t n,
                            double *Cv, double *lam, uint32_t *status) {
    const double c = dscal[0];
    const double w1 = w[1];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x + 1; i <= n; i += stride) {
        const double xi = xs[i - 1];
        double a = __dsub_rn(w1, w[i]);
        a = __dsub_rn(a, __dmul_rn((double)(i - 1), xi));
        a = __dadd_rn(a, __dmul_rn((double)(n - i), xi));
        a = __dsub_rn(a, w[i + 1]);
        const double cv = __dsub_rn(c, a);
        const int32_t v = perm[i - 1];
        Cv[v] = cv;
        if (cv > 0.0) {
            lam[v] = __ddiv_rn(c, cv);
        } else {
            lam[v] = __longlong_as_double(0x7ff0000000000000LL);
            atomicOr(status, DEV_DEGENERATE);
        }
    }
}

__device__ __forceinline__ void atomic_max_pos_double(double *addr, double v) {
    // non-negative doubles order like their bit patterns
    atomicMax((unsigned long long *)addr, (unsigned long long)__double_as_longlong(v));
}

__global__ void k_max_lambda(const double *lam, int64_t n, double *dscal) {
    double m = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) m = fmax(m, lam[v]);
    for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) atomic_max_pos_double(&dscal[1], m);
}

// Tie groups of the sorted states: positions [lo, hi] (1-based) with equal x.
__global__ void k_groups(const double *xs, int64_t n, int32_t *glo, int32_t *ghi) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double v = xs[i];
        // xs is non-increasing: first index with xs <= v, last index with xs >= v
        int64_t lo = 0, hi = i;
        while (lo < hi) {
            const int64_t m = (lo + hi) >> 1;
            if (xs[m] > v) lo = m + 1;
            else hi = m;
        }
        int64_t a = i, b = n - 1;
        while (a < b) {
            const int64_t m = (a + b + 1) >> 1;
            if (xs[m] < v) b = m - 1;
            else a = m;
        }
        glo[i] = (int32_t)(lo + 1);
        ghi[i] = (int32_t)(a + 1);
    }
}

// ------------------------------------------------------------- transpose

__global__ void k_edge_keys(const int64_t *rp, const int32_t *col, int64_t n, uint64_t *keys, int32_t *vals) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        for (int64_t e = rp[u]; e < rp[u + 1]; ++e) {
            keys[e] = ((uint64_t)(uint32_t)col[e] << 32) | (uint32_t)u;
            vals[e] = (int32_t)u;
        }
    }
}

// key(v) = (highest-degree out-neighbour of v, ties to the smallest id) << 32 | v;
// vertices without neighbours use themselves.
__global__ void k_hub_keys(const int64_t *rp, const int32_t *col, int64_t n, uint64_t *keys, int32_t *vals) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        int32_t best = (int32_t)v;
        int64_t bdeg = -1;
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
            const int32_t u = col[e];
            const int64_t d = rp[u + 1] - rp[u];
            if (d > bdeg || (d == bdeg && u < best)) {
                bdeg = d;
                best = u;
            }
        }
        keys[v] = ((uint64_t)(uint32_t)best << 32) | (uint32_t)v;
        vals[v] = (int32_t)v;
    }
}


__global__ void k_indeg(const int32_t *col, int64_t nnz, long long *cnt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride)
        atomicAdd((unsigned long long *)&cnt[col[e]], 1ULL);
}

}  // namespace

// Stable sort of (keys, vals) in place using the given scratch (same sizes).
static percis_status merge_sort(percis_ctx *ctx, uint64_t *keys, int32_t *vals, uint64_t *k2, int32_t *v2, int64_t n) {
    uint64_t *ka = keys, *kb = k2;
    int32_t *va = vals, *vb = v2;
    const int grid = grid_for(ctx, n, 256);
    for (int64_t w = 1; w < n; w <<= 1) {
        k_merge_pass<<<grid, 256, 0, ctx->stream>>>(ka, va, kb, vb, n, w);
        PERCIS_CHECK_LAUNCH(ctx, "merge pass");
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {
        PERCIS_CUDA(ctx, cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
        PERCIS_CUDA(ctx, cudaMemcpyAsync(vals, va, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
    }
    return PERCIS_OK;
}

// Lane order of batched sources: vertices sorted by (highest-degree neighbour,
// id).  Only the batched form needs it, so it is built on first use.
percis_status prep_vorder(percis_ctx *ctx) {
    if (ctx->vorder_ready) return PERCIS_OK;
    const int64_t n = ctx->n;
    {
        PERCIS_TRY(ensure(ctx, ctx->vorder, sizeof(int32_t) * n, "vertex order"));
        DevBuf k1, k2, v2;
        cudaError_t e = cudaMalloc(&k1.p, sizeof(uint64_t) * n);
        if (e == cudaSuccess) e = cudaMalloc(&k2.p, sizeof(uint64_t) * n);
        if (e == cudaSuccess) e = cudaMalloc(&v2.p, sizeof(int32_t) * n);
        percis_status rs = PERCIS_OK;
        if (e != cudaSuccess) {
            cudaGetLastError();
            rs = set_err(ctx, PERCIS_E_OOM, "vertex order scratch");
        } else {
            k_hub_keys<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(ctx->rp.as<int64_t>(), ctx->col.as<int32_t>(),
                                                                     n, k1.as<uint64_t>(), ctx->vorder.as<int32_t>());
            ctx->launches++;
            rs = merge_sort(ctx, k1.as<uint64_t>(), ctx->vorder.as<int32_t>(), k2.as<uint64_t>(), v2.as<int32_t>(), n);
        }
        cudaStreamSynchronize(ctx->stream);
        cudaFree(k1.p);
        cudaFree(k2.p);
        cudaFree(v2.p);
        if (rs != PERCIS_OK) return rs;
    }
    ctx->vorder_ready = true;
    return PERCIS_OK;
}

percis_status prep_graph(percis_ctx *ctx) {
    const int64_t n = ctx->n, nnz = ctx->nnz;
    PERCIS_TRY(ensure(ctx, ctx->status, 64, "status"));
    uint32_t *st = ctx->status.as<uint32_t>();
    PERCIS_CUDA(ctx, cudaMemsetAsync(st, 0, 64, ctx->stream));
    k_check_csr<<<grid_for(ctx, std::max(n, nnz), 256), 256, 0, ctx->stream>>>(ctx->rp.as<int64_t>(),
                                                                             ctx->col.as<int32_t>(), n, nnz, st);
    PERCIS_CHECK_LAUNCH(ctx, "check csr");
    uint32_t hst = 0;
    PERCIS_CUDA(ctx, cudaMemcpyAsync(&hst, st, 4, cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (hst) return set_err(ctx, PERCIS_E_INVALID, "malformed CSR (row_ptr not monotone or column out of range)");

    if (ctx->directed) {
        PERCIS_TRY(ensure(ctx, ctx->irp, sizeof(int64_t) * (n + 1), "in-CSR offsets"));
        PERCIS_TRY(ensure(ctx, ctx->icol, sizeof(int32_t) * std::max<int64_t>(nnz, 1), "in-CSR columns"));
        DevBuf k1, k2, v2;
        size_t kb = sizeof(uint64_t) * std::max<int64_t>(nnz, 1);
        cudaError_t e = cudaMalloc(&k1.p, kb);
        if (e == cudaSuccess) e = cudaMalloc(&k2.p, kb);
        if (e == cudaSuccess) e = cudaMalloc(&v2.p, sizeof(int32_t) * std::max<int64_t>(nnz, 1));
        percis_status rs = PERCIS_OK;
        if (e != cudaSuccess) {
            rs = set_err(ctx, PERCIS_E_OOM, "transpose scratch");
        } else {
            int32_t *icol = ctx->icol.as<int32_t>();
            k_edge_keys<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(ctx->rp.as<int64_t>(), ctx->col.as<int32_t>(),
                                                                      n, k1.as<uint64_t>(), icol);
            ctx->launches++;
            rs = merge_sort(ctx, k1.as<uint64_t>(), icol, k2.as<uint64_t>(), v2.as<int32_t>(), nnz);
            if (rs == PERCIS_OK) {
                long long *cnt = (long long *)ctx->irp.as<int64_t>();
                // in-degree counts into a temporary, then exclusive scan into irp
                DevBuf tmp;
                e = cudaMalloc(&tmp.p, sizeof(long long) * (n + 1));
                if (e != cudaSuccess) rs = set_err(ctx, PERCIS_E_OOM, "in-degree scratch");
                else {
                    cudaMemsetAsync(tmp.p, 0, sizeof(long long) * (n + 1), ctx->stream);
                    k_indeg<<<grid_for(ctx, nnz, 256), 256, 0, ctx->stream>>>(ctx->col.as<int32_t>(), nnz,
                                                                            tmp.as<long long>());
                    ctx->launches++;
                    rs = scan_exclusive_i64(ctx, tmp.as<int64_t>(), (int64_t *)cnt, n);
                    cudaStreamSynchronize(ctx->stream);
                    cudaFree(tmp.p);
                }
            }
        }
        cudaStreamSynchronize(ctx->stream);
        cudaFree(k1.p);
        cudaFree(k2.p);
        cudaFree(v2.p);
        if (rs != PERCIS_OK) return rs;
        PERCIS_CUDA(ctx, cudaGetLastError());
    }
    ctx->vorder_ready = false;  // built on first use by the batched form
    if (!ctx->skip_diam) {
        int64_t D = 0;
        PERCIS_TRY(vertex_diam_ub(ctx, &D));
        ctx->vertex_diam = D;
    }
    return PERCIS_OK;
}

percis_status prep_states(percis_ctx *ctx) {
    const int64_t n = ctx->n;
    uint32_t *st = ctx->status.as<uint32_t>();
    PERCIS_CUDA(ctx, cudaMemsetAsync(st, 0, 64, ctx->stream));
    k_check_states<<<grid_for(ctx, n, 256), 256, 0, ctx->stream>>>(ctx->x.as<double>(), n, st);
    PERCIS_CHECK_LAUNCH(ctx, "check states");

    PERCIS_TRY(ensure(ctx, ctx->xs, sizeof(double) * n, "xs"));
    PERCIS_TRY(ensure(ctx, ctx->perm, sizeof(int32_t) * n, "perm"));
    PERCIS_TRY(ensure(ctx, ctx->w, sizeof(double) * (n + 2), "w"));
    PERCIS_TRY(ensure(ctx, ctx->ci, sizeof(double) * (n + 2), "ci"));
    PERCIS_TRY(ensure(ctx, ctx->r, sizeof(double) * (n + 2), "r"));
    PERCIS_TRY(ensure(ctx, ctx->Cv, sizeof(double) * n, "Cv"));
    PERCIS_TRY(ensure(ctx, ctx->lam, sizeof(double) * n, "lambda"));
    PERCIS_TRY(ensure(ctx, ctx->grp_lo, sizeof(int32_t) * n, "groups"));
    PERCIS_TRY(ensure(ctx, ctx->grp_hi, sizeof(int32_t) * n, "groups"));
    PERCIS_TRY(ensure(ctx, ctx->dscal, 64, "scalars"));
    // sort scratch: keys, keys2, vals2 (reuse the sigma buffer space if large)
    PERCIS_TRY(ensure(ctx, ctx->pc_tmp, (sizeof(uint64_t) * 2 + sizeof(int32_t)) * n + 64, "sort scratch"));
    uint64_t *k1 = ctx->pc_tmp.as<uint64_t>();
    uint64_t *k2 = k1 + n;
    int32_t *v2 = (int32_t *)(k2 + n);
    int32_t *perm = ctx->perm.as<int32_t>();
    const int g = grid_for(ctx, n, 256);
    k_state_keys<<<g, 256, 0, ctx->stream>>>(ctx->x.as<double>(), n, k1, perm);
    PERCIS_CHECK_LAUNCH(ctx, "state keys");
    PERCIS_TRY(merge_sort(ctx, k1, perm, k2, v2, n));
    k_gather_sorted<<<g, 256, 0, ctx->stream>>>(ctx->x.as<double>(), perm, n, ctx->xs.as<double>());
    PERCIS_CHECK_LAUNCH(ctx, "gather sorted");
    static bool smem_set = false;
    if (!smem_set) {
        PERCIS_CUDA(ctx, cudaFuncSetAttribute(k_tables, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              (int)sizeof(TableSlots)));
        smem_set = true;
    }
    k_nonzero_prefix<<<1, 32, 0, ctx->stream>>>(ctx->xs.as<double>(), n, ctx->dscal.as<double>());
    PERCIS_CHECK_LAUNCH(ctx, "non-zero states");
    k_tables<<<1, 256, sizeof(TableSlots), ctx->stream>>>(ctx->xs.as<double>(), n, ctx->w.as<double>(),
                                                         ctx->ci.as<double>(), ctx->r.as<double>(),
                                                         ctx->dscal.as<double>());
    PERCIS_CHECK_LAUNCH(ctx, "tables");
    PERCIS_CUDA(ctx, cudaMemsetAsync(ctx->dscal.as<double>() + 1, 0, sizeof(double), ctx->stream));
    k_cv_lambda<<<g, 256, 0, ctx->stream>>>(ctx->xs.as<double>(), perm, ctx->w.as<double>(), ctx->dscal.as<double>(),
                                            n, ctx->Cv.as<double>(), ctx->lam.as<double>(), st);
    PERCIS_CHECK_LAUNCH(ctx, "cv lambda");
    k_max_lambda<<<g, 256, 0, ctx->stream>>>(ctx->lam.as<double>(), n, ctx->dscal.as<double>());
    PERCIS_CHECK_LAUNCH(ctx, "max lambda");
    k_groups<<<g, 256, 0, ctx->stream>>>(ctx->xs.as<double>(), n, ctx->grp_lo.as<int32_t>(),
                                         ctx->grp_hi.as<int32_t>());
    PERCIS_CHECK_LAUNCH(ctx, "tie groups");
    double sc[2];
    uint32_t hst = 0;
    PERCIS_CUDA(ctx, cudaMemcpyAsync(sc, ctx->dscal.p, sizeof(sc), cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaMemcpyAsync(&hst, st, 4, cudaMemcpyDeviceToHost, ctx->stream));
    PERCIS_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (hst & DEV_BAD_STATE) return set_err(ctx, PERCIS_E_INVALID, "states must lie in [0,1] (no NaN)");
    ctx->c_host = sc[0];
    ctx->dhat_host = sc[1];
    if (hst & DEV_DEGENERATE)
        return set_err(ctx, PERCIS_E_DEGENERATE, "some C_v <= 0: percolation centrality undefined (all other states equal)");
    return PERCIS_OK;
}

}  // namespace percis
