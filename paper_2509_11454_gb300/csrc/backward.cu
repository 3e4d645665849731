// Adjoint of the fixed-sample estimator (importance-sampling gradient; not
// in the paper).  With the phase-2 sample held fixed,
//   F_v(x) = (C/l) sum_i a_i(v) R(x_{s_i} - x_{t_i}) / (R_i C_v(x)),
// so F = p~ at the current states, and for an upstream gradient g
//   grad[u] = (C/l) sum_i (1[u = s_i] - 1[u = t_i]) S_i / R_i
//             - (Gamma D_u - (P_<(u) - P_>(u)) - gamma_u D_u),
//   S_i = sum_{v in I_i} g_v / C_v,   gamma_v = g_v F_v / C_v,
//   Gamma = sum_v gamma_v,  D_u = #{w: x_w < x_u} - #{w: x_w > x_u},
//   P_<(u), P_>(u) = sum of gamma over states below / above x_u.
// (dC/dx_u = D_u, dA_v/dx_u = sgn(x_u - x_v) for v != u and D_u for v = u,
// with the ramp's derivative at 0 taken as 0.)  The P sums come from one
// exclusive scan of gamma in sorted-state order and the tie groups.
#include "common.cuh"
#include "internal.h"

namespace percis {

namespace {

__global__ void k_bw_samples(int64_t count, const int32_t *s, const int32_t *t, const int32_t *kind,
                             const int32_t *ilen, const long long *path_off, const int32_t *arena, const double *g,
                             const double *Cv, const double *x, const double *dscal, double ell, double *grad) {
    const double C = dscal[0];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        if (kind[i] != 0) continue;
        const int32_t si = s[i], ti = t[i];
        const long long off = path_off[i];
        double S = 0.0;
        for (int q = 0; q < ilen[i]; ++q) {
            const int32_t v = arena[off + q];
            S += g[v] / Cv[v];
        }
        const double coef = (C / ell) * S / (x[si] - x[ti]);
        atomicAdd(&grad[si], coef);
        atomicAdd(&grad[ti], -coef);
    }
}

__global__ void k_bw_gamma(int64_t n, const int32_t *perm, const double *g, const double *lam,
                           const unsigned long long *cnt, const double *Cv, double ell, double *gs) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t v = perm[i];
        const double F = lam[v] * (double)cnt[v] / ell;
        gs[i] = g[v] * F / Cv[v];
    }
}

__global__ void k_bw_final(int64_t n, const int32_t *perm, const int32_t *glo, const int32_t *ghi, const double *gs,
                           const double *G, double *grad) {
    const double Gamma = G[n];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int32_t u = perm[i];
        const int64_t lo = glo[i], hi = ghi[i];  // 1-based tie group of position i+1
        const double P_gt = G[lo - 1];
        const double P_lt = Gamma - G[hi];
        const double Du = (double)((n - hi) - (lo - 1));
        const double term = Gamma * Du - (P_lt - P_gt) - gs[i] * Du;
        grad[u] -= term;
    }
}

}  // namespace

percis_status backward_fixed(percis_ctx *ctx, const double *g, double *grad) {
    const int64_t n = ctx->n, count = ctx->phase_count;
    PERCIS_CUDA(ctx, cudaMemsetAsync(grad, 0, sizeof(double) * n, ctx->stream));
    const int block = 256;
    k_bw_samples<<<grid_for(ctx, count, block), block, 0, ctx->stream>>>(
        count, ctx->pair_s.as<int32_t>(), ctx->pair_t.as<int32_t>(), ctx->kind.as<int32_t>(),
        ctx->ilen.as<int32_t>(), ctx->path_off.as<long long>(), ctx->arena.as<int32_t>(), g, ctx->Cv.as<double>(),
        ctx->x.as<double>(), ctx->dscal.as<double>(), (double)ctx->last_ell, grad);
    PERCIS_CHECK_LAUNCH(ctx, "backward samples");
    PERCIS_TRY(ensure(ctx, ctx->grad_tmp, sizeof(double) * (2 * n + 2), "backward scan"));
    double *gs = ctx->grad_tmp.as<double>();
    double *G = gs + n;
    k_bw_gamma<<<grid_for(ctx, n, block), block, 0, ctx->stream>>>(n, ctx->perm.as<int32_t>(), g,
                                                                  ctx->lam.as<double>(),
                                                                  ctx->cnt.as<unsigned long long>(),
                                                                  ctx->Cv.as<double>(), (double)ctx->last_ell, gs);
    PERCIS_CHECK_LAUNCH(ctx, "backward gamma");
    PERCIS_TRY(scan_exclusive_f64(ctx, gs, G, n));
    PERCIS_TRY(prep_groups(ctx));
    k_bw_final<<<grid_for(ctx, n, block), block, 0, ctx->stream>>>(n, ctx->perm.as<int32_t>(),
                                                                  ctx->grp_lo.as<int32_t>(),
                                                                  ctx->grp_hi.as<int32_t>(), gs, G, grad);
    PERCIS_CHECK_LAUNCH(ctx, "backward final");
    return PERCIS_OK;
}

}  // namespace percis
