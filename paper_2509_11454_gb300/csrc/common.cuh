// Device helpers shared by the PercIS kernels: Philox4x32-10 uniforms, a
// bounded grid-wide barrier for cooperative launches, warp scans, and the
// status bits kernels report to the host.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace percis {

// Status bits written by kernels into a device word (atomicOr).
enum : uint32_t {
    DEV_TIMEOUT = 1u << 0,         // a bounded wait ran out
    DEV_NEED_LEVELS = 1u << 1,     // frontier history too short; host grows it and reruns
    DEV_SIGMA_OVERFLOW = 1u << 2,  // some sigma >= 2^53
    DEV_ARENA_OVERFLOW = 1u << 3,  // path arena too small; host grows it and reruns
    DEV_BAD_PATH = 1u << 4,        // backtrack found no predecessor (sigma inexact)
    DEV_BAD_STATE = 1u << 5,       // x NaN or outside [0,1]
    DEV_DEGENERATE = 1u << 6,      // some C_v <= 0
    DEV_SIGMA_WIDE = 1u << 7,      // some sigma >= 2^32: 32-bit storage too narrow
    DEV_BAD_INPUT = 1u << 8,       // a column index outside [0, n) (unvalidated input)
};

constexpr double kTwo53 = 9007199254740992.0;

// Storage of the batched sigma counts.  Mode 0: 32-bit integers (exact below
// 2^32), mode 1: 64-bit integers (exact below 2^53, the FP64 range), mode 2:
// FP64.  Sums are always formed in 64-bit integers (modes 0, 1) or FP64.
template <int SM>
struct SigmaMode;
template <>
struct SigmaMode<0> {
    using ST = unsigned int;
    using S = unsigned long long;
    static constexpr unsigned long long limit = 1ull << 32;
    static constexpr uint32_t flag = DEV_SIGMA_WIDE;
};
template <>
struct SigmaMode<1> {
    using ST = unsigned long long;
    using S = unsigned long long;
    static constexpr unsigned long long limit = 1ull << 53;
    static constexpr uint32_t flag = DEV_SIGMA_OVERFLOW;
};
template <>
struct SigmaMode<2> {
    using ST = double;
    using S = double;
    static constexpr unsigned long long limit = 1ull << 53;
    static constexpr uint32_t flag = DEV_SIGMA_OVERFLOW;
};

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon et al., SC'11): ten rounds, multipliers 0xD2511F53 /
// 0xCD9E8D57, key increments 0x9E3779B9 / 0xBB67AE85.
__device__ __forceinline__ void philox4x32_10(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t &c3, uint32_t k0,
                                              uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
}

// Two uniforms in (0,1]: counter (i_lo, i_hi, tag, j), key = seed.
// u = ((w >> 11) + 1) * 2^-53 with w the 64-bit words (out1:out0), (out3:out2).
__device__ __forceinline__ void uniforms2(uint64_t seed, uint64_t i, uint32_t tag, uint32_t j, double &ua,
                                          double &ub) {
    uint32_t c0 = (uint32_t)i, c1 = (uint32_t)(i >> 32), c2 = tag, c3 = j;
    philox4x32_10(c0, c1, c2, c3, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint64_t wa = ((uint64_t)c1 << 32) | c0;
    const uint64_t wb = ((uint64_t)c3 << 32) | c2;
    ua = __dmul_rn((double)((wa >> 11) + 1), 0x1p-53);
    ub = __dmul_rn((double)((wb >> 11) + 1), 0x1p-53);
}

__device__ __forceinline__ double uniform_at(uint64_t seed, uint64_t i, uint32_t tag, uint32_t step) {
    double a, b;
    uniforms2(seed, i, tag, step >> 1, a, b);
    return (step & 1) ? b : a;
}

// ------------------------------------------------------------ timers/atomics

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int64_t ld_relaxed_s64(const int64_t *p) {
    return (int64_t)ld_relaxed_u64((const uint64_t *)p);
}

// ------------------------------------------------------------ grid barrier
// Sense-by-generation barrier for cooperative launches (all blocks are
// co-resident, so it cannot deadlock).  Every wait is bounded: after
// budget_ns the waiting block sets DEV_TIMEOUT and every later barrier
// returns false at once, so a kernel that sees `false` must exit.
struct GridBarrier {
    uint32_t count;
    uint32_t gen;
};

__device__ __forceinline__ bool grid_sync(GridBarrier *bar, uint32_t *status, uint64_t budget_ns) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const uint32_t my_gen = ld_acquire_u32(&bar->gen);
        __threadfence();
        const uint32_t prev = atomicAdd(&bar->count, 1u);
        if (prev == gridDim.x - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            while (ld_acquire_u32(&bar->gen) == my_gen) {
                if (ld_relaxed_u32(status) & DEV_TIMEOUT) {
                    ok = 0;
                    break;
                }
                if (globaltimer_ns() - t0 > budget_ns) {
                    atomicOr(status, DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        if (ld_relaxed_u32(status) & DEV_TIMEOUT) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ------------------------------------------------------------ warp helpers

__device__ __forceinline__ double warp_inclusive_scan(double v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const double o = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v = __dadd_rn(v, o);
    }
    return v;
}

__device__ __forceinline__ uint64_t warp_or64(uint64_t v) {
    const uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)v);
    const uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(v >> 32));
    return ((uint64_t)hi << 32) | lo;
}

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src) {
    return __shfl_sync(0xffffffffu, v, src);
}

}  // namespace percis
