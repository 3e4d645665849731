// percis_bfs_noalloc: the single-source sigma-counting BFS for callers that
// cannot allocate device memory.  Some callers hand all of the device memory
// to their own pool when they start (a serving process that reserves HBM up
// front) or cannot afford cudaMalloc's implicit device synchronisation on a
// latency-critical path; they cannot create a percis_ctx, whose buffers come
// from cudaMalloc.  This entry point needs nothing but the caller's buffers
// and one fixed scratch array compiled into the library.
//
// The scratch array (frontier queues and a control block) is a file-scope
// __device__ array, so every GPU that loads the library holds it until the
// process exits.  Host code cannot use the array's name as a device address:
// the first call on each device looks the address up with
// cudaGetSymbolAddress while that device is current, and passes it to the
// kernel.  All calls share the array and it keeps the last call's contents, so
// each call clears what must start at zero; calls that overlap on the GPU (on
// different streams) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace percis {

namespace {

constexpr int64_t kNoAllocMaxN = PERCIS_NOALLOC_MAX_N;
constexpr size_t kCtlBytes = 256;
constexpr size_t kScratchBytes = kCtlBytes + 2 * sizeof(int32_t) * (size_t)kNoAllocMaxN;
constexpr int kBlock = 256;
constexpr double kDefaultBudgetS = 10.0;

struct NoAllocCtl {
    uint32_t bar_count, bar_gen;  // GridBarrier
    uint32_t status;
    int32_t qsize[2];
    int32_t found;
};
static_assert(sizeof(NoAllocCtl) <= kCtlBytes, "control block");

// 8 MiB + 256 B for PERCIS_NOALLOC_MAX_N = 2^20: two frontier queues of n int32.
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

__global__ void __launch_bounds__(kBlock) k_bfs_noalloc(int64_t n, const int64_t *rp, const int32_t *col,
                                                        const int64_t *irp, const int32_t *icol, int32_t s,
                                                        int32_t t, int32_t *dist, double *sigma,
                                                        unsigned char *scratch, uint64_t budget_ns) {
    NoAllocCtl *ctl = reinterpret_cast<NoAllocCtl *>(scratch);
    int32_t *qa = reinterpret_cast<int32_t *>(scratch + kCtlBytes);
    int32_t *qb = qa + kNoAllocMaxN;
    GridBarrier *bar = reinterpret_cast<GridBarrier *>(ctl);
    uint32_t *status = &ctl->status;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = tid; v < n; v += nthreads) {
        dist[v] = -1;
        sigma[v] = 0.0;
    }
    if (!grid_sync(bar, status, budget_ns)) return;
    if (tid == 0) {
        dist[s] = 0;
        sigma[s] = 1.0;
        qa[0] = s;
        ctl->qsize[0] = 1;
        ctl->qsize[1] = 0;
        ctl->found = 0;
    }
    if (!grid_sync(bar, status, budget_ns)) return;
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = tid >> 5, nwarps = nthreads >> 5;
    int32_t *cur = qa, *nxt = qb;
    // a target equal to the source is settled at level 0: nothing to expand
    for (int L = 0; t < 0 || t != s; ++L) {
        const int nq = (int)ld_relaxed_u32((const uint32_t *)&ctl->qsize[L & 1]);
        // expand level L: claim unreached out-neighbours for level L+1
        for (int64_t k = gwarp; k < nq; k += nwarps) {
            const int32_t u = __ldcg(&cur[k]);
            const int64_t e0 = rp[u], e1 = rp[u + 1];
            for (int64_t base = e0; base < e1; base += 32) {
                const int64_t e = base + lane;
                bool mine = false;
                int32_t v = 0;
                if (e < e1) {
                    v = col[e];
                    if ((uint64_t)(int64_t)v >= (uint64_t)n) {
                        atomicOr(status, DEV_BAD_INPUT);  // skip the entry instead of faulting
                    } else if (__ldcg(&dist[v]) < 0) {
                        mine = atomicCAS(&dist[v], -1, L + 1) == -1;
                    }
                }
                const unsigned m = __ballot_sync(0xffffffffu, mine);
                if (m) {
                    const int leader = __ffs(m) - 1;
                    int pos = 0;
                    if (lane == leader) pos = atomicAdd(&ctl->qsize[(L + 1) & 1], __popc(m));
                    pos = __shfl_sync(0xffffffffu, pos, leader);
                    if (mine) nxt[pos + __popc(m & ((1u << lane) - 1u))] = v;
                }
            }
        }
        if (!grid_sync(bar, status, budget_ns)) return;
        const int nn = (int)ld_relaxed_u32((const uint32_t *)&ctl->qsize[(L + 1) & 1]);
        if (tid == 0) ctl->qsize[L & 1] = 0;
        // sigma of the new level: sum over in-neighbours at level L
        for (int64_t k = gwarp; k < nn; k += nwarps) {
            const int32_t w = __ldcg(&nxt[k]);
            double acc = 0.0;
            for (int64_t e = irp[w] + lane; e < irp[w + 1]; e += 32) {
                const int32_t u = icol[e];
                if ((uint64_t)(int64_t)u >= (uint64_t)n) atomicOr(status, DEV_BAD_INPUT);
                else if (__ldcg(&dist[u]) == L) acc += __ldcg(&sigma[u]);
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (lane == 0) {
                sigma[w] = acc;
                if (acc >= kTwo53) atomicOr(status, DEV_SIGMA_OVERFLOW);
                if (w == t) atomicExch(&ctl->found, 1);
            }
        }
        if (!grid_sync(bar, status, budget_ns)) return;
        if (nn == 0) break;
        // only values fixed until every block passes the next barrier decide the exit
        if (t >= 0 && ld_relaxed_u32((const uint32_t *)&ctl->found)) break;
        int32_t *tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
}

// Per-device set-up, done once with the device current.
struct DeviceSlot {
    unsigned char *scratch = nullptr;
    int grid = 0;
};
constexpr int kMaxDevices = 64;
DeviceSlot g_slots[kMaxDevices];
std::mutex g_slot_mutex;

percis_status device_slot(int dev, DeviceSlot **out) {
    if (dev < 0 || dev >= kMaxDevices) return PERCIS_E_INVALID;
    std::lock_guard<std::mutex> lock(g_slot_mutex);
    DeviceSlot &sl = g_slots[dev];
    if (!sl.scratch) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return PERCIS_E_CUDA;
        }
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bfs_noalloc, kBlock, 0) != cudaSuccess) {
            cudaGetLastError();
            return PERCIS_E_CUDA;
        }
        sl.grid = std::max(1, per_sm) * sms;
        sl.scratch = static_cast<unsigned char *>(p);
    }
    *out = &sl;
    return PERCIS_OK;
}

}  // namespace
}  // namespace percis

using namespace percis;

extern "C" percis_status percis_bfs_noalloc(int64_t n, const int64_t *row_ptr, const int32_t *col,
                                            const int64_t *in_row_ptr, const int32_t *in_col, int32_t source,
                                            int32_t target, int32_t *dist, double *sigma, void *stream,
                                            double timeout_s, int32_t *sigma_overflow) {
    if (sigma_overflow) *sigma_overflow = 0;
    if (n < 1 || n > kNoAllocMaxN || !row_ptr || !col || !dist || !sigma) return PERCIS_E_INVALID;
    if (source < 0 || source >= n || target >= n) return PERCIS_E_INVALID;
    if ((in_row_ptr == nullptr) != (in_col == nullptr)) return PERCIS_E_INVALID;
    if (!(timeout_s > 0.0)) timeout_s = kDefaultBudgetS;
    uint64_t budget_ns = timeout_s < 1e9 ? (uint64_t)(timeout_s * 1e9) : ~0ull;
    if (budget_ns == 0) budget_ns = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the memset, launch, copy and synchronisation below cannot be captured
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return PERCIS_E_CUDA;
    }
    if (cap != cudaStreamCaptureStatusNone) return PERCIS_E_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PERCIS_E_CUDA;
    }
    DeviceSlot *sl = nullptr;
    const percis_status st = device_slot(dev, &sl);
    if (st != PERCIS_OK) return st;
    const int64_t *irp = in_row_ptr ? in_row_ptr : row_ptr;
    const int32_t *icol = in_col ? in_col : col;
    int32_t tgt = target < 0 ? -1 : target;
    unsigned char *scratch = sl->scratch;
    // barrier counters, queue sizes and status must start at zero
    if (cudaMemsetAsync(scratch, 0, kCtlBytes, s) != cudaSuccess) {
        cudaGetLastError();
        return PERCIS_E_CUDA;
    }
    void *args[] = {&n, &row_ptr, &col, &irp, &icol, &source, &tgt, &dist, &sigma, &scratch, &budget_ns};
    if (cudaLaunchCooperativeKernel((const void *)k_bfs_noalloc, dim3(sl->grid), dim3(kBlock), args, 0, s) !=
        cudaSuccess) {
        cudaGetLastError();
        return PERCIS_E_CUDA;
    }
    uint32_t status = 0;
    if (cudaMemcpyAsync(&status, scratch + offsetof(NoAllocCtl, status), sizeof(status), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return PERCIS_E_CUDA;
    }
    if (sigma_overflow) *sigma_overflow = (status & DEV_SIGMA_OVERFLOW) ? 1 : 0;
    if (status & DEV_TIMEOUT) return PERCIS_E_TIMEOUT;
    if (status & DEV_BAD_INPUT) return PERCIS_E_INVALID;
    return PERCIS_OK;
}
