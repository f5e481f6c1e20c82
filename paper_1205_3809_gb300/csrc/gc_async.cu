// Asynchronous form of Algorithm 2 ("Iterative", Sec. 3.2) as the paper runs
// it on shared-memory machines: in Phase 1 every worklist vertex takes the
// smallest color no neighbour holds *right now* -- it reads the one shared
// color array while other threads write it, so it sees some of this round's
// tentative colors (Gauss-Seidel) -- and Phase 2 sends the later of two
// equally colored neighbours back to the worklist.  The result depends on
// the schedule; it is checked for validity only (a proper coloring, colors
// at most degree + 1), and is the comparison point for the synchronous form
// (fewer rounds and, usually, fewer colors, at the price of determinism).
//
// One warp per worklist vertex in both phases; the host reads the worklist
// size after each round (two launches per round).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>

#include "gc.h"

namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// w precedes v in the tie-break order (keys, then index).
__device__ __forceinline__ bool precedes(const uint32_t* __restrict__ prio, int32_t w, int32_t v) {
    if (prio) {
        const uint32_t pw = __ldg(prio + w), pv = __ldg(prio + v);
        if (pw != pv) return pw < pv;
    }
    return w < v;
}

// Live color of w: an L2-coherent load (no L1 copy), so a color another SM
// has just written can be seen.
__device__ __forceinline__ int32_t live(const int32_t* color, int32_t w) { return __ldcg(color + w); }

// Phase 1 for worklist U: the smallest color > 0 that no neighbour holds at
// the time it is read, searched in windows of 256 colors.
__global__ void async_phase1_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                    const int32_t* __restrict__ U, const unsigned* __restrict__ nU,
                                    int32_t* color) {
    const unsigned lane = lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n_u = (int64_t)*nU;
    for (int64_t t = gw; t < n_u; t += W) {
        const int32_t v = __ldg(U + t);
        const int32_t b = __ldg(rowptr + v), e = __ldg(rowptr + v + 1);
        int32_t c = 0;
        for (int32_t base = 0; c == 0; base += 256) {
            uint32_t m[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int32_t i = b + (int32_t)lane; i < e; i += 32) {
                const int32_t x = live(color, __ldg(colidx + i)) - 1 - base;
                const uint32_t bit = (x >= 0 && x < 256) ? 1u << (x & 31) : 0u;
#pragma unroll
                for (int q = 0; q < 8; ++q) m[q] |= (x >> 5) == q ? bit : 0u;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) m[q] = __reduce_or_sync(kFull, m[q]);
#pragma unroll
            for (int q = 7; q >= 0; --q)
                if (m[q] != kFull) c = base + q * 32 + __ffs(~m[q]);
        }
        if (lane == 0) color[v] = c;
    }
}

// Phase 2 for worklist U: v goes to R if a preceding neighbour holds its color.
__global__ void async_phase2_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                    const uint32_t* __restrict__ prio, const int32_t* __restrict__ U,
                                    const unsigned* __restrict__ nU, const int32_t* color, int32_t* R,
                                    unsigned* nR) {
    const unsigned lane = lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t n_u = (int64_t)*nU;
    for (int64_t t = gw; t < n_u; t += W) {
        const int32_t v = __ldg(U + t);
        const int32_t b = __ldg(rowptr + v), e = __ldg(rowptr + v + 1);
        const int32_t cv = __ldcg(color + v);
        bool hit = false;
        for (int32_t i = b + (int32_t)lane; i < e && !hit; i += 32) {
            const int32_t w = __ldg(colidx + i);
            hit = __ldcg(color + w) == cv && precedes(prio, w, v);
        }
        if (__any_sync(kFull, hit) && lane == 0) R[atomicAdd(nR, 1u)] = v;
    }
}

__global__ void iota_kernel(int32_t* U, int32_t n, int32_t* color) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        U[i] = (int32_t)i;
        color[i] = 0;
    }
}

__global__ void max_kernel(const int32_t* __restrict__ color, int32_t n, int32_t* out) {
    int m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, __ldcg(color + i));
    m = __reduce_max_sync(kFull, m);
    if (lane_id() == 0 && m) atomicMax(out, m);
}

struct AsyncCache {
    void* ws = nullptr;
    size_t bytes = 0;
    int sms = 0;
};
std::mutex g_async_mu;
std::map<int, AsyncCache> g_async;

}  // namespace

extern "C" int gc_color_async(const int32_t* rowptr, const int32_t* colidx, int32_t n, const uint32_t* priority,
                              int32_t* colors_out, int32_t* ncolors, int32_t* rounds, int32_t max_rounds,
                              void* stream) {
    if (n < 0 || !ncolors || !rounds || (n > 0 && (!rowptr || !colors_out))) return GC_ERR_INVALID;
    *ncolors = 0;
    *rounds = 0;
    if (n == 0) return GC_OK;
    if (!colidx) {  // allowed only for a graph without edges
        int32_t nnz = -1;
        if (cudaMemcpyAsync(&nnz, rowptr + n, 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess ||
            cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
            return GC_ERR_CUDA;
        if (nnz != 0) return GC_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lock(g_async_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GC_ERR_CUDA;
    AsyncCache& ac = g_async[dev];
    if (!ac.sms && cudaDeviceGetAttribute(&ac.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return GC_ERR_CUDA;
    const size_t need = 2 * (size_t)n * 4 + 256;
    if (ac.bytes < need) {
        if (ac.ws) {
            cudaDeviceSynchronize();
            cudaFree(ac.ws);
            ac.ws = nullptr;
            ac.bytes = 0;
        }
        if (cudaMalloc(&ac.ws, need) != cudaSuccess) {
            (void)cudaGetLastError();
            return GC_ERR_OOM;
        }
        ac.bytes = need;
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* cnt = (unsigned*)ac.ws;               // cnt[0], cnt[1]: worklist sizes; cnt[2]: max color
    int32_t* L[2] = {(int32_t*)((char*)ac.ws + 256), (int32_t*)((char*)ac.ws + 256) + n};
    const int grid = ac.sms * 8;
    if (cudaMemsetAsync(cnt, 0, 16, s) != cudaSuccess) return GC_ERR_CUDA;
    iota_kernel<<<grid, 256, 0, s>>>(L[0], n, colors_out);
    unsigned size = (unsigned)n;
    if (cudaMemcpyAsync(cnt, &size, 4, cudaMemcpyHostToDevice, s) != cudaSuccess) return GC_ERR_CUDA;
    const int32_t limit = max_rounds > 0 ? max_rounds : n;
    int32_t r = 0;
    while (size > 0) {
        if (r >= limit) {
            *rounds = r;
            return GC_ERR_MAX_ROUNDS;
        }
        const int a = r & 1;
        async_phase1_kernel<<<grid, 256, 0, s>>>(rowptr, colidx, L[a], cnt + a, colors_out);
        if (cudaMemsetAsync(cnt + (a ^ 1), 0, 4, s) != cudaSuccess) return GC_ERR_CUDA;
        async_phase2_kernel<<<grid, 256, 0, s>>>(rowptr, colidx, priority, L[a], cnt + a, colors_out, L[a ^ 1],
                                                 cnt + (a ^ 1));
        if (cudaGetLastError() != cudaSuccess) return GC_ERR_CUDA;
        if (cudaMemcpyAsync(&size, cnt + (a ^ 1), 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return GC_ERR_CUDA;
        ++r;
    }
    max_kernel<<<grid, 256, 0, s>>>(colors_out, n, (int32_t*)(cnt + 2));
    int32_t mc = 0;
    if (cudaMemcpyAsync(&mc, cnt + 2, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GC_ERR_CUDA;
    *ncolors = mc;
    *rounds = r;
    return GC_OK;
}
