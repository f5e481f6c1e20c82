// Device code of the batched path: many independent graphs colored in one
// persistent launch.
//
// The graphs arrive as per-graph CSRs laid end to end: graph g has
// n_g = voff[g+1] - voff[g] vertices and nnz_g = eoff[g+1] - eoff[g]
// adjacency entries; its rowptr (n_g + 1 entries, starting at 0) sits at
// rowptr_cat[voff[g] + g ..], its colidx (ids local to the graph) at
// colidx_cat[eoff[g] ..].  The batch is colored as the disjoint union: vertex
// i of graph g becomes global vertex voff[g] + i, which keeps the order of
// indices inside every graph, so synchronous rounds give each graph exactly
// the coloring it would get alone (a vertex's rounds see only its own
// connected component).  The union's rowptr is built once when the batch is
// planned; its colidx is rebuilt by every run from the caller's colidx_cat.
#pragma once

#include "gc_device.cuh"

namespace gc {

struct BatchFlags {
    int bad_rowptr;   // a graph's rowptr does not start at 0, end at nnz_g, or stay in [0, nnz_g]
    int bad_colidx;   // a local id outside [0, n_g)
    int pad[30];
};

// The graph holding position x of a nondecreasing offset array off[0..G]
// (off[0] = 0, x < off[G]): the last g with off[g] <= x, which skips empty
// graphs.
__device__ __forceinline__ int32_t graph_of(const int64_t* __restrict__ off, int32_t G, int64_t x) {
    int32_t lo = 0, hi = G - 1;
    while (lo < hi) {
        const int32_t mid = (lo + hi + 1) >> 1;
        if (__ldg(off + mid) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Union rowptr: rowptr_g[v] = eoff[g] + (graph g's rowptr entry of v), and
// rowptr_g[N] = eoff[G].  Checks that every graph's rowptr starts at 0 and
// ends at nnz_g; an entry outside [0, nnz_g] is flagged and clamped.
__global__ void batch_rowptr_kernel(const int32_t* __restrict__ rowptr_cat, const int64_t* __restrict__ voff,
                                    const int64_t* __restrict__ eoff, int32_t G, int64_t N,
                                    int32_t* __restrict__ rowptr_g, BatchFlags* fl) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    int bad = 0;
    for (int64_t v = tid; v < N; v += T) {
        const int32_t g = graph_of(voff, G, v);
        const int64_t nnz_g = __ldg(eoff + g + 1) - __ldg(eoff + g);
        int64_t local = __ldg(rowptr_cat + v + g);
        if (local < 0 || local > nnz_g) {
            bad = 1;
            local = local < 0 ? 0 : nnz_g;
        }
        rowptr_g[v] = (int32_t)(__ldg(eoff + g) + local);
    }
    for (int64_t g = tid; g < G; g += T) {
        const int64_t first = __ldg(rowptr_cat + __ldg(voff + g) + g);
        const int64_t last = __ldg(rowptr_cat + __ldg(voff + g + 1) + g);
        if (first != 0 || last != __ldg(eoff + g + 1) - __ldg(eoff + g)) bad = 1;
    }
    if (tid == 0) rowptr_g[N] = (int32_t)__ldg(eoff + G);
    if (__any_sync(kFull, bad) && lane_id() == 0) atomicExch(&fl->bad_rowptr, 1);
}

// Union colidx: colidx_g[e] = voff[g] + colidx_cat[e] for the graph g that
// owns entry e.  A warp takes a span of 512 consecutive entries (coalesced
// loads and stores, 16 in flight per lane); each lane walks its entries in
// increasing order, so its graph only moves forward.  A local id outside
// [0, n_g) is flagged and replaced by 0, so every id stays inside the union.
constexpr int kRebaseSpan = 512;

__global__ void __launch_bounds__(256) batch_colidx_kernel(const int32_t* __restrict__ colidx_cat,
                                                           const int64_t* __restrict__ voff,
                                                           const int64_t* __restrict__ eoff, int32_t G,
                                                           int64_t NNZ, int32_t* __restrict__ colidx_g,
                                                           BatchFlags* fl) {
    const unsigned lane = lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t spans = (NNZ + kRebaseSpan - 1) / kRebaseSpan;
    int bad = 0;
    for (int64_t sp = gw; sp < spans; sp += W) {
        const int64_t s0 = sp * kRebaseSpan;
        int32_t g = graph_of(eoff, G, s0);
        int64_t gend = __ldg(eoff + g + 1);
        int32_t x[kRebaseSpan / 32];
#pragma unroll
        for (int i = 0; i < kRebaseSpan / 32; ++i) {
            const int64_t e = s0 + i * 32 + lane;
            x[i] = e < NNZ ? __ldg(colidx_cat + e) : 0;
        }
#pragma unroll
        for (int i = 0; i < kRebaseSpan / 32; ++i) {
            const int64_t e = s0 + i * 32 + lane;
            if (e < NNZ) {
                while (e >= gend) {
                    ++g;
                    gend = __ldg(eoff + g + 1);
                }
                const int64_t vb = __ldg(voff + g), ng = __ldg(voff + g + 1) - vb;
                int32_t local = x[i];
                if (local < 0 || (int64_t)local >= ng) {
                    bad = 1;
                    local = 0;
                }
                colidx_g[e] = (int32_t)(vb + local);
            }
        }
    }
    if (__any_sync(kFull, bad) && lane == 0) atomicExch(&fl->bad_colidx, 1);
}

// Per-graph results: ncolors[g] = max color, rounds[g] = max settle round
// over graph g's vertices (both zeroed beforehand, so an empty graph keeps
// 0).  The union's vertices are split into equal chunks, one per warp, so a
// large graph does not serialise on one warp: a chunk inside one graph is
// reduced by the warp and written with one atomicMax per result; a chunk
// that crosses graphs lets each lane fold its own run of vertices per graph.
constexpr int kReduceChunk = 4096;

__global__ void batch_reduce_kernel(const int32_t* __restrict__ colors, const int32_t* __restrict__ settle,
                                    const int64_t* __restrict__ voff, int32_t G, int64_t N,
                                    int32_t* __restrict__ ncolors, int32_t* __restrict__ rounds) {
    const unsigned lane = lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t chunks = (N + kReduceChunk - 1) / kReduceChunk;
    for (int64_t ch = gw; ch < chunks; ch += W) {
        const int64_t v0 = ch * kReduceChunk, v1 = min(N, v0 + kReduceChunk);
        int32_t g = graph_of(voff, G, v0);
        int64_t gend = __ldg(voff + g + 1);
        if (gend >= v1) {
            int mc = 0, mr = 0;
            for (int64_t v = v0 + lane; v < v1; v += 32) {
                mc = max(mc, __ldcg(colors + v));
                mr = max(mr, __ldcg(settle + v));
            }
            mc = __reduce_max_sync(kFull, mc);
            mr = __reduce_max_sync(kFull, mr);
            if (lane == 0) {
                atomicMax(ncolors + g, mc);
                atomicMax(rounds + g, mr);
            }
        } else {
            int mc = 0, mr = 0;
            for (int64_t v = v0 + lane; v < v1; v += 32) {
                if (v >= gend) {
                    if (mc | mr) {
                        atomicMax(ncolors + g, mc);
                        atomicMax(rounds + g, mr);
                    }
                    mc = mr = 0;
                    while (v >= gend) {
                        ++g;
                        gend = __ldg(voff + g + 1);
                    }
                }
                mc = max(mc, __ldcg(colors + v));
                mr = max(mr, __ldcg(settle + v));
            }
            if (mc | mr) {
                atomicMax(ncolors + g, mc);
                atomicMax(rounds + g, mr);
            }
        }
    }
}

}  // namespace gc
