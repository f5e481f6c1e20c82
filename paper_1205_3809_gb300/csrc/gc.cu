// Host driver and C ABI of libgc.so (declarations and contracts in gc.h).
//
// One call of gc_color_ex:
//   1. stats_kernel scans rowptr: max degree, vertices per degree bin, shape
//      checks; one device-to-host copy decides the color width (16-bit color
//      state when every first-fit color fits, i.e. max degree + 1 <= 65535)
//      and sizes the workspace;
//   2. pass1_kernel (rows of up to 256 entries) + pass1_long_kernel (longer
//      rows): round 1 (closed form, all colors 1), its conflict test, and
//      round 2's colors (all 2);
//   3. rounds_persistent_kernel: every later round in one cooperative launch
//      (or, with loop_mode = 1, one round_kernel launch per round; with
//      loop_mode = 2, graph_round_kernel in a CUDA graph's conditional loop);
//   4. one device-to-host copy of the round state and telemetry.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "gc.h"
#include "gc_batch.cuh"
#include "gc_device.cuh"
#include "gc_local.cuh"

namespace {

using gc::Params;
using gc::RoundState;
using gc::Stats;

std::mutex g_mu;
int g_last_cuda_error = 0;
int64_t g_last_launches = 0;

// Record of the last successful coloring call (for the telemetry queries).
struct LastCall {
    int valid = 0;
    int device = -1;
    int32_t rounds = 0;
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t cap = 0;
    const int32_t* d_sizes = nullptr;          // device, workspace
    const unsigned long long* d_vol = nullptr; // device, workspace
    const unsigned long long* d_ns = nullptr;  // device, workspace (persistent launch with telemetry)
    int timed = 0;
    float ms[4] = {0, 0, 0, 0};
};
LastCall g_last;

struct DeviceCache {
    void* ws = nullptr;        // coloring workspace
    size_t ws_bytes = 0;
    void* in = nullptr;        // device copies of host inputs (gc_color_host)
    size_t in_bytes = 0;
    void* host = nullptr;      // pinned host staging for results
    size_t host_bytes = 0;
    int sms = 0;
    int coop = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t copy = nullptr;                 // host inputs: colidx copies in chunks
    cudaEvent_t chunk_ev[16] = {};               // one per chunk copied
    cudaEvent_t start_ev = nullptr;              // orders the copies after the caller's stream
};

// Host inputs of gc_color_host: colidx goes to the device in chunks of whole
// 32-vertex tasks on a copy stream, and round 1 runs on each chunk as soon as
// it has arrived, so the copy overlaps the setup scan and round 1.
constexpr int kMaxChunks = 16;
struct HostInput {
    const int32_t* h_colidx;
    int32_t* d_colidx;
    int nchunks;
    int32_t vb[kMaxChunks + 1];                  // chunk c covers vertices [vb[c], vb[c+1])
    int64_t eb[kMaxChunks + 1];                  // and adjacency entries [eb[c], eb[c+1])
};

std::map<int, DeviceCache> g_cache;

#define GC_CUDA(call)                                       \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) {                            \
            g_last_cuda_error = (int)e_;                    \
            (void)cudaGetLastError();                       \
            return e_ == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA; \
        }                                                   \
    } while (0)

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// An NVTX range over a host-side scope (entry points, setup, rounds), for
// profilers that filter or group by range; a no-op without one attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Queue the chunk copies of a host colidx on the copy stream, after the work
// already queued on s; chunk c's event fires when it has arrived.
int issue_host_chunks(DeviceCache& dc, const HostInput& hin, cudaStream_t s) {
    if (!dc.copy) GC_CUDA(cudaStreamCreateWithFlags(&dc.copy, cudaStreamNonBlocking));
    if (!dc.start_ev) GC_CUDA(cudaEventCreateWithFlags(&dc.start_ev, cudaEventDisableTiming));
    for (int c = 0; c < hin.nchunks; ++c)
        if (!dc.chunk_ev[c]) GC_CUDA(cudaEventCreateWithFlags(&dc.chunk_ev[c], cudaEventDisableTiming));
    GC_CUDA(cudaEventRecord(dc.start_ev, s));
    GC_CUDA(cudaStreamWaitEvent(dc.copy, dc.start_ev, 0));
    for (int c = 0; c < hin.nchunks; ++c) {
        const int64_t e0 = hin.eb[c], e1 = hin.eb[c + 1];
        if (e1 > e0)
            GC_CUDA(cudaMemcpyAsync(hin.d_colidx + e0, hin.h_colidx + e0, (size_t)(e1 - e0) * sizeof(int32_t),
                                    cudaMemcpyHostToDevice, dc.copy));
        GC_CUDA(cudaEventRecord(dc.chunk_ev[c], dc.copy));
    }
    return GC_OK;
}

int device_cache(DeviceCache** out) {
    int dev = 0;
    GC_CUDA(cudaGetDevice(&dev));
    DeviceCache& c = g_cache[dev];
    if (c.sms == 0) {
        GC_CUDA(cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, dev));
        GC_CUDA(cudaDeviceGetAttribute(&c.coop, cudaDevAttrCooperativeLaunch, dev));
    }
    *out = &c;
    return GC_OK;
}

int ensure_device(void** p, size_t* have, size_t need) {
    if (*have >= need && *p) return GC_OK;
    if (*p) {
        GC_CUDA(cudaDeviceSynchronize());
        GC_CUDA(cudaFree(*p));
        *p = nullptr;
        *have = 0;
    }
    GC_CUDA(cudaMalloc(p, need));
    *have = need;
    return GC_OK;
}

int ensure_host(void** p, size_t* have, size_t need) {
    if (*have >= need && *p) return GC_OK;
    if (*p) {
        GC_CUDA(cudaFreeHost(*p));
        *p = nullptr;
        *have = 0;
    }
    GC_CUDA(cudaMallocHost(p, need));
    *have = need;
    return GC_OK;
}

// A device workspace of `need` bytes, unless the caller's testing limit
// (workspace_limit_mb) forbids growing the one held to that size: then
// GC_ERR_OOM, as if cudaMalloc had refused, and the old workspace stays.
int ensure_device_limited(void** p, size_t* have, size_t need, int32_t limit_mb) {
    if (limit_mb > 0 && need > *have && need > ((size_t)limit_mb << 20)) return GC_ERR_OOM;
    return ensure_device(p, have, need);
}

struct Layout {
    size_t st, stats, rs, rv, rt, x0, x1, act0, act1, stat, hubs, defer;
    size_t S[2], M[2], H[2], Hc[2], O[2];
    size_t total;
};

Layout make_layout(int64_t n, int64_t nnz, size_t elem, const Stats& hs, int64_t round_cap) {
    Layout L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + std::max<size_t>(bytes, 16), 256);
        return o;
    };
    L.st = take(sizeof(RoundState));
    L.stats = take(sizeof(Stats));
    L.rs = take((size_t)round_cap * sizeof(int32_t));
    L.rv = take((size_t)round_cap * sizeof(unsigned long long));
    L.rt = take((size_t)(round_cap + 1) * sizeof(unsigned long long));
    L.x0 = take((size_t)n * elem);
    L.x1 = take((size_t)n * elem);
    L.act0 = take((size_t)nnz * sizeof(int32_t));
    L.act1 = take((size_t)nnz * sizeof(int32_t));
    L.stat = take((size_t)n * 8 * sizeof(uint32_t));
    L.hubs = take((size_t)hs.cap[gc::kBinH] * sizeof(gc::HubRecord));
    L.defer = take((size_t)hs.defer * sizeof(int32_t));
    for (int b = 0; b < 2; ++b) {
        L.S[b] = take((size_t)hs.cap[gc::kBinS] * sizeof(int4));
        L.M[b] = take((size_t)hs.cap[gc::kBinM] * sizeof(int4));
        L.H[b] = take((size_t)hs.cap[gc::kBinH] * sizeof(int4));
        L.Hc[b] = take((size_t)hs.cap[gc::kBinH] * sizeof(int32_t));
        L.O[b] = take((size_t)hs.hub_chunks * sizeof(int32_t));
    }
    L.total = off;
    return L;
}

// Loop mode 2: rounds 2.. as one CUDA graph: a condition kernel, then a while
// node whose body is one round kernel and the condition kernel, so the loop
// runs on the device without a cooperative launch or host round trips.  The
// graph is built for this call's parameters and freed after it has run.
template <typename T, bool P>
int run_rounds_graph(const gc_options& o, DeviceCache& dc, Params<T>& p, cudaStream_t s, int64_t* launches) {
    int per_sm = 0;
    GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gc::graph_round_kernel<T, P>, o.block_threads, 0));
    if (per_sm < 1) return GC_ERR_CUDA;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t exec = nullptr;
    GC_CUDA(cudaGraphCreate(&g, 0));
    int rc = GC_OK;
    auto check = [&](cudaError_t e) {
        if (e != cudaSuccess && rc == GC_OK) {
            g_last_cuda_error = (int)e;
            (void)cudaGetLastError();
            rc = e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA;
        }
        return e == cudaSuccess;
    };
    cudaGraphConditionalHandle handle;
    int before = 1, inside = 0;
    if (check(cudaGraphConditionalHandleCreate(&handle, g, 0, 0))) {
        cudaGraphNodeParams pre = {};
        pre.type = cudaGraphNodeTypeKernel;
        void* pre_args[] = {&p, &before, &handle};
        pre.kernel.func = (void*)gc::graph_cond_kernel<T>;
        pre.kernel.gridDim = dim3(1);
        pre.kernel.blockDim = dim3(1);
        pre.kernel.kernelParams = pre_args;
        cudaGraphNode_t n_pre = nullptr, n_while = nullptr;
        cudaGraphNodeParams wp = {};
        wp.type = cudaGraphNodeTypeConditional;
        wp.conditional.handle = handle;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        if (check(cudaGraphAddNode(&n_pre, g, nullptr, nullptr, 0, &pre)) &&
            check(cudaGraphAddNode(&n_while, g, &n_pre, nullptr, 1, &wp))) {
            cudaGraph_t body = wp.conditional.phGraph_out[0];
            cudaGraphNodeParams rk = {};
            rk.type = cudaGraphNodeTypeKernel;
            void* rk_args[] = {&p};
            rk.kernel.func = (void*)gc::graph_round_kernel<T, P>;
            rk.kernel.gridDim = dim3((unsigned)(per_sm * dc.sms));
            rk.kernel.blockDim = dim3((unsigned)o.block_threads);
            rk.kernel.kernelParams = rk_args;
            cudaGraphNodeParams ck = pre;
            void* ck_args[] = {&p, &inside, &handle};
            ck.kernel.kernelParams = ck_args;
            cudaGraphNode_t n_round = nullptr, n_cond = nullptr;
            if (check(cudaGraphAddNode(&n_round, body, nullptr, nullptr, 0, &rk)) &&
                check(cudaGraphAddNode(&n_cond, body, &n_round, nullptr, 1, &ck)) &&
                check(cudaGraphInstantiate(&exec, g, 0)) && check(cudaGraphLaunch(exec, s)))
                *launches += 1;
        }
    }
    if (exec) {
        check(cudaStreamSynchronize(s));
        cudaGraphExecDestroy(exec);
    }
    cudaGraphDestroy(g);
    return rc;
}

template <typename T, bool P>
int run_rounds_p(const gc_options& o, DeviceCache& dc, Params<T>& p, cudaStream_t s, int64_t* launches,
                 const HostInput* hin) {
    const int threads = o.block_threads;
    {
        // one warp task per 32 vertices, per input chunk when the input is still arriving
        const int nch = hin ? hin->nchunks : 1;
        for (int c = 0; c < nch; ++c) {
            const int32_t v0 = hin ? hin->vb[c] : 0, v1 = hin ? hin->vb[c + 1] : p.n;
            if (hin) GC_CUDA(cudaStreamWaitEvent(s, dc.chunk_ev[c], 0));
            if (v1 <= v0) continue;
            const int64_t want = ((int64_t)v1 - v0 + 255) / 256;
            const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)dc.sms * 8));
            gc::pass1_kernel<T><<<grid, 256, 0, s>>>(p, v0, v1);
            GC_CUDA(cudaGetLastError());
            *launches += 1;
        }
        gc::pass1_long_kernel<T><<<dc.sms * gc::kPass1LongBlocksPerSm, 256, 0, s>>>(p);
        GC_CUDA(cudaGetLastError());
        *launches += 1;
        if (o.telemetry) GC_CUDA(cudaEventRecord(dc.ev[2], s));
    }
    if (o.loop_mode == 2) return run_rounds_graph<T, P>(o, dc, p, s, launches);
    if (o.loop_mode == 0) {
        int per_sm = 0;
        GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, gc::rounds_persistent_kernel<T, P>, threads, 0));
        if (per_sm < 1 || !dc.coop) return GC_ERR_CUDA;
        dim3 grid(per_sm * dc.sms), block(threads);
        void* args[] = {&p};
        GC_CUDA(cudaLaunchCooperativeKernel((const void*)gc::rounds_persistent_kernel<T, P>, grid, block,
                                            args, 0, s));
        *launches += 1;
        return GC_OK;
    }
    // loop_mode 1: the host reads |U_k| after each pass
    size_t have = dc.host_bytes;
    int rc = ensure_host(&dc.host, &have, 4096);
    if (rc != GC_OK) return rc;
    dc.host_bytes = have;
    // pinned slots: a copy of one round's counts read back, then hs[0] size, hs[1]
    // status, hs[2] rounds; every iteration synchronises the stream before a slot
    // is rewritten
    static_assert(sizeof(gc::RoundCounts) + 16 <= 4096, "staging slots");
    gc::RoundCounts* h = (gc::RoundCounts*)dc.host;
    int32_t* hs = (int32_t*)((char*)dc.host + sizeof(gc::RoundCounts));
    RoundState* st = p.st;
    int k = 2;
    for (;; ++k) {
        GC_CUDA(cudaMemcpyAsync(h, &st->rc[k % 3], sizeof(gc::RoundCounts), cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaStreamSynchronize(s));
        const unsigned nS = h->s, nM = h->m, nH = gc::hub_count(h->hc), nHC = gc::hub_chunks(h->hc);
        const unsigned size = nS + nM + nH;
        if (size == 0) break;
        if (k > p.max_rounds) {
            hs[1] = gc::kStatusMaxRounds;
            GC_CUDA(cudaMemcpyAsync(&st->status, &hs[1], sizeof(int), cudaMemcpyHostToDevice, s));
            break;
        }
        if (k - 1 < p.round_cap) {
            hs[0] = (int32_t)size;
            GC_CUDA(cudaMemcpyAsync(p.round_sizes + (k - 1), &hs[0], sizeof(int32_t),
                                    cudaMemcpyHostToDevice, s));
        }
        GC_CUDA(cudaMemsetAsync(&st->rc[(k + 2) % 3], 0, sizeof(gc::RoundCounts), s));
        const int64_t tasks = (int64_t)nHC + (nM + gc::kMedPerTask - 1) / gc::kMedPerTask + (nS + 31) / 32;
        const int64_t warps_per_block = threads / 32;
        const int grid = (int)std::max<int64_t>(
            1, std::min<int64_t>((tasks + warps_per_block - 1) / warps_per_block, (int64_t)dc.sms * 8));
        gc::round_kernel<T, P><<<grid, threads, 0, s>>>(p, k, nS, nM, nHC);
        GC_CUDA(cudaGetLastError());
        *launches += 1;
    }
    hs[2] = k - 1;
    GC_CUDA(cudaMemcpyAsync(&st->rounds, &hs[2], sizeof(int), cudaMemcpyHostToDevice, s));
    GC_CUDA(cudaStreamSynchronize(s));
    return GC_OK;
}

// The round kernels are compiled twice: with a priority array (its order
// kept as a bit in the active lists) and without (index order).
template <typename T>
int run_rounds(const gc_options& o, DeviceCache& dc, Params<T>& p, cudaStream_t s, int64_t* launches,
               const HostInput* hin = nullptr) {
    return p.prio ? run_rounds_p<T, true>(o, dc, p, s, launches, hin)
                  : run_rounds_p<T, false>(o, dc, p, s, launches, hin);
}

int normalise(const gc_options* opt, gc_options* o) {
    std::memset(o, 0, sizeof(*o));
    if (opt) *o = *opt;
    if (o->small_max_degree == 0) o->small_max_degree = gc::kSmallMaxLimit;
    if (o->medium_max_degree == 0) o->medium_max_degree = gc::kMedMaxLimit;
    if (o->block_threads == 0) o->block_threads = 256;
    if (o->tail_volume <= 0) o->tail_volume = -1;
    if (o->narrow_color_limit < 0) return GC_ERR_INVALID;
    if (o->small_max_degree < 1 || o->small_max_degree > gc::kSmallMaxLimit) return GC_ERR_INVALID;
    if (o->medium_max_degree < o->small_max_degree || o->medium_max_degree > gc::kMedMaxLimit)
        return GC_ERR_INVALID;
    if (o->block_threads != 128 && o->block_threads != 256) return GC_ERR_INVALID;
    if (o->loop_mode < 0 || o->loop_mode > 2) return GC_ERR_INVALID;
    if (o->color_bits != 0 && o->color_bits != 16 && o->color_bits != 32) return GC_ERR_INVALID;
    if (o->max_rounds < 0 || o->validate < 0 || o->validate > 1) return GC_ERR_INVALID;
    if (o->telemetry != 0 && o->telemetry != 1) return GC_ERR_INVALID;
    if (o->batch_mode < 0 || o->batch_mode > 2) return GC_ERR_INVALID;
    if (o->local_shared_bytes != 0 && o->local_shared_bytes < 16384) return GC_ERR_INVALID;
    if (o->barrier_poll_limit < 0 || o->workspace_limit_mb < 0) return GC_ERR_INVALID;
    return GC_OK;
}

int validate_locked(const int32_t* rowptr, const int32_t* colidx, int32_t n, cudaStream_t s,
                    DeviceCache& dc, int64_t* launches) {
    // workspace head is reused for the validation record
    int rc = ensure_device(&dc.ws, &dc.ws_bytes, std::max<size_t>(dc.ws_bytes, 4096));
    if (rc != GC_OK) return rc;
    gc::ValidateOut* out = (gc::ValidateOut*)dc.ws;
    Stats* stats = (Stats*)((char*)dc.ws + 1024);
    GC_CUDA(cudaMemsetAsync(dc.ws, 0, 2048, s));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)dc.sms * 8));
    gc::stats_kernel<<<grid, 256, 0, s>>>(rowptr, n, gc::kSmallMaxLimit, gc::kMedMaxLimit, stats);
    GC_CUDA(cudaGetLastError());
    size_t hb = dc.host_bytes;
    rc = ensure_host(&dc.host, &hb, 4096);
    if (rc != GC_OK) return rc;
    dc.host_bytes = hb;
    GC_CUDA(cudaMemcpyAsync(dc.host, stats, sizeof(Stats), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    Stats hs;
    std::memcpy(&hs, dc.host, sizeof(Stats));
    *launches += 1;
    if (hs.bad || hs.nnz < 0) return GC_ERR_BAD_GRAPH;
    if (hs.nnz > 0 && !colidx) return GC_ERR_INVALID;
    const int vgrid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n * 32 + 255) / 256, (int64_t)dc.sms * 16));
    gc::validate_kernel<<<vgrid, 256, 0, s>>>(rowptr, colidx, n, out);
    GC_CUDA(cudaGetLastError());
    *launches += 1;
    GC_CUDA(cudaMemcpyAsync(dc.host, out, sizeof(gc::ValidateOut), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    gc::ValidateOut ho;
    std::memcpy(&ho, dc.host, sizeof(ho));
    if (ho.bad_index || ho.self_loop || ho.sum_fwd != ho.sum_bwd) return GC_ERR_BAD_GRAPH;
    return GC_OK;
}

int color_locked(const int32_t* rowptr, const int32_t* colidx, int32_t n, const uint32_t* priority,
                 int32_t* colors_out, int32_t* ncolors, int32_t* rounds, cudaStream_t s,
                 const gc_options* opt, int32_t* round_sizes, int32_t round_sizes_cap,
                 HostInput* hin = nullptr) {
    gc_options o;
    int rc = normalise(opt, &o);
    if (rc != GC_OK) return rc;
    if (n < 0 || !ncolors || !rounds || (round_sizes && round_sizes_cap < 0)) return GC_ERR_INVALID;
    g_last.valid = 0;
    if (n > 0 && (!rowptr || !colors_out)) return GC_ERR_INVALID;
    int64_t launches = 0;
    if (n == 0) {
        *ncolors = 0;
        *rounds = 0;
        g_last_launches = 0;
        return GC_OK;
    }
    DeviceCache* dcp = nullptr;
    rc = device_cache(&dcp);
    if (rc != GC_OK) return rc;
    DeviceCache& dc = *dcp;
    if (hin) {
        rc = issue_host_chunks(dc, *hin, s);
        if (rc != GC_OK) return rc;
    }
    if (o.validate) {
        if (hin) GC_CUDA(cudaStreamWaitEvent(s, dc.chunk_ev[hin->nchunks - 1], 0));
        rc = validate_locked(rowptr, colidx, n, s, dc, &launches);
        if (rc != GC_OK) return rc;
    }
    const int32_t max_rounds = o.max_rounds > 0 ? o.max_rounds : n;
    // telemetry covers the first min(rounds, max(4096, caller cap), 2^20) rounds
    const int64_t round_cap = std::max<int64_t>(1, std::min<int64_t>(
        max_rounds, std::max<int64_t>(4096, std::min<int64_t>(round_sizes ? round_sizes_cap : 0, 1 << 20))));

    // 1. setup scan (its record lives in a small fixed head of the workspace)
    rc = ensure_device_limited(&dc.ws, &dc.ws_bytes, std::max<size_t>(dc.ws_bytes, 4096), o.workspace_limit_mb);
    if (rc != GC_OK) return rc;
    size_t hb = dc.host_bytes;
    rc = ensure_host(&dc.host, &hb, std::max<size_t>(4096, sizeof(RoundState) + (size_t)round_cap * 4));
    if (rc != GC_OK) return rc;
    dc.host_bytes = hb;
    if (o.telemetry && !dc.ev[0])
        for (int i = 0; i < 4; ++i) GC_CUDA(cudaEventCreate(&dc.ev[i]));
    if (o.telemetry) GC_CUDA(cudaEventRecord(dc.ev[0], s));
    {
        NvtxRange range("gc setup scan");
        Stats* stats = (Stats*)dc.ws;
        GC_CUDA(cudaMemsetAsync(stats, 0, sizeof(Stats), s));
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)dc.sms * 8));
        gc::stats_kernel<<<grid, 256, 0, s>>>(rowptr, n, o.small_max_degree, o.medium_max_degree, stats);
        GC_CUDA(cudaGetLastError());
        launches += 1;
        if (o.telemetry) GC_CUDA(cudaEventRecord(dc.ev[1], s));
        GC_CUDA(cudaMemcpyAsync(dc.host, stats, sizeof(Stats), cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaStreamSynchronize(s));
    }
    Stats hs;
    std::memcpy(&hs, dc.host, sizeof(Stats));
    if (hs.bad || hs.nnz < 0) return GC_ERR_BAD_GRAPH;
    if (hs.nnz > 0 && !colidx) return GC_ERR_INVALID;
    // 16-bit color words (flag + 15-bit color) unless asked for 32; a color
    // that does not fit makes the rounds stop with an overflow status, and the
    // call starts over with 32-bit words.
    int bits = o.color_bits == 32 ? 32 : 16;
    Layout L;
    char* base = nullptr;
    RoundState* st = nullptr;
    for (;;) {
        const size_t elem = bits == 16 ? 2 : 4;
        L = make_layout(n, hs.nnz, elem, hs, round_cap);
        rc = ensure_device_limited(&dc.ws, &dc.ws_bytes, L.total, o.workspace_limit_mb);
        if (rc != GC_OK) return rc;
        base = (char*)dc.ws;
        st = (RoundState*)(base + L.st);
        GC_CUDA(cudaMemsetAsync(st, 0, sizeof(RoundState), s));
        GC_CUDA(cudaMemsetAsync(base + L.rv, 0, (size_t)round_cap * sizeof(unsigned long long), s));
        GC_CUDA(cudaMemsetAsync(base + L.hubs, 0, (size_t)hs.cap[gc::kBinH] * sizeof(gc::HubRecord), s));

        auto fill = [&](auto& p) {
            using PT = std::remove_reference_t<decltype(p)>;
            using T = std::remove_pointer_t<decltype(PT::X0)>;
            p.rowptr = rowptr;
            p.colidx = colidx;
            p.prio = priority;
            p.n = n;
            p.s_max = o.small_max_degree;
            p.m_max = o.medium_max_degree;
            p.max_rounds = max_rounds;
            p.tail_volume = o.tail_volume;
            p.barrier_polls = o.barrier_poll_limit > 0 ? (uint32_t)o.barrier_poll_limit : gc::kBarrierMaxPolls;
            p.color_limit = bits == 16 ? (o.narrow_color_limit > 0 ? (uint32_t)o.narrow_color_limit : 0x8000u)
                                       : 0x80000000u;
            p.X0 = (T*)(base + L.x0);
            p.X1 = (T*)(base + L.x1);
            p.colors_out = colors_out;
            p.settle_round = nullptr;
            p.act0 = (int32_t*)(base + L.act0);
            p.act1 = (int32_t*)(base + L.act1);
            p.stat = (uint32_t*)(base + L.stat);
            p.SA = (int4*)(base + L.S[0]);
            p.MA = (int4*)(base + L.M[0]);
            p.HA = (int4*)(base + L.H[0]);
            p.HcA = (int32_t*)(base + L.Hc[0]);
            p.OA = (int32_t*)(base + L.O[0]);
            p.SB = (int4*)(base + L.S[1]);
            p.MB = (int4*)(base + L.M[1]);
            p.HB = (int4*)(base + L.H[1]);
            p.HcB = (int32_t*)(base + L.Hc[1]);
            p.OB = (int32_t*)(base + L.O[1]);
            p.defer = (int32_t*)(base + L.defer);
            p.hubs = (gc::HubRecord*)(base + L.hubs);
            p.st = st;
            p.round_sizes = (int32_t*)(base + L.rs);
            p.round_vol = (unsigned long long*)(base + L.rv);
            p.round_ns = o.telemetry && o.loop_mode == 0 ? (unsigned long long*)(base + L.rt) : nullptr;
            p.round_cap = (int32_t)round_cap;
        };
        NvtxRange range(bits == 16 ? "gc rounds (16-bit colors)" : "gc rounds (32-bit colors)");
        if (bits == 16) {
            Params<uint16_t> p;
            fill(p);
            rc = run_rounds(o, dc, p, s, &launches, hin);
        } else {
            Params<int32_t> p;
            fill(p);
            rc = run_rounds(o, dc, p, s, &launches, hin);
        }
        if (rc != GC_OK) return rc;
        if (bits == 32) break;
        int status = 0;
        GC_CUDA(cudaMemcpyAsync(dc.host, &st->status, sizeof(int), cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaStreamSynchronize(s));
        std::memcpy(&status, dc.host, sizeof(int));
        if (status != gc::kStatusColorOverflow) break;
        bits = 32;
    }

    // 4. results
    if (o.telemetry) GC_CUDA(cudaEventRecord(dc.ev[3], s));
    GC_CUDA(cudaMemcpyAsync(dc.host, st, sizeof(RoundState), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    RoundState hst;
    std::memcpy(&hst, dc.host, sizeof(RoundState));
    if (hst.status == gc::kStatusTimeout) return GC_ERR_TIMEOUT;
    g_last.valid = 1;
    GC_CUDA(cudaGetDevice(&g_last.device));
    g_last.rounds = hst.rounds;
    g_last.n = n;
    g_last.nnz = hs.nnz;
    g_last.cap = (int32_t)round_cap;
    g_last.d_sizes = (const int32_t*)(base + L.rs);
    g_last.d_vol = (const unsigned long long*)(base + L.rv);
    g_last.d_ns = o.telemetry && o.loop_mode == 0 ? (const unsigned long long*)(base + L.rt) : nullptr;
    g_last.timed = o.telemetry;
    if (o.telemetry) {
        GC_CUDA(cudaEventElapsedTime(&g_last.ms[0], dc.ev[0], dc.ev[1]));
        GC_CUDA(cudaEventElapsedTime(&g_last.ms[1], dc.ev[1], dc.ev[2]));
        GC_CUDA(cudaEventElapsedTime(&g_last.ms[2], dc.ev[2], dc.ev[3]));
        GC_CUDA(cudaEventElapsedTime(&g_last.ms[3], dc.ev[0], dc.ev[3]));
    }
    *rounds = hst.rounds;
    *ncolors = hst.max_color;
    if (round_sizes && round_sizes_cap > 0) {
        const int64_t m = std::min<int64_t>({(int64_t)hst.rounds, (int64_t)round_sizes_cap, round_cap});
        round_sizes[0] = n;
        if (m > 1) {
            GC_CUDA(cudaMemcpyAsync(dc.host, base + L.rs + sizeof(int32_t), (size_t)(m - 1) * sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, s));
            GC_CUDA(cudaStreamSynchronize(s));
            std::memcpy(round_sizes + 1, dc.host, (size_t)(m - 1) * sizeof(int32_t));
        }
    }
    g_last_launches = launches;
    if (hst.status == gc::kStatusMaxRounds) return GC_ERR_MAX_ROUNDS;
    return GC_OK;
}


// ---------------------------------------------------------------------------
// Coloring without any allocation (gc_color_noalloc).
//
// Some callers cannot allocate device memory while they run: a framework
// whose caching allocator has already reserved the device's memory, a
// service with a fixed memory plan that allocates nothing after start-up,
// or a caller that must not let cudaMalloc / cudaFree synchronise the
// device.  For them the workspace lives in this file-scope device array,
// which every GPU that loads the library holds until the process exits.
// The array's name is only a host-side stand-in for the device object, so
// its device address is fetched once per device with cudaGetSymbolAddress
// (that happens on the first call on each device).  Every call shares the
// array and the array keeps the last call's contents: everything that must
// start at zero is cleared on the call's stream, and calls that overlap on
// the GPU (two streams, or two host threads on different streams) would
// race on it.  Host staging uses stack memory, never pinned allocations.
constexpr size_t kNoAllocBytes = 64ull << 20;  // 64 MiB
constexpr int kNoAllocMaxDevices = 64;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocDevice {
    int ready = 0;
    int sms = 0;
    int coop = 0;
    void* scratch = nullptr;  // device address of g_noalloc_scratch on that device
};
NoAllocDevice g_noalloc_dev[kNoAllocMaxDevices];

int noalloc_device(NoAllocDevice** out) {
    int dev = 0;
    GC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return GC_ERR_INVALID;
    NoAllocDevice& d = g_noalloc_dev[dev];
    if (!d.ready) {
        void* ptr = nullptr;
        GC_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        GC_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
        GC_CUDA(cudaDeviceGetAttribute(&d.coop, cudaDevAttrCooperativeLaunch, dev));
        d.scratch = ptr;
        d.ready = 1;
    }
    *out = &d;
    return GC_OK;
}

int color_noalloc_locked(const int32_t* rowptr, const int32_t* colidx, int32_t n,
                         const uint32_t* priority, int32_t* colors_out, int32_t* ncolors,
                         int32_t* rounds, cudaStream_t s) {
    if (n < 0 || !ncolors || !rounds) return GC_ERR_INVALID;
    if (n > 0 && (!rowptr || !colors_out)) return GC_ERR_INVALID;
    // the telemetry queries describe gc_color / gc_color_ex calls only; this call
    // keeps no per-round record, so it leaves them with nothing to report
    g_last.valid = 0;
    g_last_launches = 0;
    if (n == 0) {
        *ncolors = 0;
        *rounds = 0;
        return GC_OK;
    }
    gc_options o;
    int rc = normalise(nullptr, &o);
    if (rc != GC_OK) return rc;
    NoAllocDevice* nd = nullptr;
    rc = noalloc_device(&nd);
    if (rc != GC_OK) return rc;
    char* base = (char*)nd->scratch;

    // setup scan, its record at the start of the scratch array
    Stats hs;
    {
        Stats* stats = (Stats*)base;
        GC_CUDA(cudaMemsetAsync(stats, 0, sizeof(Stats), s));
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)nd->sms * 8));
        gc::stats_kernel<<<grid, 256, 0, s>>>(rowptr, n, o.small_max_degree, o.medium_max_degree, stats);
        GC_CUDA(cudaGetLastError());
        GC_CUDA(cudaMemcpyAsync(&hs, stats, sizeof(Stats), cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaStreamSynchronize(s));
    }
    int64_t launches = 1;
    if (hs.bad || hs.nnz < 0) return GC_ERR_BAD_GRAPH;
    if (hs.nnz > 0 && !colidx) return GC_ERR_INVALID;

    DeviceCache dc;  // only the device attributes run_rounds reads; nothing is allocated
    dc.sms = nd->sms;
    dc.coop = nd->coop;
    const int64_t round_cap = 1;  // no per-round telemetry
    int bits = 16;
    RoundState* st = nullptr;
    for (;;) {
        const size_t elem = bits == 16 ? 2 : 4;
        const Layout L = make_layout(n, hs.nnz, elem, hs, round_cap);
        if (L.total > kNoAllocBytes) return GC_ERR_TOO_LARGE;
        st = (RoundState*)(base + L.st);
        GC_CUDA(cudaMemsetAsync(st, 0, sizeof(RoundState), s));
        GC_CUDA(cudaMemsetAsync(base + L.rv, 0, (size_t)round_cap * sizeof(unsigned long long), s));
        GC_CUDA(cudaMemsetAsync(base + L.hubs, 0, (size_t)hs.cap[gc::kBinH] * sizeof(gc::HubRecord), s));
        auto fill = [&](auto& p) {
            using PT = std::remove_reference_t<decltype(p)>;
            using T = std::remove_pointer_t<decltype(PT::X0)>;
            p.rowptr = rowptr;
            p.colidx = colidx;
            p.prio = priority;
            p.n = n;
            p.s_max = o.small_max_degree;
            p.m_max = o.medium_max_degree;
            p.max_rounds = n;
            p.tail_volume = o.tail_volume;
            p.barrier_polls = gc::kBarrierMaxPolls;
            p.color_limit = bits == 16 ? 0x8000u : 0x80000000u;
            p.X0 = (T*)(base + L.x0);
            p.X1 = (T*)(base + L.x1);
            p.colors_out = colors_out;
            p.settle_round = nullptr;
            p.act0 = (int32_t*)(base + L.act0);
            p.act1 = (int32_t*)(base + L.act1);
            p.stat = (uint32_t*)(base + L.stat);
            p.SA = (int4*)(base + L.S[0]);
            p.MA = (int4*)(base + L.M[0]);
            p.HA = (int4*)(base + L.H[0]);
            p.HcA = (int32_t*)(base + L.Hc[0]);
            p.OA = (int32_t*)(base + L.O[0]);
            p.SB = (int4*)(base + L.S[1]);
            p.MB = (int4*)(base + L.M[1]);
            p.HB = (int4*)(base + L.H[1]);
            p.HcB = (int32_t*)(base + L.Hc[1]);
            p.OB = (int32_t*)(base + L.O[1]);
            p.defer = (int32_t*)(base + L.defer);
            p.hubs = (gc::HubRecord*)(base + L.hubs);
            p.st = st;
            p.round_sizes = (int32_t*)(base + L.rs);
            p.round_vol = (unsigned long long*)(base + L.rv);
            p.round_ns = nullptr;
            p.round_cap = (int32_t)round_cap;
        };
        if (bits == 16) {
            Params<uint16_t> p;
            fill(p);
            rc = run_rounds(o, dc, p, s, &launches);
        } else {
            Params<int32_t> p;
            fill(p);
            rc = run_rounds(o, dc, p, s, &launches);
        }
        if (rc != GC_OK) return rc;
        RoundState hst;
        GC_CUDA(cudaMemcpyAsync(&hst, st, sizeof(RoundState), cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaStreamSynchronize(s));
        if (bits == 16 && hst.status == gc::kStatusColorOverflow) {
            bits = 32;
            continue;
        }
        if (hst.status == gc::kStatusTimeout) return GC_ERR_TIMEOUT;
        if (hst.status == gc::kStatusMaxRounds) return GC_ERR_MAX_ROUNDS;
        *rounds = hst.rounds;
        *ncolors = hst.max_color;
        g_last_launches = launches;
        return GC_OK;
    }
}

// ---------------------------------------------------------------------------
// Batched coloring (gc_batch_*): many independent graphs in one persistent
// launch, as the disjoint union of the graphs (device side: gc_batch.cuh).
//
// gc_batch_create does everything that needs the host: it checks the
// offsets, builds the union rowptr, scans its degrees, picks the color width
// (16-bit state whenever max degree + 1 < 2^15, so a run can never overflow),
// sizes and allocates the plan's own workspace, and optionally validates the
// union graph.  gc_batch_run then only enqueues device work (memsets and
// kernels; no allocation, no host synchronisation), so a stream capture of
// it is a CUDA graph of the whole batch, which gc_batch_launch_graph builds
// once and replays.

template <typename T>
void fill_workspace(Params<T>& p, char* base, const Layout& L, RoundState* st, int64_t round_cap) {
    p.X0 = (T*)(base + L.x0);
    p.X1 = (T*)(base + L.x1);
    p.act0 = (int32_t*)(base + L.act0);
    p.act1 = (int32_t*)(base + L.act1);
    p.stat = (uint32_t*)(base + L.stat);
    p.SA = (int4*)(base + L.S[0]);
    p.MA = (int4*)(base + L.M[0]);
    p.HA = (int4*)(base + L.H[0]);
    p.HcA = (int32_t*)(base + L.Hc[0]);
    p.OA = (int32_t*)(base + L.O[0]);
    p.SB = (int4*)(base + L.S[1]);
    p.MB = (int4*)(base + L.M[1]);
    p.HB = (int4*)(base + L.H[1]);
    p.HcB = (int32_t*)(base + L.Hc[1]);
    p.OB = (int32_t*)(base + L.O[1]);
    p.defer = (int32_t*)(base + L.defer);
    p.hubs = (gc::HubRecord*)(base + L.hubs);
    p.st = st;
    p.round_sizes = (int32_t*)(base + L.rs);
    p.round_vol = (unsigned long long*)(base + L.rv);
    p.round_ns = nullptr;
    p.round_cap = (int32_t)round_cap;
}

}  // namespace

struct gc_batch {
    int device = -1;
    int32_t G = 0;
    int64_t N = 0, NNZ = 0;
    const int32_t* colidx_cat = nullptr;
    const uint32_t* prio = nullptr;
    int32_t* colors_out = nullptr;
    int32_t* ncolors_out = nullptr;
    int32_t* rounds_out = nullptr;
    gc_options o{};
    int bits = 16;
    int sms = 0;
    int per_sm = 0;           // co-resident blocks of the rounds kernel per SM
    gc::Stats hs{};
    Layout L{};
    int64_t round_cap = 1;
    // plan-owned memory: [head: round state .. of the coloring layout][voff][eoff][rowptr_g][colidx_g][settle][flags]
    void* ws = nullptr;
    size_t ws_bytes = 0;
    size_t off_voff = 0, off_eoff = 0, off_rowptr = 0, off_colidx = 0, off_settle = 0, off_flags = 0;
    int64_t launches_per_run = 0;
    // 1: all graphs share the rounds kernel's grid; 2: one thread block per graph
    int mode = 1;
    uint32_t local_smem = 0;  // mode 2: dynamic shared memory per block
    size_t off_queue = 0, off_order = 0, off_lanes = 0, off_ovf = 0, off_wl0 = 0, off_wl1 = 0, off_gcol8 = 0,
           off_gcol32 = 0;
    int32_t* ucolidx = nullptr;  // mode 2: union colidx, allocated when validation or features need it
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// Rebuild the union colidx from the caller's colidx_cat (local ids -> union ids).
// The union colidx buffer: part of the plan in mode 1; in mode 2 (which reads
// the caller's local ids directly) allocated the first time it is needed.
int union_colidx(gc_batch& b, int32_t** out) {
    if (b.mode == 1) {
        *out = (int32_t*)((char*)b.ws + b.off_colidx);
        return GC_OK;
    }
    if (!b.ucolidx) {
        const cudaError_t e = cudaMalloc(&b.ucolidx, (size_t)std::max<int64_t>(b.NNZ, 1) * 4);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            b.ucolidx = nullptr;
            return e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA;
        }
    }
    *out = b.ucolidx;
    return GC_OK;
}

int batch_rebase(gc_batch& b, cudaStream_t s, int64_t* launches) {
    char* base = (char*)b.ws;
    gc::BatchFlags* fl = (gc::BatchFlags*)(base + b.off_flags);
    GC_CUDA(cudaMemsetAsync(&fl->bad_colidx, 0, sizeof(int), s));
    if (b.NNZ == 0) return GC_OK;
    int32_t* colidx_g = nullptr;
    const int rc = union_colidx(b, &colidx_g);
    if (rc != GC_OK) return rc;
    const int64_t spans = (b.NNZ + gc::kRebaseSpan - 1) / gc::kRebaseSpan;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((spans + 7) / 8, (int64_t)b.sms * 8));
    gc::batch_colidx_kernel<<<grid, 256, 0, s>>>(b.colidx_cat, (const int64_t*)(base + b.off_voff),
                                                 (const int64_t*)(base + b.off_eoff), b.G, b.NNZ, colidx_g, fl);
    GC_CUDA(cudaGetLastError());
    ++*launches;
    return GC_OK;
}

// Mode 2: the two launches of the one-block-per-graph kernel (byte colors for
// every graph, then 32-bit colors for the graphs whose colors outgrew a byte).
template <bool P>
int batch_enqueue_local(gc_batch& b, cudaStream_t s) {
    char* base = (char*)b.ws;
    gc::LocalParams lp;
    lp.rowptr_g = (const int32_t*)(base + b.off_rowptr);
    lp.colidx_cat = b.colidx_cat;
    lp.prio = b.prio;
    lp.voff = (const int64_t*)(base + b.off_voff);
    lp.order = (const int32_t*)(base + b.off_order);
    lp.lanes_log2 = (const uint8_t*)(base + b.off_lanes);
    lp.G = b.G;
    lp.max_rounds = b.o.max_rounds;
    lp.smem_bytes = b.local_smem;
    lp.wl0 = (int4*)(base + b.off_wl0);
    lp.wl1 = (int4*)(base + b.off_wl1);
    lp.gcol8 = (uint8_t*)(base + b.off_gcol8);
    lp.gcol32 = (int32_t*)(base + b.off_gcol32);
    lp.colors_out = b.colors_out;
    lp.ncolors_out = b.ncolors_out;
    lp.rounds_out = b.rounds_out;
    lp.ovf_list = (int32_t*)(base + b.off_ovf);
    lp.q = (gc::LocalQueue*)(base + b.off_queue);
    lp.st = (RoundState*)(base + b.L.st);
    lp.fl = (gc::BatchFlags*)(base + b.off_flags);
    lp.round_sizes = (int32_t*)(base + b.L.rs);
    lp.round_vol = (unsigned long long*)(base + b.L.rv);
    lp.round_cap = (int32_t)b.round_cap;
    GC_CUDA(cudaMemsetAsync(lp.st, 0, sizeof(RoundState), s));
    GC_CUDA(cudaMemsetAsync(lp.q, 0, sizeof(gc::LocalQueue), s));
    GC_CUDA(cudaMemsetAsync(&lp.fl->bad_colidx, 0, sizeof(int), s));
    GC_CUDA(cudaMemsetAsync(lp.round_sizes, 0, (size_t)b.round_cap * sizeof(int32_t), s));
    GC_CUDA(cudaMemsetAsync(lp.round_vol, 0, (size_t)b.round_cap * sizeof(unsigned long long), s));
    gc::batch_local_kernel<uint8_t, P><<<b.sms, gc::kLocalThreads, b.local_smem, s>>>(lp, 0);
    GC_CUDA(cudaGetLastError());
    gc::batch_local_kernel<uint32_t, P><<<b.sms, gc::kLocalThreads, b.local_smem, s>>>(lp, 1);
    GC_CUDA(cudaGetLastError());
    b.launches_per_run = 2;
    return GC_OK;
}

// Dynamic shared memory of the mode-2 kernels (the same for all four forms):
// all the block may have, less what they declare statically.
int local_kernels_setup(int device, uint32_t* smem_bytes) {
    int optin = 0;
    GC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    const void* kernels[] = {(const void*)gc::batch_local_kernel<uint8_t, false>,
                             (const void*)gc::batch_local_kernel<uint8_t, true>,
                             (const void*)gc::batch_local_kernel<uint32_t, false>,
                             (const void*)gc::batch_local_kernel<uint32_t, true>};
    size_t stat = 0;
    for (const void* k : kernels) {
        cudaFuncAttributes fa;
        GC_CUDA(cudaFuncGetAttributes(&fa, k));
        stat = std::max(stat, fa.sharedSizeBytes);
    }
    const int dyn = optin - (int)align_up(stat, 1024);
    if (dyn < 4096) return GC_ERR_CUDA;
    for (const void* k : kernels)
        GC_CUDA(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    *smem_bytes = (uint32_t)dyn;
    return GC_OK;
}

template <typename T>
int batch_enqueue_typed(gc_batch& b, cudaStream_t s) {
    char* base = (char*)b.ws;
    const int64_t* voff = (const int64_t*)(base + b.off_voff);
    int32_t* rowptr_g = (int32_t*)(base + b.off_rowptr);
    int32_t* colidx_g = (int32_t*)(base + b.off_colidx);
    int32_t* settle = (int32_t*)(base + b.off_settle);
    RoundState* st = (RoundState*)(base + b.L.st);
    GC_CUDA(cudaMemsetAsync(st, 0, sizeof(RoundState), s));
    GC_CUDA(cudaMemsetAsync(base + b.L.rv, 0, (size_t)b.round_cap * sizeof(unsigned long long), s));
    GC_CUDA(cudaMemsetAsync(base + b.L.hubs, 0, (size_t)b.hs.cap[gc::kBinH] * sizeof(gc::HubRecord), s));
    int64_t launches = 0;
    int rc = batch_rebase(b, s, &launches);
    if (rc != GC_OK) return rc;
    Params<T> p;
    p.rowptr = rowptr_g;
    p.colidx = colidx_g;
    p.prio = b.prio;
    p.n = (int32_t)b.N;
    p.s_max = b.o.small_max_degree;
    p.m_max = b.o.medium_max_degree;
    p.max_rounds = b.o.max_rounds > 0 ? b.o.max_rounds : (int32_t)b.N;
    p.tail_volume = b.o.tail_volume;
    p.barrier_polls = b.o.barrier_poll_limit > 0 ? (uint32_t)b.o.barrier_poll_limit : gc::kBarrierMaxPolls;
    p.color_limit = b.bits == 16 ? 0x8000u : 0x80000000u;
    p.colors_out = b.colors_out;
    p.settle_round = settle;
    fill_workspace(p, base, b.L, st, b.round_cap);
    {
        const int64_t want = (b.N + 255) / 256;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)b.sms * 8));
        gc::pass1_kernel<T><<<grid, 256, 0, s>>>(p, 0, (int32_t)b.N);
        GC_CUDA(cudaGetLastError());
        gc::pass1_long_kernel<T><<<b.sms * gc::kPass1LongBlocksPerSm, 256, 0, s>>>(p);
        GC_CUDA(cudaGetLastError());
        launches += 2;
    }
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(b.per_sm * b.sms));
        cfg.blockDim = dim3((unsigned)b.o.block_threads);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        if (b.prio) {
            GC_CUDA(cudaLaunchKernelEx(&cfg, gc::rounds_persistent_kernel<T, true>, p));
        } else {
            GC_CUDA(cudaLaunchKernelEx(&cfg, gc::rounds_persistent_kernel<T, false>, p));
        }
        ++launches;
    }
    {
        GC_CUDA(cudaMemsetAsync(b.ncolors_out, 0, (size_t)b.G * sizeof(int32_t), s));
        GC_CUDA(cudaMemsetAsync(b.rounds_out, 0, (size_t)b.G * sizeof(int32_t), s));
        const int64_t chunks = (b.N + gc::kReduceChunk - 1) / gc::kReduceChunk;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((chunks + 7) / 8, (int64_t)b.sms * 8));
        gc::batch_reduce_kernel<<<grid, 256, 0, s>>>(b.colors_out, settle, voff, b.G, b.N, b.ncolors_out,
                                                     b.rounds_out);
        GC_CUDA(cudaGetLastError());
        ++launches;
    }
    b.launches_per_run = launches;
    return GC_OK;
}

int batch_enqueue(gc_batch& b, cudaStream_t s) {
    int dev = -1;
    GC_CUDA(cudaGetDevice(&dev));
    if (dev != b.device) return GC_ERR_INVALID;
    if (b.G == 0 || b.N == 0) return GC_OK;
    if (b.mode == 2) return b.prio ? batch_enqueue_local<true>(b, s) : batch_enqueue_local<false>(b, s);
    return b.bits == 16 ? batch_enqueue_typed<uint16_t>(b, s) : batch_enqueue_typed<int32_t>(b, s);
}

void batch_free(gc_batch* b) {
    if (!b) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (b->device >= 0) cudaSetDevice(b->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    if (b->ws || b->ucolidx) cudaDeviceSynchronize();
    if (b->ws) cudaFree(b->ws);
    if (b->ucolidx) cudaFree(b->ucolidx);
    cudaSetDevice(cur);
    (void)cudaGetLastError();
    delete b;
}

int batch_create_locked(const int32_t* rowptr_cat, const int32_t* colidx_cat, const int64_t* voff_h,
                        const int64_t* eoff_h, int32_t G, const uint32_t* prio, int32_t* colors_out,
                        int32_t* ncolors_out, int32_t* rounds_out, const gc_options* opt, cudaStream_t s,
                        gc_batch* b) {
    int rc = normalise(opt, &b->o);
    if (rc != GC_OK) return rc;
    if (b->o.loop_mode != 0) return GC_ERR_INVALID;
    if (G < 0 || !voff_h || !eoff_h) return GC_ERR_INVALID;
    if (voff_h[0] != 0 || eoff_h[0] != 0) return GC_ERR_INVALID;
    for (int32_t g = 0; g < G; ++g)
        if (voff_h[g + 1] < voff_h[g] || eoff_h[g + 1] < eoff_h[g]) return GC_ERR_INVALID;
    const int64_t N = voff_h[G], NNZ = eoff_h[G];
    if (N >= INT32_MAX || NNZ >= INT32_MAX) return GC_ERR_INVALID;
    if (G > 0 && (!rowptr_cat || !ncolors_out || !rounds_out)) return GC_ERR_INVALID;
    if (N > 0 && !colors_out) return GC_ERR_INVALID;
    if (NNZ > 0 && !colidx_cat) return GC_ERR_INVALID;
    GC_CUDA(cudaGetDevice(&b->device));
    GC_CUDA(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device));
    int coop = 0;
    GC_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, b->device));
    if (!coop) return GC_ERR_CUDA;
    b->G = G;
    b->N = N;
    b->NNZ = NNZ;
    b->colidx_cat = colidx_cat;
    b->prio = prio;
    b->colors_out = colors_out;
    b->ncolors_out = ncolors_out;
    b->rounds_out = rounds_out;
    if (G == 0 || N == 0) {
        // nothing to color; per-graph results are all zero
        if (G > 0) {
            GC_CUDA(cudaMemsetAsync(ncolors_out, 0, (size_t)G * 4, s));
            GC_CUDA(cudaMemsetAsync(rounds_out, 0, (size_t)G * 4, s));
            GC_CUDA(cudaStreamSynchronize(s));
        }
        return GC_OK;
    }

    // head: offsets, union rowptr, flags, stats (sized before the degrees are known)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + std::max<size_t>(bytes, 16), 256);
        return o;
    };
    const size_t h_voff = take((size_t)(G + 1) * 8), h_eoff = take((size_t)(G + 1) * 8);
    const size_t h_rowptr = take((size_t)(N + 1) * 4), h_flags = take(sizeof(gc::BatchFlags));
    const size_t h_stats = take(sizeof(Stats));
    const size_t head = off;
    void* tmp = nullptr;
    GC_CUDA(cudaMalloc(&tmp, head));
    auto fail = [&](int code) {
        cudaStreamSynchronize(s);
        cudaFree(tmp);
        return code;
    };
    char* hb = (char*)tmp;
    if (cudaMemcpyAsync(hb + h_voff, voff_h, (size_t)(G + 1) * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(hb + h_eoff, eoff_h, (size_t)(G + 1) * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(hb + h_flags, 0, sizeof(gc::BatchFlags), s) != cudaSuccess ||
        cudaMemsetAsync(hb + h_stats, 0, sizeof(Stats), s) != cudaSuccess)
        return fail(GC_ERR_CUDA);
    {
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, (int64_t)b->sms * 8));
        gc::batch_rowptr_kernel<<<grid, 256, 0, s>>>(rowptr_cat, (const int64_t*)(hb + h_voff),
                                                     (const int64_t*)(hb + h_eoff), G, N,
                                                     (int32_t*)(hb + h_rowptr), (gc::BatchFlags*)(hb + h_flags));
        gc::stats_kernel<<<grid, 256, 0, s>>>((const int32_t*)(hb + h_rowptr), (int32_t)N,
                                              b->o.small_max_degree, b->o.medium_max_degree,
                                              (Stats*)(hb + h_stats));
        if (cudaGetLastError() != cudaSuccess) return fail(GC_ERR_CUDA);
    }
    gc::BatchFlags hf;
    if (cudaMemcpyAsync(&hf, hb + h_flags, sizeof(hf), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&b->hs, hb + h_stats, sizeof(Stats), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(GC_ERR_CUDA);
    if (hf.bad_rowptr || b->hs.bad || b->hs.nnz != NNZ) return fail(GC_ERR_BAD_GRAPH);
    b->bits = b->o.color_bits == 32 || b->hs.max_degree + 1 >= 0x8000 ? 32 : 16;
    const int32_t max_rounds = b->o.max_rounds > 0 ? b->o.max_rounds : (int32_t)N;
    b->round_cap = std::max<int64_t>(1, std::min<int64_t>(max_rounds, 4096));

    // Mode: one block per graph pays off when no graph is a large share of the
    // batch's work (vertices + entries): then the graphs keep every SM busy.
    int64_t max_work = 0;
    for (int32_t g = 0; g < G; ++g)
        max_work = std::max<int64_t>(max_work, (voff_h[g + 1] - voff_h[g]) + (eoff_h[g + 1] - eoff_h[g]));
    b->mode = b->o.batch_mode != 0 ? b->o.batch_mode : (max_work * b->sms <= 2 * (N + NNZ) ? 2 : 1);
    if (b->mode == 2) {
        rc = local_kernels_setup(b->device, &b->local_smem);
        if (rc != GC_OK) return fail(rc);
        b->local_smem = std::min<uint32_t>(
            b->local_smem, b->o.local_shared_bytes > 0 ? (uint32_t)b->o.local_shared_bytes : 164u * 1024u);
        b->bits = 8;
        off = align_up(head, 256);
        b->L = Layout{};
        b->L.st = take(sizeof(RoundState));
        b->L.rs = take((size_t)b->round_cap * sizeof(int32_t));
        b->L.rv = take((size_t)b->round_cap * sizeof(unsigned long long));
        b->off_queue = take(sizeof(gc::LocalQueue));
        b->off_order = take((size_t)G * 4);
        b->off_lanes = take((size_t)G);
        b->off_ovf = take((size_t)G * 4);
        b->off_wl0 = take((size_t)N * sizeof(int4));
        b->off_wl1 = take((size_t)N * sizeof(int4));
        b->off_gcol8 = take((size_t)N);
        b->off_gcol32 = take((size_t)N * 4);
        b->ws_bytes = off;
        b->off_voff = h_voff;
        b->off_eoff = h_eoff;
        b->off_rowptr = h_rowptr;
        b->off_flags = h_flags;
        // queue order: most work first; lanes per vertex from the average degree
        const int64_t tpv = b->o.local_thread_degree == 0 ? 32 : b->o.local_thread_degree;
        std::vector<int32_t> order((size_t)G);
        std::vector<uint8_t> lanes((size_t)G);
        for (int32_t g = 0; g < G; ++g) {
            order[(size_t)g] = g;
            const int64_t ng = voff_h[g + 1] - voff_h[g], eg = eoff_h[g + 1] - eoff_h[g];
            const int64_t avg = ng > 0 ? (eg + ng - 1) / ng : 0;
            int lg = 2;
            while (lg < 5 && (int64_t(1) << lg) * 2 < avg) ++lg;  // about avg/2 lanes, 4..32
            lanes[(size_t)g] = (uint8_t)(avg <= tpv ? 0 : lg);
        }
        std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) {
            return (voff_h[a + 1] - voff_h[a]) + (eoff_h[a + 1] - eoff_h[a]) >
                   (voff_h[c + 1] - voff_h[c]) + (eoff_h[c + 1] - eoff_h[c]);
        });
        void* ws = nullptr;
        if (b->o.workspace_limit_mb > 0 && b->ws_bytes > ((size_t)b->o.workspace_limit_mb << 20))
            return fail(GC_ERR_OOM);
        const cudaError_t e = cudaMalloc(&ws, b->ws_bytes);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA);
        }
        b->ws = ws;
        char* base = (char*)b->ws;
        if (cudaMemcpyAsync(base, tmp, head, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(base + b->off_order, order.data(), (size_t)G * 4, cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemcpyAsync(base + b->off_lanes, lanes.data(), (size_t)G, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return fail(GC_ERR_CUDA);
        fail(GC_OK);  // waits for the copies, frees the head copy
        b->per_sm = 1;
    } else {
    if (b->mode != 1) return fail(GC_ERR_INVALID);
    b->L = make_layout(N, NNZ, b->bits == 16 ? 2 : 4, b->hs, b->round_cap);
    off = align_up(head, 256);
    const size_t lay = take(b->L.total);
    b->off_colidx = take((size_t)NNZ * 4);
    b->off_settle = take((size_t)N * 4);
    b->ws_bytes = off;
    b->off_voff = h_voff;
    b->off_eoff = h_eoff;
    b->off_rowptr = h_rowptr;
    b->off_flags = h_flags;
    {
        void* ws = nullptr;
        if (b->o.workspace_limit_mb > 0 && b->ws_bytes > ((size_t)b->o.workspace_limit_mb << 20))
            return fail(GC_ERR_OOM);
        const cudaError_t e = cudaMalloc(&ws, b->ws_bytes);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? GC_ERR_OOM : GC_ERR_CUDA);
        }
        b->ws = ws;
    }
    if (cudaMemcpyAsync(b->ws, tmp, head, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return fail(GC_ERR_CUDA);
    fail(GC_OK);  // frees the head copy after the stream drains
    // the coloring layout's offsets are relative to its own base
    Layout& L = b->L;
    size_t* fields[] = {&L.st, &L.stats, &L.rs, &L.rv, &L.rt, &L.x0, &L.x1, &L.act0, &L.act1, &L.stat, &L.hubs,
                        &L.defer, &L.S[0], &L.S[1], &L.M[0], &L.M[1], &L.H[0], &L.H[1], &L.Hc[0], &L.Hc[1],
                        &L.O[0], &L.O[1]};
    for (size_t* f : fields) *f += lay;

    int per_sm = 0;
    if (b->bits == 16) {
        GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gc::rounds_persistent_kernel<uint16_t, true>,
                                                              b->o.block_threads, 0));
    } else {
        GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gc::rounds_persistent_kernel<int32_t, true>,
                                                              b->o.block_threads, 0));
    }
    if (per_sm < 1) return GC_ERR_CUDA;
    b->per_sm = per_sm;
    }

    if (b->o.validate) {
        char* base = (char*)b->ws;
        gc::BatchFlags* fl = (gc::BatchFlags*)(base + b->off_flags);
        const int64_t spans = (NNZ + gc::kRebaseSpan - 1) / gc::kRebaseSpan;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((spans + 7) / 8, (int64_t)b->sms * 8));
        int32_t* colidx_g = nullptr;
        rc = union_colidx(*b, &colidx_g);
        if (rc != GC_OK) return rc;
        GC_CUDA(cudaMemsetAsync(fl, 0, sizeof(gc::BatchFlags), s));
        if (NNZ > 0) {
            gc::batch_colidx_kernel<<<grid, 256, 0, s>>>(colidx_cat, (const int64_t*)(base + b->off_voff),
                                                         (const int64_t*)(base + b->off_eoff), G, NNZ, colidx_g,
                                                         fl);
            GC_CUDA(cudaGetLastError());
        }
        GC_CUDA(cudaMemcpyAsync(&hf, fl, sizeof(hf), cudaMemcpyDeviceToHost, s));
        GC_CUDA(cudaStreamSynchronize(s));
        if (hf.bad_colidx) return GC_ERR_BAD_GRAPH;
        DeviceCache* dcp = nullptr;
        rc = device_cache(&dcp);
        if (rc != GC_OK) return rc;
        int64_t launches = 0;
        rc = validate_locked((const int32_t*)(base + b->off_rowptr), colidx_g, (int32_t)N, s, *dcp, &launches);
        if (rc != GC_OK) return rc;
    }
    GC_CUDA(cudaStreamSynchronize(s));
    return GC_OK;
}

int batch_status(gc_batch* b, cudaStream_t s, int32_t* max_rounds, int32_t* max_colors) {
    if (b->G == 0 || b->N == 0) {
        if (max_rounds) *max_rounds = 0;
        if (max_colors) *max_colors = 0;
        return GC_OK;
    }
    char* base = (char*)b->ws;
    RoundState hst;
    gc::BatchFlags hf;
    GC_CUDA(cudaMemcpyAsync(&hst, base + b->L.st, sizeof(hst), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaMemcpyAsync(&hf, base + b->off_flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    if (max_rounds) *max_rounds = hst.rounds;
    if (max_colors) *max_colors = hst.max_color;
    if (hf.bad_colidx) return GC_ERR_BAD_GRAPH;
    if (hst.status == gc::kStatusTimeout) return GC_ERR_TIMEOUT;
    if (hst.status == gc::kStatusMaxRounds) return GC_ERR_MAX_ROUNDS;
    if (hst.status != 0) return GC_ERR_CUDA;
    return GC_OK;
}
}  // namespace

extern "C" {

int gc_color_ex(const int32_t* rowptr, const int32_t* colidx, int32_t n, const uint32_t* priority,
                int32_t* colors_out, int32_t* ncolors, int32_t* rounds, void* stream,
                const gc_options* opt, int32_t* round_sizes, int32_t round_sizes_cap) {
    std::lock_guard<std::mutex> lock(g_mu);
    NvtxRange range("gc_color");
    g_last_cuda_error = 0;
    return color_locked(rowptr, colidx, n, priority, colors_out, ncolors, rounds, (cudaStream_t)stream,
                        opt, round_sizes, round_sizes_cap);
}

int gc_color(const int32_t* rowptr, const int32_t* colidx, int32_t n, const uint32_t* priority,
             int32_t* colors_out, int32_t* ncolors, int32_t* rounds) {
    return gc_color_ex(rowptr, colidx, n, priority, colors_out, ncolors, rounds, nullptr, nullptr,
                       nullptr, 0);
}

int gc_color_host(const int32_t* rowptr, const int32_t* colidx, int32_t n, const uint32_t* priority,
                  int32_t* colors_out, int32_t* ncolors, int32_t* rounds, void* stream,
                  const gc_options* opt) {
    std::lock_guard<std::mutex> lock(g_mu);
    NvtxRange range("gc_color_host");
    g_last_cuda_error = 0;
    if (n < 0 || !ncolors || !rounds) return GC_ERR_INVALID;
    if (n == 0) {
        *ncolors = 0;
        *rounds = 0;
        return GC_OK;
    }
    if (!rowptr || !colors_out) return GC_ERR_INVALID;
    const int64_t nnz = rowptr[n];
    if (rowptr[0] != 0 || nnz < 0) return GC_ERR_BAD_GRAPH;
    if (nnz > 0 && !colidx) return GC_ERR_INVALID;
    DeviceCache* dcp = nullptr;
    int rc = device_cache(&dcp);
    if (rc != GC_OK) return rc;
    DeviceCache& dc = *dcp;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t b_rp = align_up((size_t)(n + 1) * 4, 256), b_ci = align_up((size_t)nnz * 4 + 4, 256),
                 b_pr = priority ? align_up((size_t)n * 4, 256) : 0, b_co = align_up((size_t)n * 4, 256);
    rc = ensure_device_limited(&dc.in, &dc.in_bytes, b_rp + b_ci + b_pr + b_co, opt ? opt->workspace_limit_mb : 0);
    if (rc != GC_OK) return rc;
    char* base = (char*)dc.in;
    int32_t* d_rp = (int32_t*)base;
    int32_t* d_ci = (int32_t*)(base + b_rp);
    uint32_t* d_pr = priority ? (uint32_t*)(base + b_rp + b_ci) : nullptr;
    int32_t* d_co = (int32_t*)(base + b_rp + b_ci + b_pr);
    GC_CUDA(cudaMemcpyAsync(d_rp, rowptr, (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, s));
    if (priority) GC_CUDA(cudaMemcpyAsync(d_pr, priority, (size_t)n * 4, cudaMemcpyHostToDevice, s));
    // colidx in chunks of about equal size, cut at multiples of 32 vertices
    HostInput hin;
    hin.h_colidx = colidx;
    hin.d_colidx = d_ci;
    hin.nchunks = (int)std::max<int64_t>(1, std::min<int64_t>(8, nnz / (1 << 20)));
    hin.vb[0] = 0;
    hin.eb[0] = 0;
    for (int c = 1; c < hin.nchunks; ++c) {
        const int64_t target = nnz * c / hin.nchunks;
        int32_t v = (int32_t)(std::lower_bound(rowptr, rowptr + n + 1, (int32_t)target) - rowptr);
        v = std::max(hin.vb[c - 1], std::min(n, v & ~31));
        hin.vb[c] = v;
        // (clamped, so the copies stay inside both buffers even for a malformed
        // rowptr, which the setup scan then rejects)
        hin.eb[c] = std::min<int64_t>(nnz, std::max<int64_t>(hin.eb[c - 1], rowptr[v]));
    }
    hin.vb[hin.nchunks] = n;
    hin.eb[hin.nchunks] = nnz;
    rc = color_locked(d_rp, d_ci, n, d_pr, d_co, ncolors, rounds, s, opt, nullptr, 0, &hin);
    if (rc != GC_OK) return rc;
    GC_CUDA(cudaMemcpyAsync(colors_out, d_co, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    return GC_OK;
}

int gc_validate_csr(const int32_t* rowptr, const int32_t* colidx, int32_t n, void* stream) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_last_cuda_error = 0;
    if (n < 0 || (n > 0 && !rowptr)) return GC_ERR_INVALID;
    if (n == 0) return GC_OK;
    DeviceCache* dcp = nullptr;
    int rc = device_cache(&dcp);
    if (rc != GC_OK) return rc;
    int64_t launches = 0;
    rc = validate_locked(rowptr, colidx, n, (cudaStream_t)stream, *dcp, &launches);
    g_last_launches = launches;
    return rc;
}

const char* gc_strerror(int code) {
    switch (code) {
        case GC_OK: return "ok";
        case GC_ERR_INVALID: return "invalid argument";
        case GC_ERR_CUDA: return "CUDA runtime error";
        case GC_ERR_OOM: return "out of device memory";
        case GC_ERR_MAX_ROUNDS: return "worklist not empty after max_rounds rounds";
        case GC_ERR_TIMEOUT: return "a bounded device-side wait timed out";
        case GC_ERR_BAD_GRAPH: return "graph rejected (CSR shape, index range, self loop or asymmetry)";
        case GC_ERR_TOO_LARGE: return "graph needs more scratch memory than gc_color_noalloc's fixed buffer holds";
        default: return "unknown gc_status";
    }
}

int gc_last_cuda_error(void) { return g_last_cuda_error; }

int gc_last_round_stats(int32_t* sizes, int64_t* volumes, int32_t cap) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_last.valid || cap < 0) return GC_ERR_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g_last.device) return GC_ERR_INVALID;
    const int32_t m = std::min({g_last.rounds, cap, g_last.cap});
    if (m <= 0) return 0;
    if (sizes) {
        sizes[0] = g_last.n;
        if (m > 1) GC_CUDA(cudaMemcpy(sizes + 1, g_last.d_sizes + 1, (size_t)(m - 1) * 4, cudaMemcpyDeviceToHost));
    }
    if (volumes) {
        volumes[0] = g_last.nnz;
        if (m > 1) GC_CUDA(cudaMemcpy(volumes + 1, g_last.d_vol + 1, (size_t)(m - 1) * 8, cudaMemcpyDeviceToHost));
    }
    return m;
}

int gc_last_round_ns(int64_t* ns, int32_t cap) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_last.valid || !g_last.d_ns || !ns || cap < 0) return GC_ERR_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != g_last.device) return GC_ERR_INVALID;
    const int32_t m = std::min({g_last.rounds, cap, g_last.cap});
    if (m <= 0) return 0;
    ns[0] = 0;
    if (m > 1) {
        // starts of passes 2..m+1 (the one after the last round marks the end)
        std::vector<unsigned long long> t((size_t)m);
        GC_CUDA(cudaMemcpy(t.data(), g_last.d_ns + 1, (size_t)m * 8, cudaMemcpyDeviceToHost));
        for (int32_t k = 2; k <= m; ++k) ns[k - 1] = (int64_t)(t[k - 1] - t[k - 2]);
    }
    return m;
}

int gc_last_phase_ms(float* ms, int32_t cap) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_last.valid || !g_last.timed || !ms || cap < 0) return GC_ERR_INVALID;
    const int m = std::min(cap, 4);
    for (int i = 0; i < m; ++i) ms[i] = g_last.ms[i];
    return m;
}

int gc_release(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    int cur = 0;
    cudaGetDevice(&cur);
    for (auto& kv : g_cache) {
        cudaSetDevice(kv.first);
        cudaDeviceSynchronize();
        if (kv.second.ws) cudaFree(kv.second.ws);
        if (kv.second.in) cudaFree(kv.second.in);
        if (kv.second.host) cudaFreeHost(kv.second.host);
        for (int i = 0; i < 4; ++i)
            if (kv.second.ev[i]) cudaEventDestroy(kv.second.ev[i]);
        for (int i = 0; i < kMaxChunks; ++i)
            if (kv.second.chunk_ev[i]) cudaEventDestroy(kv.second.chunk_ev[i]);
        if (kv.second.start_ev) cudaEventDestroy(kv.second.start_ev);
        if (kv.second.copy) cudaStreamDestroy(kv.second.copy);
    }
    g_cache.clear();
    g_last.valid = 0;
    cudaSetDevice(cur);
    (void)cudaGetLastError();
    return GC_OK;
}

size_t gc_workspace_bytes(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    auto it = g_cache.find(dev);
    return it == g_cache.end() ? 0 : it->second.ws_bytes + it->second.in_bytes;
}

int64_t gc_last_launch_count(void) { return g_last_launches; }

int gc_color_noalloc(const int32_t* rowptr, const int32_t* colidx, int32_t n, const uint32_t* priority,
                     int32_t* colors_out, int32_t* ncolors, int32_t* rounds, void* stream) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_last_cuda_error = 0;
    return color_noalloc_locked(rowptr, colidx, n, priority, colors_out, ncolors, rounds,
                                (cudaStream_t)stream);
}

size_t gc_noalloc_capacity_bytes(void) { return kNoAllocBytes; }

int gc_batch_create(const int32_t* rowptr_cat, const int32_t* colidx_cat, const int64_t* vertex_offsets,
                    const int64_t* edge_offsets, int32_t num_graphs, const uint32_t* priority,
                    int32_t* colors_out, int32_t* ncolors_out, int32_t* rounds_out, const gc_options* opt,
                    void* stream, gc_batch** plan) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_last_cuda_error = 0;
    if (!plan) return GC_ERR_INVALID;
    *plan = nullptr;
    NvtxRange range("gc_batch_create");
    gc_batch* b = new (std::nothrow) gc_batch();
    if (!b) return GC_ERR_OOM;
    const int rc = batch_create_locked(rowptr_cat, colidx_cat, vertex_offsets, edge_offsets, num_graphs, priority,
                                       colors_out, ncolors_out, rounds_out, opt, (cudaStream_t)stream, b);
    if (rc != GC_OK) {
        batch_free(b);
        return rc;
    }
    *plan = b;
    return GC_OK;
}

int gc_batch_run(gc_batch* plan, void* stream) {
    if (!plan) return GC_ERR_INVALID;
    NvtxRange range("gc_batch_run");
    return batch_enqueue(*plan, (cudaStream_t)stream);
}

int gc_batch_round_stats(gc_batch* plan, int32_t* sizes, int64_t* volumes, int32_t cap, int32_t* state_bits,
                         void* stream) {
    if (!plan || cap < 0) return GC_ERR_INVALID;
    gc_batch& b = *plan;
    if (state_bits) *state_bits = b.bits;
    if (b.G == 0 || b.N == 0 || cap == 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)b.ws;
    RoundState hst;
    GC_CUDA(cudaMemcpyAsync(&hst, base + b.L.st, sizeof(hst), cudaMemcpyDeviceToHost, s));
    GC_CUDA(cudaStreamSynchronize(s));
    const int32_t m = (int32_t)std::min<int64_t>({(int64_t)hst.rounds, (int64_t)cap, b.round_cap});
    if (m <= 0) return 0;
    if (sizes) {
        sizes[0] = (int32_t)b.N;
        if (m > 1)
            GC_CUDA(cudaMemcpyAsync(sizes + 1, (const int32_t*)(base + b.L.rs) + 1, (size_t)(m - 1) * 4,
                                    cudaMemcpyDeviceToHost, s));
    }
    if (volumes) {
        volumes[0] = b.NNZ;
        if (m > 1)
            GC_CUDA(cudaMemcpyAsync(volumes + 1, (const unsigned long long*)(base + b.L.rv) + 1, (size_t)(m - 1) * 8,
                                    cudaMemcpyDeviceToHost, s));
    }
    GC_CUDA(cudaStreamSynchronize(s));
    return m;
}

int gc_batch_features(gc_batch* plan, float* features, void* stream) {
    if (!plan) return GC_ERR_INVALID;
    gc_batch& b = *plan;
    int dev = -1;
    GC_CUDA(cudaGetDevice(&dev));
    if (dev != b.device) return GC_ERR_INVALID;
    if (b.G == 0 || b.N == 0) return GC_OK;
    if (!features) return GC_ERR_INVALID;
    int64_t launches = 0;
    const int rc = batch_rebase(b, (cudaStream_t)stream, &launches);
    if (rc != GC_OK) return rc;
    char* base = (char*)b.ws;
    int32_t* colidx_g = nullptr;
    if (union_colidx(b, &colidx_g) != GC_OK) return GC_ERR_CUDA;
    return gc_features((const int32_t*)(base + b.off_rowptr), colidx_g, (int32_t)b.N, features, stream);
}

int gc_batch_launch_graph(gc_batch* plan, void* stream) {
    if (!plan) return GC_ERR_INVALID;
    gc_batch& b = *plan;
    int dev = -1;
    GC_CUDA(cudaGetDevice(&dev));
    if (dev != b.device) return GC_ERR_INVALID;
    if (b.G == 0 || b.N == 0) return GC_OK;  // nothing to launch
    if (!b.exec) {
        if (!b.cap_stream) GC_CUDA(cudaStreamCreateWithFlags(&b.cap_stream, cudaStreamNonBlocking));
        GC_CUDA(cudaStreamBeginCapture(b.cap_stream, cudaStreamCaptureModeThreadLocal));
        const int rc = batch_enqueue(b, b.cap_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t ce = cudaStreamEndCapture(b.cap_stream, &graph);
        if (rc != GC_OK || ce != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            if (ce != cudaSuccess) g_last_cuda_error = (int)ce;
            (void)cudaGetLastError();
            return rc != GC_OK ? rc : GC_ERR_CUDA;
        }
        b.graph = graph;
        GC_CUDA(cudaGraphInstantiate(&b.exec, b.graph, 0));
    }
    GC_CUDA(cudaGraphLaunch(b.exec, (cudaStream_t)stream));
    return GC_OK;
}

int gc_batch_status(gc_batch* plan, void* stream, int32_t* max_rounds, int32_t* max_colors) {
    if (!plan) return GC_ERR_INVALID;
    return batch_status(plan, (cudaStream_t)stream, max_rounds, max_colors);
}

int gc_batch_destroy(gc_batch* plan) {
    std::lock_guard<std::mutex> lock(g_mu);
    batch_free(plan);
    return GC_OK;
}

int gc_color_batched(const int64_t* vertex_offsets, const int64_t* edge_offsets, int32_t num_graphs,
                     const int32_t* rowptr_cat, const int32_t* colidx_cat, const uint32_t* priority,
                     int32_t* colors_out, int32_t* ncolors_out, int32_t* rounds_out, void* stream,
                     const gc_options* opt) {
    gc_batch* plan = nullptr;
    int rc = gc_batch_create(rowptr_cat, colidx_cat, vertex_offsets, edge_offsets, num_graphs, priority, colors_out,
                             ncolors_out, rounds_out, opt, stream, &plan);
    if (rc != GC_OK) return rc;
    rc = gc_batch_run(plan, stream);
    if (rc == GC_OK) rc = gc_batch_status(plan, stream, nullptr, nullptr);
    gc_batch_destroy(plan);
    return rc;
}

namespace {
// Median of the timed runs of one candidate.
float median_ms(std::vector<float>& v) {
    std::sort(v.begin(), v.end());
    return v.empty() ? 0.f : v[v.size() / 2];
}
}  // namespace

int gc_tune(const int32_t* rowptr, const int32_t* colidx, int32_t n, const uint32_t* priority,
            int32_t* colors_scratch, const gc_options* candidates, int32_t count, int32_t reps, void* stream,
            float* ms_out, int32_t* best) {
    if (!candidates || count < 1 || reps < 1 || !ms_out || !best) return GC_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, e = nullptr;
    GC_CUDA(cudaEventCreate(&a));
    GC_CUDA(cudaEventCreate(&e));
    int rc = GC_OK;
    *best = -1;
    for (int32_t c = 0; c < count && rc == GC_OK; ++c) {
        std::vector<float> t;
        for (int32_t r = 0; r <= reps && rc == GC_OK; ++r) {
            int32_t nc = 0, rd = 0;
            std::lock_guard<std::mutex> lock(g_mu);
            g_last_cuda_error = 0;
            if (cudaEventRecord(a, s) != cudaSuccess) { rc = GC_ERR_CUDA; break; }
            rc = color_locked(rowptr, colidx, n, priority, colors_scratch, &nc, &rd, s, &candidates[c], nullptr, 0);
            if (rc != GC_OK) break;
            float ms = 0.f;
            if (cudaEventRecord(e, s) != cudaSuccess || cudaEventSynchronize(e) != cudaSuccess ||
                cudaEventElapsedTime(&ms, a, e) != cudaSuccess) { rc = GC_ERR_CUDA; break; }
            if (r > 0) t.push_back(ms);  // the first run of each candidate is a warm-up
        }
        if (rc != GC_OK) break;
        ms_out[c] = median_ms(t);
        if (*best < 0 || ms_out[c] < ms_out[*best]) *best = c;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(e);
    return rc;
}

int gc_batch_tune(const int32_t* rowptr_cat, const int32_t* colidx_cat, const int64_t* vertex_offsets,
                  const int64_t* edge_offsets, int32_t num_graphs, const uint32_t* priority, int32_t* colors_out,
                  int32_t* ncolors_out, int32_t* rounds_out, const gc_options* candidates, int32_t count,
                  int32_t reps, void* stream, float* ms_out, int32_t* best) {
    if (!candidates || count < 1 || reps < 1 || !ms_out || !best) return GC_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, e = nullptr;
    GC_CUDA(cudaEventCreate(&a));
    GC_CUDA(cudaEventCreate(&e));
    int rc = GC_OK;
    *best = -1;
    for (int32_t c = 0; c < count && rc == GC_OK; ++c) {
        gc_batch* plan = nullptr;
        rc = gc_batch_create(rowptr_cat, colidx_cat, vertex_offsets, edge_offsets, num_graphs, priority, colors_out,
                             ncolors_out, rounds_out, &candidates[c], stream, &plan);
        if (rc != GC_OK) break;
        std::vector<float> t;
        for (int32_t r = 0; r <= reps && rc == GC_OK; ++r) {
            float ms = 0.f;
            if (cudaEventRecord(a, s) != cudaSuccess) { rc = GC_ERR_CUDA; break; }
            rc = gc_batch_launch_graph(plan, stream);
            if (rc != GC_OK) break;
            if (cudaEventRecord(e, s) != cudaSuccess || cudaEventSynchronize(e) != cudaSuccess ||
                cudaEventElapsedTime(&ms, a, e) != cudaSuccess) { rc = GC_ERR_CUDA; break; }
            if (r > 0) t.push_back(ms);
        }
        if (rc == GC_OK) rc = gc_batch_status(plan, stream, nullptr, nullptr);
        gc_batch_destroy(plan);
        if (rc != GC_OK) break;
        ms_out[c] = median_ms(t);
        if (*best < 0 || ms_out[c] < ms_out[*best]) *best = c;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(e);
    return rc;
}

size_t gc_batch_workspace_bytes(const gc_batch* plan) { return plan ? plan->ws_bytes : 0; }

int64_t gc_batch_launch_count(const gc_batch* plan) { return plan ? plan->launches_per_run : 0; }

int gc_batch_mode(const gc_batch* plan) { return plan ? plan->mode : GC_ERR_INVALID; }

}  // extern "C"
