// Device code of the GB300 speculative coloring path (Algorithm 2 of the
// paper, "Iterative", Sec. 3.2, run in synchronous rounds).
//
// Fused pass k (k >= 2) over the worklist U_k, reading the colors C_k that
// round k's Phase 1 produced:
//   * Phase 2 of round k: v in U_k conflicts iff a neighbour w with
//     C_k[w] == C_k[v] precedes v ((prio[w], w) < (prio[v], v));
//   * Phase 1 of round k+1 for the conflicting v: first fit over the same
//     snapshot C_k (the smallest color > 0 no neighbour holds, Sec. 3.1).
// Both read adj(v) and C_k only, so one pass over adj(v) yields both; the
// two-phase form would read every adjacency twice.
//
// Double buffering: pass k reads X[k & 1] and writes X[(k + 1) & 1].  A
// vertex that settles in pass k writes its final color to the other buffer
// too, so both buffers hold it from then on; no copy of the whole array is
// ever needed.  Round 1 colors every vertex 1 (all colors start at 0), so
// pass 1 needs no color reads: v conflicts iff some neighbour precedes it,
// and then its round-2 color is 2.
//
// Worklists are kept per degree bin (thread / warp / block per vertex).  A
// vertex's bin never changes, so a vertex sent back is appended to the list
// of its own bin with a warp-aggregated atomic.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gc {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBinThread = 0, kBinWarp = 1, kBinBlock = 2;

// Status codes shared with gc.h (kept numerically equal).
constexpr int kStatusOk = 0;
constexpr int kStatusMaxRounds = -4;
constexpr int kStatusTimeout = -5;

// A grid barrier gives up after this long (globaltimer ns) or this many polls.
constexpr unsigned long long kBarrierTimeoutNs = 4000000000ull;
constexpr unsigned kBarrierMaxPolls = 1u << 26;

struct Stats {
    int max_degree;
    int bad;               // rowptr[0] != 0 or a negative degree
    int nnz;               // rowptr[n]
    int pad;
    unsigned bin_count[3]; // vertices per degree bin
    unsigned pad2;
};

struct RoundState {
    unsigned cnt[3][3];    // [k % 3][bin] = |U_k within bin|
    unsigned tick[3];      // work tickets handed out in pass k, slot k % 3
    unsigned defer_cnt[3]; // pass 1: vertices above the thread bin, per bin
    unsigned defer_tick;
    unsigned bar_count;
    unsigned bar_gen;
    int status;
    int rounds;
    int max_color;
    int pad;
};

template <typename T>
struct Params {
    const int32_t* __restrict__ rowptr;
    const int32_t* __restrict__ colidx;
    const uint32_t* __restrict__ prio;  // NULL = index priority
    int32_t n;
    int32_t t1, t2;                     // degree bin limits
    int32_t max_rounds;
    T* X0;
    T* X1;
    int32_t* colors_out;
    int32_t* listA0; int32_t* listA1; int32_t* listA2;  // worklists of even k
    int32_t* listB0; int32_t* listB1; int32_t* listB2;  // worklists of odd k
    RoundState* st;
    int32_t* round_sizes;               // device telemetry, round_sizes[k-1] = |U_k|
    unsigned long long* round_vol;      // device telemetry, round_vol[k-1] = vol(U_k)
    int32_t round_cap;
};

// Add a block's share of vol(U_{r}) (sum of degrees) to round_vol[r-1].
__device__ __forceinline__ void fold_volume(unsigned long long* round_vol, int32_t cap, int r,
                                            unsigned long long vol) {
    __shared__ unsigned long long s_vol;
    if (threadIdx.x == 0) s_vol = 0;
    __syncthreads();
    if (vol) atomicAdd(&s_vol, vol);
    __syncthreads();
    if (threadIdx.x == 0 && s_vol && r - 1 < cap) atomicAdd(&round_vol[r - 1], s_vol);
}

// ------------------------------------------------------------ helpers

__device__ __forceinline__ unsigned ld_cg_u32(const unsigned* p) { return __ldcg(p); }

// w precedes v: (prio[w], w) < (prio[v], v); pv = prio[v] (ignored if no prio).
__device__ __forceinline__ bool precedes(const uint32_t* __restrict__ prio, int32_t w, int32_t v,
                                         uint32_t pv) {
    if (prio) {
        const uint32_t pw = __ldg(prio + w);
        if (pw != pv) return pw < pv;
    }
    return w < v;
}

// Append v (if flag) to list with one atomic per warp.  All 32 lanes call it.
__device__ __forceinline__ void warp_append(bool flag, int32_t v, int32_t* list, unsigned* cnt) {
    const unsigned ballot = __ballot_sync(kFull, flag);
    if (ballot == 0) return;
    const unsigned lane = threadIdx.x & 31u;
    const int leader = __ffs(ballot) - 1;
    unsigned base = 0;
    if ((int)lane == leader) base = atomicAdd(cnt, (unsigned)__popc(ballot));
    base = __shfl_sync(kFull, base, leader);
    if (flag) list[base + __popc(ballot & ((1u << lane) - 1u))] = v;
}

// Bits of colors base+1 .. base+256 seen by one thread.
struct Mask256 {
    uint64_t w0, w1, w2, w3;
    __device__ __forceinline__ void clear() { w0 = w1 = w2 = w3 = 0; }
    // idx = color - 1 - base; anything outside [0, 256) is ignored
    __device__ __forceinline__ void set(unsigned idx) {
        if (idx < 256u) {
            const uint64_t bit = 1ull << (idx & 63u);
            const unsigned q = idx >> 6;
            w0 |= (q == 0u) ? bit : 0ull;
            w1 |= (q == 1u) ? bit : 0ull;
            w2 |= (q == 2u) ? bit : 0ull;
            w3 |= (q == 3u) ? bit : 0ull;
        }
    }
    __device__ __forceinline__ void warp_reduce(uint32_t r[8]) const {
        r[0] = __reduce_or_sync(kFull, (uint32_t)w0);
        r[1] = __reduce_or_sync(kFull, (uint32_t)(w0 >> 32));
        r[2] = __reduce_or_sync(kFull, (uint32_t)w1);
        r[3] = __reduce_or_sync(kFull, (uint32_t)(w1 >> 32));
        r[4] = __reduce_or_sync(kFull, (uint32_t)w2);
        r[5] = __reduce_or_sync(kFull, (uint32_t)(w2 >> 32));
        r[6] = __reduce_or_sync(kFull, (uint32_t)w3);
        r[7] = __reduce_or_sync(kFull, (uint32_t)(w3 >> 32));
    }
};

// Index of the first clear bit of an 8-word mask, or -1 if all 256 are set.
__device__ __forceinline__ int first_clear(const uint32_t r[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if (r[j] != 0xffffffffu) return j * 32 + __ffs(~r[j]) - 1;
    return -1;
}

// --------------------------------------------------- bounded grid barrier

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// All blocks of a cooperative launch meet here.  Returns false (and sets
// status = timeout) if the wait gave up; the caller then leaves the loop.
__device__ __forceinline__ bool grid_barrier(RoundState* st) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* vgen = &st->bar_gen;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&st->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&st->bar_count, 0u);
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            const unsigned long long t0 = globaltimer_ns();
            unsigned polls = 0;
            while (*vgen == gen) {
                __nanosleep(64);
                if (++polls >= kBarrierMaxPolls || globaltimer_ns() - t0 > kBarrierTimeoutNs) {
                    atomicExch(&st->status, kStatusTimeout);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        if (*((volatile int*)&st->status) == kStatusTimeout) ok = 0;
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ __forceinline__ void fold_max_color(RoundState* st, int maxc) {
    __shared__ int s_max;
    if (threadIdx.x == 0) s_max = 0;
    __syncthreads();
    const int m = __reduce_max_sync(kFull, maxc);
    if ((threadIdx.x & 31u) == 0 && m > 0) atomicMax(&s_max, m);
    __syncthreads();
    if (threadIdx.x == 0 && s_max > 0) atomicMax(&st->max_color, s_max);
}

// ------------------------------------------------------------ setup scan

// Degree statistics: max degree, vertices per bin, shape checks of rowptr.
__global__ void stats_kernel(const int32_t* __restrict__ rowptr, int32_t n, int32_t t1, int32_t t2,
                             Stats* s) {
    __shared__ unsigned s_bins[3];
    __shared__ int s_max, s_bad;
    if (threadIdx.x < 3) s_bins[threadIdx.x] = 0;
    if (threadIdx.x == 0) { s_max = 0; s_bad = 0; }
    __syncthreads();
    int mx = 0, bad = 0;
    unsigned b0 = 0, b1 = 0, b2 = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = __ldg(rowptr + v + 1) - __ldg(rowptr + v);
        if (d < 0) bad = 1;
        mx = max(mx, d);
        b0 += (d <= t1);
        b1 += (d > t1 && d <= t2);
        b2 += (d > t2);
    }
    atomicMax(&s_max, mx);
    if (bad) s_bad = 1;
    if (b0) atomicAdd(&s_bins[0], b0);
    if (b1) atomicAdd(&s_bins[1], b1);
    if (b2) atomicAdd(&s_bins[2], b2);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicMax(&s->max_degree, s_max);
        if (s_bad) s->bad = 1;
        for (int b = 0; b < 3; ++b)
            if (s_bins[b]) atomicAdd(&s->bin_count[b], s_bins[b]);
        if (blockIdx.x == 0) {
            if (__ldg(rowptr) != 0) s->bad = 1;
            s->nnz = __ldg(rowptr + n);
        }
    }
}

// ------------------------------------------------------------- pass 1

// Thread-bin vertices decide round 1 here; larger ones are deferred to
// pass1_big_kernel.  Round 1 is closed form: C_1 = 1 everywhere, so v
// conflicts iff some neighbour precedes it (early exit), and C_2[v] = 2.
template <typename T>
__global__ void __launch_bounds__(256) pass1_thread_kernel(Params<T> p) {
    RoundState* st = p.st;
    int maxc = 0;
    unsigned long long vol = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < p.n;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t vv = base + threadIdx.x;
        const bool valid = vv < p.n;
        const int32_t v = valid ? (int32_t)vv : 0;
        bool conflict = false, defer_w = false, defer_b = false;
        if (valid) {
            const int32_t b = __ldg(p.rowptr + v), e = __ldg(p.rowptr + v + 1);
            const int32_t d = e - b;
            if (d > p.t1) {
                defer_w = d <= p.t2;
                defer_b = !defer_w;
            } else {
                const uint32_t pv = p.prio ? __ldg(p.prio + v) : 0u;
                for (int32_t i = b; i < e; ++i)
                    if (precedes(p.prio, __ldg(p.colidx + i), v, pv)) { conflict = true; break; }
                if (conflict) vol += (unsigned long long)d;
                p.X0[v] = conflict ? (T)2 : (T)1;
                if (!conflict) {
                    p.X1[v] = (T)1;
                    p.colors_out[v] = 1;
                    maxc = 1;
                }
            }
        }
        warp_append(conflict, v, p.listA0, &st->cnt[2][kBinThread]);
        warp_append(defer_w, v, p.listB1, &st->defer_cnt[kBinWarp]);
        warp_append(defer_b, v, p.listB2, &st->defer_cnt[kBinBlock]);
    }
    fold_max_color(st, maxc);
    fold_volume(p.round_vol, p.round_cap, 2, vol);
}

// Round 1 for the deferred warp- and block-bin vertices, early exit on the
// first preceding neighbour.
template <typename T>
__device__ __forceinline__ void pass1_finish(const Params<T>& p, int32_t v, int32_t deg, bool conflict,
                                             int bin, int& maxc, unsigned long long& vol) {
    p.X0[v] = conflict ? (T)2 : (T)1;
    if (!conflict) {
        p.X1[v] = (T)1;
        p.colors_out[v] = 1;
        maxc = 1;
    } else {
        int32_t* list = bin == kBinWarp ? p.listA1 : p.listA2;
        list[atomicAdd(&p.st->cnt[2][bin], 1u)] = v;
        vol += (unsigned long long)deg;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) pass1_big_kernel(Params<T> p) {
    __shared__ unsigned s_task;
    RoundState* st = p.st;
    const unsigned nW = __ldcg(&st->defer_cnt[kBinWarp]);
    const unsigned nB = __ldcg(&st->defer_cnt[kBinBlock]);
    const unsigned warps = blockDim.x >> 5;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const unsigned tasksW = (nW + warps - 1) / warps;
    const unsigned total = nB + tasksW;
    int maxc = 0;
    unsigned long long vol = 0;
    for (;;) {
        if (threadIdx.x == 0) s_task = atomicAdd(&st->defer_tick, 1u);
        __syncthreads();
        unsigned t = s_task;
        __syncthreads();
        if (t >= total) break;
        if (t < nB) {
            const int32_t v = __ldcg(p.listB2 + t);
            const int32_t b = __ldg(p.rowptr + v), e = __ldg(p.rowptr + v + 1);
            const uint32_t pv = p.prio ? __ldg(p.prio + v) : 0u;
            bool conflict = false;
            for (int32_t c = b; c < e; c += blockDim.x) {
                const int32_t i = c + threadIdx.x;
                const bool hit = i < e && precedes(p.prio, __ldg(p.colidx + i), v, pv);
                if (__syncthreads_or(hit)) { conflict = true; break; }
            }
            if (threadIdx.x == 0) pass1_finish(p, v, e - b, conflict, kBinBlock, maxc, vol);
        } else {
            const unsigned i = (t - nB) * warps + warp;
            if (i < nW) {
                const int32_t v = __ldcg(p.listB1 + i);
                const int32_t b = __ldg(p.rowptr + v), e = __ldg(p.rowptr + v + 1);
                const uint32_t pv = p.prio ? __ldg(p.prio + v) : 0u;
                bool conflict = false;
                for (int32_t c = b; c < e; c += 32) {
                    const int32_t j = c + (int32_t)lane;
                    const bool hit = j < e && precedes(p.prio, __ldg(p.colidx + j), v, pv);
                    if (__any_sync(kFull, hit)) { conflict = true; break; }
                }
                if (lane == 0) pass1_finish(p, v, e - b, conflict, kBinWarp, maxc, vol);
            }
        }
    }
    fold_max_color(st, maxc);
    fold_volume(p.round_vol, p.round_cap, 2, vol);
}

// ------------------------------------------------- fused pass, k >= 2

template <typename T>
struct PassIO {
    const T* Xc;        // C_k
    T* Xn;              // receives C_{k+1} (conflicting) or the final color (settled)
    const int32_t* cur0; const int32_t* cur1; const int32_t* cur2;
    int32_t* nxt0; int32_t* nxt1; int32_t* nxt2;
    unsigned* ncnt;     // st->cnt[(k + 1) % 3]
};

template <typename T>
__device__ __forceinline__ PassIO<T> pass_io(const Params<T>& p, int k) {
    PassIO<T> io;
    const bool odd = (k & 1) != 0;
    io.Xc = odd ? p.X1 : p.X0;
    io.Xn = odd ? p.X0 : p.X1;
    io.cur0 = odd ? p.listB0 : p.listA0;
    io.cur1 = odd ? p.listB1 : p.listA1;
    io.cur2 = odd ? p.listB2 : p.listA2;
    io.nxt0 = odd ? p.listA0 : p.listB0;
    io.nxt1 = odd ? p.listA1 : p.listB1;
    io.nxt2 = odd ? p.listA2 : p.listB2;
    io.ncnt = p.st->cnt[(k + 1) % 3];
    return io;
}

// Thread per vertex (degree <= t1 <= 63): one 64-bit mask holds every color
// that can matter, since first fit never exceeds degree + 1.
template <typename T>
__device__ __forceinline__ void thread_vertex(const Params<T>& p, const PassIO<T>& io, int32_t v,
                                              bool valid, int& maxc, unsigned long long& vol) {
    bool conflict = false;
    if (valid) {
        const int32_t b = __ldg(p.rowptr + v), e = __ldg(p.rowptr + v + 1);
        const T cv = __ldcg(io.Xc + v);
        const uint32_t pv = p.prio ? __ldg(p.prio + v) : 0u;
        uint64_t mask = 0;
#pragma unroll 4
        for (int32_t i = b; i < e; ++i) {
            const int32_t w = __ldg(p.colidx + i);
            const T c = __ldcg(io.Xc + w);
            if (c == cv && precedes(p.prio, w, v, pv)) conflict = true;
            const unsigned idx = (unsigned)c - 1u;
            mask |= (idx < 64u) ? (1ull << idx) : 0ull;
        }
        if (conflict) {
            io.Xn[v] = (T)__ffsll((long long)~mask);
            vol += (unsigned long long)(e - b);
        } else {
            io.Xn[v] = cv;
            p.colors_out[v] = (int32_t)cv;
            maxc = max(maxc, (int)cv);
        }
    }
    warp_append(conflict, v, io.nxt0, &io.ncnt[kBinThread]);
}

// Warp per vertex: lanes stride over adj(v); colors in a 256-wide window are
// OR-reduced across the warp; a full window moves on and rescans.
template <typename T>
__device__ __forceinline__ void warp_vertex(const Params<T>& p, const PassIO<T>& io, int32_t v,
                                            int& maxc, unsigned long long& vol) {
    const int32_t lane = (int32_t)(threadIdx.x & 31u);
    const int32_t b = __ldg(p.rowptr + v), e = __ldg(p.rowptr + v + 1);
    const T cv = __ldcg(io.Xc + v);
    const uint32_t pv = p.prio ? __ldg(p.prio + v) : 0u;
    bool conflict = false;
    Mask256 m;
    m.clear();
#pragma unroll 2
    for (int32_t i = b + lane; i < e; i += 32) {
        const int32_t w = __ldg(p.colidx + i);
        const T c = __ldcg(io.Xc + w);
        if (c == cv && precedes(p.prio, w, v, pv)) conflict = true;
        m.set((unsigned)c - 1u);
    }
    if (!__any_sync(kFull, conflict)) {
        if (lane == 0) {
            io.Xn[v] = cv;
            p.colors_out[v] = (int32_t)cv;
        }
        maxc = max(maxc, (int)cv);
        return;
    }
    uint32_t r[8];
    m.warp_reduce(r);
    int ff = first_clear(r);
    unsigned base = 0;
    while (ff < 0) {
        base += 256u;
        m.clear();
        for (int32_t i = b + lane; i < e; i += 32) {
            const T c = __ldcg(io.Xc + __ldg(p.colidx + i));
            m.set((unsigned)c - 1u - base);
        }
        m.warp_reduce(r);
        ff = first_clear(r);
    }
    if (lane == 0) {
        io.Xn[v] = (T)(base + (unsigned)ff + 1u);
        io.nxt1[atomicAdd(&io.ncnt[kBinWarp], 1u)] = v;
        vol += (unsigned long long)(e - b);
    }
}

// Block per vertex: as the warp form, with the warps' masks OR-ed in shared memory.
template <typename T>
__device__ __forceinline__ void block_vertex(const Params<T>& p, const PassIO<T>& io, int32_t v,
                                             int& maxc, unsigned long long& vol, uint32_t* s_mask) {
    const int32_t b = __ldg(p.rowptr + v), e = __ldg(p.rowptr + v + 1);
    const T cv = __ldcg(io.Xc + v);
    const uint32_t pv = p.prio ? __ldg(p.prio + v) : 0u;
    bool conflict = false;
    Mask256 m;
    m.clear();
#pragma unroll 2
    for (int32_t i = b + (int32_t)threadIdx.x; i < e; i += (int32_t)blockDim.x) {
        const int32_t w = __ldg(p.colidx + i);
        const T c = __ldcg(io.Xc + w);
        if (c == cv && precedes(p.prio, w, v, pv)) conflict = true;
        m.set((unsigned)c - 1u);
    }
    if (!__syncthreads_or(conflict)) {
        if (threadIdx.x == 0) {
            io.Xn[v] = cv;
            p.colors_out[v] = (int32_t)cv;
        }
        maxc = max(maxc, (int)cv);
        return;
    }
    unsigned base = 0;
    for (;;) {
        if (threadIdx.x < 8) s_mask[threadIdx.x] = 0u;
        __syncthreads();
        uint32_t r[8];
        m.warp_reduce(r);
        if ((threadIdx.x & 31u) == 0) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (r[j]) atomicOr(&s_mask[j], r[j]);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 8; ++j) r[j] = s_mask[j];
        const int ff = first_clear(r);
        __syncthreads();
        if (ff >= 0) {
            if (threadIdx.x == 0) {
                io.Xn[v] = (T)(base + (unsigned)ff + 1u);
                io.nxt2[atomicAdd(&io.ncnt[kBinBlock], 1u)] = v;
                vol += (unsigned long long)(e - b);
            }
            return;
        }
        base += 256u;
        m.clear();
        for (int32_t i = b + (int32_t)threadIdx.x; i < e; i += (int32_t)blockDim.x) {
            const T c = __ldcg(io.Xc + __ldg(p.colidx + i));
            m.set((unsigned)c - 1u - base);
        }
    }
}

// One fused pass over U_k.  Work is handed out by ticket: block-bin vertices
// first (largest first helps balance), then warp-bin chunks (one vertex per
// warp), then thread-bin chunks (one vertex per thread).
template <typename T>
__device__ __forceinline__ void run_pass(const Params<T>& p, int k, unsigned nL, unsigned nM,
                                         unsigned nH, int& maxc, unsigned* s_task, uint32_t* s_mask) {
    const PassIO<T> io = pass_io(p, k);
    unsigned* tick = &p.st->tick[k % 3];
    const unsigned warps = blockDim.x >> 5;
    const unsigned tasksM = (nM + warps - 1) / warps;
    const unsigned tasksL = (nL + blockDim.x - 1) / blockDim.x;
    const unsigned total = nH + tasksM + tasksL;
    unsigned long long vol = 0;  // vol(U_{k+1}) share of this thread
    for (;;) {
        if (threadIdx.x == 0) *s_task = atomicAdd(tick, 1u);
        __syncthreads();
        unsigned t = *s_task;
        __syncthreads();
        if (t >= total) break;
        if (t < nH) {
            block_vertex(p, io, __ldcg(io.cur2 + t), maxc, vol, s_mask);
        } else if ((t -= nH) < tasksM) {
            const unsigned i = t * warps + (threadIdx.x >> 5);
            if (i < nM) warp_vertex(p, io, __ldcg(io.cur1 + i), maxc, vol);
        } else {
            t -= tasksM;
            const unsigned i = t * blockDim.x + threadIdx.x;
            const bool valid = i < nL;
            thread_vertex(p, io, valid ? __ldcg(io.cur0 + i) : 0, valid, maxc, vol);
        }
    }
    fold_volume(p.round_vol, p.round_cap, k + 1, vol);
}

// All rounds k >= 2 in one cooperative launch; a bounded grid barrier
// separates the rounds.  Every block reads the same counts after a barrier,
// so all blocks leave the loop in the same round.
template <typename T>
__global__ void __launch_bounds__(512) rounds_persistent_kernel(Params<T> p) {
    __shared__ unsigned s_task;
    __shared__ uint32_t s_mask[8];
    RoundState* st = p.st;
    int maxc = 0;
    for (int k = 2;; ++k) {
        const unsigned* c = st->cnt[k % 3];
        const unsigned nL = ld_cg_u32(c + 0), nM = ld_cg_u32(c + 1), nH = ld_cg_u32(c + 2);
        const unsigned size = nL + nM + nH;
        if (size == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) st->rounds = k - 1;
            break;
        }
        if (k > p.max_rounds) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                st->rounds = k - 1;
                st->status = kStatusMaxRounds;
            }
            break;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            unsigned* z = st->cnt[(k + 2) % 3];
            z[0] = z[1] = z[2] = 0u;
            st->tick[(k + 2) % 3] = 0u;
            if (k - 1 < p.round_cap) p.round_sizes[k - 1] = (int32_t)size;
        }
        run_pass(p, k, nL, nM, nH, maxc, &s_task, s_mask);
        if (!grid_barrier(st)) break;
    }
    fold_max_color(st, maxc);
}

// One pass per launch (loop mode 1): counts come from the host.
template <typename T>
__global__ void __launch_bounds__(512) round_kernel(Params<T> p, int k, unsigned nL, unsigned nM,
                                                    unsigned nH) {
    __shared__ unsigned s_task;
    __shared__ uint32_t s_mask[8];
    int maxc = 0;
    run_pass(p, k, nL, nM, nH, maxc, &s_task, s_mask);
    fold_max_color(p.st, maxc);
}

// ------------------------------------------------------------ validation

__device__ __forceinline__ uint64_t fmix64(uint64_t k) {
    // MurmurHash3 64-bit finaliser (Appleby)
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

struct ValidateOut {
    unsigned long long sum_fwd, sum_bwd;
    int bad_index, self_loop;
};

// Range and self-loop checks per entry; symmetry via hash sums of the entry
// multiset E and of its transpose (equal when E is symmetric).
__global__ void validate_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                int32_t n, ValidateOut* out) {
    const unsigned lane = threadIdx.x & 31u;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long f = 0, g = 0;
    int bad = 0, loop = 0;
    for (int64_t v = warp; v < n; v += nwarps) {
        const int32_t b = __ldg(rowptr + v), e = __ldg(rowptr + v + 1);
        for (int32_t i = b + (int32_t)lane; i < e; i += 32) {
            const int32_t w = __ldg(colidx + i);
            if (w < 0 || w >= n) { bad = 1; continue; }
            if (w == (int32_t)v) loop = 1;
            f += fmix64(((uint64_t)(uint32_t)v << 32) | (uint32_t)w);
            g += fmix64(((uint64_t)(uint32_t)w << 32) | (uint32_t)v);
        }
    }
    if (f) atomicAdd(&out->sum_fwd, f);
    if (g) atomicAdd(&out->sum_bwd, g);
    if (bad) out->bad_index = 1;
    if (loop) out->self_loop = 1;
}

}  // namespace gc
