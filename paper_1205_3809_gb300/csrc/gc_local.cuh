// Batched coloring with one thread block per graph.
//
// When a batch holds many small graphs, each graph's whole color array fits
// in one SM's shared memory (one byte per vertex: up to about 227,000
// vertices), so a block can run every synchronous round of Algorithm 2
// (Sec. 3.2) for its graph on its own: the neighbour colors it gathers come
// from shared memory instead of L2, the rounds are separated by block
// barriers instead of grid barriers, and graphs are handed out from a queue
// (largest first), one at a time, to persistent blocks, one per SM.
//
// Round k over the worklist U_k (U_1 = all vertices, every color 1):
//   A. every v in U_k reads its whole row against the colors C_k; v conflicts
//      if a neighbour that precedes v holds its color, and then takes the
//      smallest color no neighbour holds (first fit over C_k); conflicting
//      vertices and their new colors are appended to U_{k+1};
//   B. after a block barrier the new colors are written, giving C_{k+1}.
// This is exactly the Jacobi form the other paths run (Phase 2 of round k
// and Phase 1 of round k+1 read the same snapshot), so every graph gets the
// colors, color count and round count it gets alone.
//
// A warp takes 32 worklist entries {v, row start, degree, new color} at a
// time, one per lane (the next 32 are loaded, and L2 is asked for their
// rows, while these are worked on).  Graphs of average degree up to 32 (by
// default) take one thread per vertex, eight entries of its row in flight
// (a row longer than twice the warp's mean is read by the whole warp);
// denser graphs read each row with a group of L = 4..32 lanes (about half
// the average degree): 32/L vertices side by side, four such steps with
// their loads issued together, L entries of each row per step (longer rows
// loop), and the group ORs its findings in one warp reduction before handing
// them to the vertex's lane.  Findings: bits 1..31 mark colors 1..31 among
// the neighbours, bit 0 a conflict.  When colors 1..31 are all taken, the
// vertex's lane rescans its row in windows of 32 colors.
//
// A color above 255 does not fit a byte: the block gives the graph up and
// appends it to an overflow list, which a second launch colors with 32-bit
// colors.  A graph whose colors do not fit shared memory keeps the colors
// of its first vertices there and the rest in global memory.
#pragma once

#include "gc_batch.cuh"

namespace gc {

constexpr int kLocalThreads = 1024;
constexpr int kLocalWarps = kLocalThreads / 32;
constexpr int kLocalLog = 128;  // rounds whose telemetry a block holds until its graph is done

struct LocalQueue {
    unsigned next[2];   // next graph to take, per pass (byte colors, 32-bit colors)
    unsigned ovf;       // graphs handed to the 32-bit pass
    unsigned pad[29];
};

struct LocalParams {
    const int32_t* __restrict__ rowptr_g;   // union rowptr: row of global vertex x is colidx_cat[rowptr_g[x] ..]
    const int32_t* __restrict__ colidx_cat; // ids local to each graph
    const uint32_t* __restrict__ prio;      // union-indexed keys, or NULL (index priority)
    const int64_t* __restrict__ voff;       // G + 1 vertex offsets
    const int32_t* __restrict__ order;      // graphs in the order the queue hands them out
    const uint8_t* __restrict__ lanes_log2; // per graph: log2 of the lanes per vertex (0, or 2..5)
    int32_t G;
    int32_t max_rounds;                     // 0: n_g
    uint32_t smem_bytes;                    // dynamic shared memory per block
    int4* wl0;                              // worklists {v, row start, degree, new color}, union-indexed (N each)
    int4* wl1;
    uint8_t* gcol8;                         // byte colors of graphs that exceed shared memory (N)
    int32_t* gcol32;                        // colors of the 32-bit pass (N)
    int32_t* colors_out;
    int32_t* ncolors_out;
    int32_t* rounds_out;
    int32_t* ovf_list;                      // G
    LocalQueue* q;
    RoundState* st;                         // batch status, max rounds, max color
    BatchFlags* fl;
    int32_t* round_sizes;                   // telemetry: [k-1] += |U_k| (k >= 2)
    unsigned long long* round_vol;          // telemetry: [k-1] += entries round k reads (k >= 2)
    int32_t round_cap;
};

template <typename C> struct LocalColor;
template <> struct LocalColor<uint8_t> { static constexpr uint32_t kMax = 255u; };
template <> struct LocalColor<uint32_t> { static constexpr uint32_t kMax = 0x7fffffffu; };

// w precedes v: smaller key first, ties by index.
template <bool P>
__device__ __forceinline__ bool local_precedes(const uint32_t* __restrict__ prio, int64_t v0, int32_t w,
                                               int32_t v, uint32_t pv) {
    if constexpr (P) {
        const uint32_t pw = __ldg(prio + v0 + w);
        return pw < pv || (pw == pv && w < v);
    } else {
        return w < v;
    }
}

// First fit above color 31 for a vertex whose neighbours hold all of 1..31:
// its lane rescans the row once per window of 32 colors (rare).
template <typename Store>
__device__ __noinline__ uint32_t local_rescan(const int32_t* __restrict__ colidx, int32_t b, int32_t e,
                                              const Store col, int32_t n) {
    for (uint32_t lo = 32;; lo += 32) {
        uint32_t mm = 0;
        for (int32_t i = b; i < e; ++i) {
            const int32_t w = (int32_t)min((uint32_t)__ldg(colidx + i), (uint32_t)(n - 1));
            const uint32_t c = (uint32_t)col.get(w);
            if (c - lo < 32u) mm |= 1u << (c - lo);
        }
        if (mm != kFull) return lo + (uint32_t)__ffs(~mm) - 1u;
    }
}

// Findings word: bit c for a neighbour color c in 1..31, bit 0 for a
// conflict (a preceding neighbour holds v's color).
__device__ __forceinline__ uint32_t color_bit(uint32_t c) {
    uint32_t r;  // shl clamps shifts of 32 and more to 32, giving 0
    asm("shl.b32 %0, 1, %1;" : "=r"(r) : "r"(c));
    return r & ~1u;
}

// Findings of one neighbour w (color c) for vertex v (color cv, key pv).
template <bool P>
__device__ __forceinline__ uint32_t local_entry(const uint32_t* __restrict__ prio, int64_t v0, int32_t w, uint32_t c,
                                                int32_t v, uint32_t cv, uint32_t pv) {
    uint32_t m = color_bit(c);
    if (c == cv && local_precedes<P>(prio, v0, w, v, pv)) m |= 1u;
    return m;
}

// A neighbour id, kept inside the graph (an id outside [0, n) is an input
// error: it is recorded in `seen` and read as n - 1).
__device__ __forceinline__ int32_t local_id(int32_t w, int32_t n, uint32_t& seen) {
    seen = max(seen, (uint32_t)w);
    return (int32_t)min((uint32_t)w, (uint32_t)(n - 1));
}

// Ask L2 for the lines of a row that a later step reads.
__device__ __forceinline__ void local_prefetch_row(const int32_t* row, int32_t d) {
    for (int32_t o = 0; o < d; o += 32) asm volatile("prefetch.global.L2 [%0];" :: "l"(row + o));
    if (d > 1) asm volatile("prefetch.global.L2 [%0];" :: "l"(row + d - 1));
}

// Worklist entry idx of round k: U_1 is every vertex, in order.
__device__ __forceinline__ int4 local_load_entry(int k, const int4* __restrict__ U, const int32_t* __restrict__ rp,
                                                 int32_t idx, int32_t cnt) {
    int4 t = make_int4(0, 0, 0, 0);
    if (idx < cnt) {
        if (k == 1) {
            const int32_t b = __ldg(rp + idx);
            t = make_int4(idx, b, __ldg(rp + idx + 1) - b, 0);
        } else {
            t = __ldcg(U + idx);
        }
    }
    return t;
}

// Colors of the current graph: in shared memory, or -- for a graph larger
// than shared memory (SPLIT) -- its first `cap` vertices there and the rest
// in global memory.
template <typename C, bool SPLIT>
struct ColorStore {
    C* s;          // shared: vertices [0, cap)
    C* g;          // global, indexed like s (used from cap on)
    int32_t cap;
    __device__ __forceinline__ C get(int32_t w) const {
        if constexpr (SPLIT) return w < cap ? s[w] : g[w];
        return s[w];
    }
    __device__ __forceinline__ void set(int32_t w, C c) const {
        if constexpr (SPLIT) {
            if (w < cap) s[w] = c; else g[w] = c;
        } else {
            s[w] = c;
        }
    }
};

struct LocalShared {
    int g;
    unsigned cnt;
    int ovf, bad, maxc;
    unsigned long long vol;
    // per-round telemetry of the current graph (rounds 2..kLocalLog+1), added
    // to the batch's totals once the graph is done, so that a graph handed to
    // the 32-bit pass is not counted twice
    int32_t log_cnt[kLocalLog];
    unsigned long long log_vol[kLocalLog];
};

// All rounds of graph g, run by the whole block.
template <typename C, bool P, bool SPLIT>
__device__ __forceinline__ void local_color_graph(const LocalParams& p, LocalShared& sh, C* s_col, int g,
                                                  int64_t v0, int32_t n) {
    const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    {
        const int32_t* __restrict__ rp = p.rowptr_g + v0;
        const int lg = __ldg(p.lanes_log2 + g);
        const int L = 1 << lg;
        const unsigned j = lane & (unsigned)(L - 1);     // my lane in my group
        const unsigned gi = lane >> lg;                   // my group
        const int G = 32 >> lg;                           // groups (vertices side by side) per warp
        const unsigned gmask = L == 32 ? kFull : ((1u << L) - 1u) << (gi << lg);
        ColorStore<C, SPLIT> col;
        col.s = s_col;
        if constexpr (sizeof(C) == 1) {
            col.g = reinterpret_cast<C*>(p.gcol8 + v0);
        } else {
            col.g = reinterpret_cast<C*>(p.gcol32 + v0);
        }
        col.cap = (int32_t)(p.smem_bytes / sizeof(C));
        int4* const wl0 = p.wl0 + v0;
        int4* const wl1 = p.wl1 + v0;
        for (int32_t i = (int32_t)tid; i < n; i += kLocalThreads) col.set(i, (C)1);
        if (tid == 0) {
            sh.ovf = 0;
            sh.bad = 0;
            sh.maxc = 0;
        }
        __syncthreads();
        const int32_t maxr = p.max_rounds > 0 ? p.max_rounds : n;
        int32_t cnt = n;
        int k = 1;
        while (cnt > 0) {
            if (k > maxr) {
                if (tid == 0) atomicExch(&p.st->status, kStatusMaxRounds);
                break;
            }
            const int4* U = (k & 1) ? wl1 : wl0;  // U_k (k >= 2); U_1 is every vertex
            int4* Nv = (k & 1) ? wl0 : wl1;        // U_{k+1}
            if (tid == 0) {
                sh.cnt = 0u;
                sh.vol = 0ull;
            }
            __syncthreads();
            // Phase A
            unsigned vol = 0;
            constexpr int kStride = kLocalWarps * 32;
            int4 nxt = local_load_entry(k, U, rp, (int32_t)(warp * 32 + lane), cnt);
            for (int32_t base = (int32_t)warp * 32; base < cnt; base += kStride) {
                const int4 cur = nxt;
                nxt = local_load_entry(k, U, rp, base + kStride + (int32_t)lane, cnt);
                local_prefetch_row(p.colidx_cat + nxt.y, nxt.z);  // the next step's row, while this one runs
                const bool act = base + (int32_t)lane < cnt;
                const int32_t v = cur.x, b = cur.y, d = cur.z;
                const uint32_t cv = act ? (uint32_t)col.get(v) : 0u;
                uint32_t pv = 0;
                if constexpr (P) pv = act ? __ldg(p.prio + v0 + v) : 0u;
                uint32_t mine = 0;  // findings for this lane's vertex
                uint32_t seen = 0;  // largest neighbour id read (as unsigned)
                if (lg == 0) {
                    // one thread per vertex: eight entries of the row in flight.  A row
                    // longer than twice the warp's mean (and than 16) is read by the
                    // whole warp instead, so that one long row does not hold 31 idle
                    // lanes for its length.
                    const int32_t dsum = (int32_t)__reduce_add_sync(kFull, act ? (unsigned)d : 0u);
                    const bool longrow = act && (int64_t)d > max((int64_t)16, (2 * (int64_t)dsum + 31) / 32);
                    unsigned lb = __ballot_sync(kFull, longrow);
                    while (lb) {
                        const int o = __ffs(lb) - 1;
                        lb &= lb - 1;
                        const int32_t ob = __shfl_sync(kFull, b, o), od = __shfl_sync(kFull, d, o);
                        const int32_t ov = __shfl_sync(kFull, v, o);
                        const uint32_t ocv = __shfl_sync(kFull, cv, o);
                        const uint32_t opv = P ? __shfl_sync(kFull, pv, o) : 0u;
                        uint32_t m = 0;
                        for (int32_t i0 = 0; i0 < od; i0 += 128) {
                            int32_t x[4];
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int32_t i = i0 + 32 * u + (int32_t)lane;
                                x[u] = i < od ? local_id(__ldg(p.colidx_cat + ob + i), n, seen) : -1;
                            }
#pragma unroll
                            for (int u = 0; u < 4; ++u)
                                if (x[u] >= 0)
                                    m |= local_entry<P>(p.prio, v0, x[u], (uint32_t)col.get(x[u]), ov, ocv, opv);
                        }
                        m = __reduce_or_sync(kFull, m);
                        if ((int)lane == o) mine = m;
                    }
                    if (act && !longrow) {
                        int32_t i = b;
                        const int32_t e = b + d;
                        for (; i + 8 <= e; i += 8) {
                            int32_t x[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u) x[u] = local_id(__ldg(p.colidx_cat + i + u), n, seen);
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                mine |= local_entry<P>(p.prio, v0, x[u], (uint32_t)col.get(x[u]), v, cv, pv);
                        }
                        for (; i < e; ++i) {
                            const int32_t x = local_id(__ldg(p.colidx_cat + i), n, seen);
                            mine |= local_entry<P>(p.prio, v0, x, (uint32_t)col.get(x), v, cv, pv);
                        }
                    }
                } else
                for (int s0 = 0; s0 < L; s0 += 4) {
                    int32_t sv[4], sb[4], sd[4], w[4];
                    uint32_t scv[4], spv[4], m[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int src = (s0 + u) * G + (int)gi;  // the lane whose vertex my group reads
                        sv[u] = __shfl_sync(kFull, v, src);
                        sb[u] = __shfl_sync(kFull, b, src);
                        sd[u] = __shfl_sync(kFull, d, src);
                        scv[u] = __shfl_sync(kFull, cv, src);
                        spv[u] = P ? __shfl_sync(kFull, pv, src) : 0u;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        w[u] = (int32_t)j < sd[u] ? local_id(__ldg(p.colidx_cat + sb[u] + j), n, seen) : 0;
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        m[u] = (int32_t)j < sd[u]
                                   ? local_entry<P>(p.prio, v0, w[u], (uint32_t)col.get(w[u]), sv[u], scv[u], spv[u])
                                   : 0u;
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        for (int32_t i = sb[u] + L + (int32_t)j; i < sb[u] + sd[u]; i += L) {
                            const int32_t x = local_id(__ldg(p.colidx_cat + i), n, seen);
                            m[u] |= local_entry<P>(p.prio, v0, x, (uint32_t)col.get(x), sv[u], scv[u], spv[u]);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint32_t r = __shfl_sync(kFull, __reduce_or_sync(gmask, m[u]), (int)(lane % G) << lg);
                        if ((int)lane / G == s0 + u) mine = r;
                    }
                }
                if (seen >= (uint32_t)n) sh.bad = 1;
                uint32_t newc = 0;
                if (act && (mine & 1u)) {
                    const uint32_t avail = ~mine & ~1u;
                    newc = avail ? (uint32_t)__ffs(avail) - 1u : local_rescan(p.colidx_cat, b, b + d, col, n);
                }
                if (act) vol += (unsigned)d;
                const bool app = newc != 0u;
                const unsigned bal = __ballot_sync(kFull, app);
                unsigned pos = 0;
                if (lane == 0 && bal) pos = atomicAdd(&sh.cnt, (unsigned)__popc(bal));
                pos = __shfl_sync(kFull, pos, 0) + (unsigned)__popc(bal & ((1u << lane) - 1u));
                if (app) {
                    __stcg(Nv + pos, make_int4(v, b, d, (int32_t)newc));
                    if (newc > LocalColor<C>::kMax) sh.ovf = 1;
                }
            }
            vol = __reduce_add_sync(kFull, vol);
            if (lane == 0 && vol) atomicAdd(&sh.vol, (unsigned long long)vol);
            __syncthreads();
            const int32_t cnt_next = (int32_t)sh.cnt;
            if (tid == 0 && k >= 2) {
                if (k - 2 < kLocalLog) {
                    sh.log_cnt[k - 2] = cnt;
                    sh.log_vol[k - 2] = sh.vol;
                } else if (k - 1 < p.round_cap) {
                    atomicAdd(p.round_sizes + (k - 1), cnt);
                    atomicAdd(p.round_vol + (k - 1), sh.vol);
                }
            }
            if (sh.ovf) break;
            // Phase B: C_{k+1}
            for (int32_t i = (int32_t)tid; i < cnt_next; i += kLocalThreads) {
                const int4 t = __ldcg(Nv + i);
                col.set(t.x, (C)t.w);
            }
            __syncthreads();
            cnt = cnt_next;
            ++k;
        }
        __syncthreads();
        if (sh.ovf) {
            if (tid == 0) p.ovf_list[atomicAdd(&p.q->ovf, 1u)] = g;
        } else {
            int mc = 0;
            for (int32_t i = (int32_t)tid; i < n; i += kLocalThreads) {
                const int c = (int)col.get(i);
                mc = max(mc, c);
                p.colors_out[v0 + i] = c;
            }
            mc = __reduce_max_sync(kFull, mc);
            if (lane == 0 && mc) atomicMax(&sh.maxc, mc);
            for (int r = (int)tid; r < min(k - 2, kLocalLog); r += kLocalThreads)
                if (r + 1 < p.round_cap) {
                    atomicAdd(p.round_sizes + r + 1, sh.log_cnt[r]);
                    atomicAdd(p.round_vol + r + 1, sh.log_vol[r]);
                }
            __syncthreads();
            if (tid == 0) {
                p.ncolors_out[g] = sh.maxc;
                p.rounds_out[g] = k - 1;
                atomicMax(&p.st->rounds, k - 1);
                atomicMax(&p.st->max_color, sh.maxc);
                if (sh.bad) atomicExch(&p.fl->bad_colidx, 1);
            }
        }
    }
}

template <typename C, bool P>  // C: color type (byte or 32-bit); P: a priority array is given
__global__ void __launch_bounds__(kLocalThreads, 1) batch_local_kernel(LocalParams p, int pass) {
    extern __shared__ __align__(16) unsigned char s_dyn[];
    __shared__ LocalShared sh;
    const unsigned tid = threadIdx.x;
    for (;;) {
        if (tid == 0) sh.g = (int)atomicAdd(&p.q->next[pass], 1u);
        __syncthreads();
        const int qi = sh.g;
        const int limit = pass == 0 ? p.G : (int)__ldcg(&p.q->ovf);
        if (qi >= limit) break;
        const int g = pass == 0 ? __ldg(p.order + qi) : __ldcg(p.ovf_list + qi);
        const int64_t v0 = __ldg(p.voff + g);
        const int32_t n = (int32_t)(__ldg(p.voff + g + 1) - v0);
        if ((uint64_t)n * sizeof(C) <= p.smem_bytes) {
            local_color_graph<C, P, false>(p, sh, reinterpret_cast<C*>(s_dyn), g, v0, n);
        } else {
            local_color_graph<C, P, true>(p, sh, reinterpret_cast<C*>(s_dyn), g, v0, n);
        }
        __syncthreads();  // shared memory and sh are reused by the next graph
    }
}

}  // namespace gc
