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
// vertex that settles writes its final color to both buffers, so no copy of
// the whole array is ever needed.  Round 1 colors every vertex 1 (all colors
// start at 0), so pass 1 needs no color reads: v conflicts iff some
// neighbour precedes it, and then its round-2 color is 2.
//
// Active lists.  A color word carries a flag bit once its vertex has settled
// (its color is final).  A vertex v still in U reads each neighbour's word
// anyway (the conflict test and first fit need this round's color), and a
// flagged neighbour is then folded into v's static mask (the colors 1..256
// held by settled neighbours, kept per vertex across rounds) and dropped
// from v's active list, which pass k rewrites compacted into the other of
// two buffers.  Later rounds read only the neighbours that had not settled,
// plus v's static mask; first fit looks at static | this round's colors.  A
// first fit beyond 256 rescans the original row (every neighbour).  The
// flag makes 16-bit state hold colors < 2^15: a larger color sets an
// overflow status and the host reruns with 32-bit state.
//
// Work is split into warp-sized tasks, binned by the current active length:
//   S bin (length <= s_max <= 32): 32 worklist entries per task (down to 4
//     in the small rounds at the end), their lists walked as one flat range;
//   M bin (s_max < length <= m_max <= 256): up to 16 worklist entries per
//     task, each list read by the whole warp in turn (colors 1..64 in
//     registers);
//   H bin (length > m_max): one chunk of up to 1024 entries of one list per
//     task; a list of one chunk is decided by its warp, and the chunks of a
//     longer list OR their conflict flag and color windows into a per-vertex
//     record, write their survivors at offsets taken from an atomic counter,
//     and the warp that finishes the last chunk decides.
// Tasks are dealt to warps round-robin; no block-wide barrier is taken
// inside a round.
//
// Priority: the round kernels are instantiated for index priority (the test
// is one compare) and for a priority array, whose (key, index) order round 2
// evaluates once per kept neighbour and stores in bit 31 of the active-list
// entry.  Loops: all rounds in one cooperative launch with a bounded grid
// barrier (optionally handing the last rounds to block 0), one launch per
// round, or a CUDA graph whose while node repeats a round kernel and a
// one-thread condition kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gc {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBinS = 0, kBinM = 1, kBinH = 2;
constexpr int kPerLane = 8;                   // adjacency entries per lane in a hub chunk
constexpr int kSmallMaxLimit = 32;            // S bin: length <= 32
constexpr int kMedMaxLimit = 32 * kPerLane;   // M bin: length <= 256
constexpr int kHubSub = 32 * kPerLane;        // 256 entries: one sub-block of a hub chunk
constexpr int kChunk = 4 * kHubSub;           // 1024 entries per H-bin task
constexpr int kPass1Flat = 256;               // pass 1: longer rows go to pass1_long_kernel
constexpr int kPass1LongBlocksPerSm = 8;      // pass 1, long rows: grid of 8 blocks per SM
#ifndef GC_FLAT_BATCHES
#define GC_FLAT_BATCHES 4
#endif
#ifndef GC_MIN_BLOCKS
#define GC_MIN_BLOCKS 4
#endif
#ifndef GC_MED_PER_TASK
#define GC_MED_PER_TASK 16
#endif

constexpr int kFlatBatches = GC_FLAT_BATCHES;  // flat tasks: batches in flight together
constexpr int kMedPerTask = GC_MED_PER_TASK;   // M-bin vertices per task
constexpr int kShortPerTaskMin = 4;            // S-bin vertices per task in a small round
constexpr int kMinBlocks = GC_MIN_BLOCKS;      // round kernels: blocks per SM the registers allow
constexpr int kWarpsPerBlockMax = 8;          // blocks of <= 256 threads

// Status codes shared with gc.h (kept numerically equal), and one internal.
constexpr int kStatusOk = 0;
constexpr int kStatusMaxRounds = -4;
constexpr int kStatusTimeout = -5;
constexpr int kStatusColorOverflow = -100;    // 16-bit state too narrow: rerun with 32-bit

// A grid barrier gives up after this long (globaltimer ns) or this many polls.
constexpr unsigned long long kBarrierTimeoutNs = 4000000000ull;
constexpr unsigned kBarrierMaxPolls = 1u << 26;

// Settled flag and color field of a color word.
template <typename T> struct Word;
template <> struct Word<uint16_t> { static constexpr uint32_t kFlag = 0x8000u; };
template <> struct Word<int32_t> { static constexpr uint32_t kFlag = 0x80000000u; };

template <typename T>
__device__ __forceinline__ uint32_t word_raw(T x) {
    return sizeof(T) == 2 ? (uint32_t)(uint16_t)x : (uint32_t)x;
}
template <typename T>
__device__ __forceinline__ uint32_t word_color(T x) { return word_raw(x) & (Word<T>::kFlag - 1u); }
template <typename T>
__device__ __forceinline__ bool word_settled(T x) { return (word_raw(x) & Word<T>::kFlag) != 0u; }

struct Stats {
    int max_degree;
    int bad;                      // rowptr[0] != 0 or a negative degree
    int nnz;                      // rowptr[n]
    unsigned defer;               // vertices with degree > kPass1Flat
    unsigned cap[3];              // list capacities: degree >= 1, > s_max, > m_max
    unsigned pad;
    unsigned long long hub_chunks;  // sum over degree > m_max of ceil(degree / kChunk)
};

// One round's worklist counters.  Every warp appends through them, so each
// sits on its own 128-byte line (its own L2 slice): on one line, the atomics
// of all bins queued at one slice, which then served a quarter more requests
// than any other.  A hub's two counters (its worklist position and its first
// chunk) share one 64-bit word, taken with one atomic.
struct RoundCounts {
    alignas(128) unsigned s;               // |U_k in S|
    alignas(128) unsigned m;               // |U_k in M|
    alignas(128) unsigned long long hc;    // |U_k in H| (bits 0..31) | chunks of U_k in H (bits 32..63)
    alignas(128) unsigned vol;             // active entries round k reads
};

__host__ __device__ __forceinline__ unsigned hub_count(unsigned long long hc) { return (unsigned)hc; }
__host__ __device__ __forceinline__ unsigned hub_chunks(unsigned long long hc) { return (unsigned)(hc >> 32); }

// The append counters, the two barrier words and the result words sit on
// separate 128-byte lines, so that blocks polling the barrier do not slow
// down the atomics of blocks still working.
struct RoundState {
    RoundCounts rc[3];     // [k % 3]: the counts of U_k
    alignas(128) unsigned defer_cnt;  // pass 1: vertices above kPass1Flat
    alignas(128) unsigned task_next[3];  // [k % 3]: tasks of round k claimed so far (beyond the first two per warp)
    alignas(128) unsigned bar_count;
    alignas(128) unsigned bar_gen;
    alignas(128) int status;
    int status_at_barrier; // status as the last block to reach the latest barrier saw it
    int rounds;
    int max_color;
    int graph_round;       // loop mode 2: the round the graph's next iteration runs
};

// Per H-bin vertex of the current round (indexed by its worklist position).
struct HubRecord {
    unsigned mask[8];      // colors 1..256 seen by any chunk this round
    unsigned stat[8];      // colors 1..256 of neighbours found settled this round
    unsigned conflict;
    unsigned done;         // chunks finished
    unsigned kept;         // active entries kept for the next round
    unsigned pad[13];
};

template <typename T>
struct Params {
    const int32_t* __restrict__ rowptr;
    const int32_t* __restrict__ colidx;
    const uint32_t* __restrict__ prio;  // NULL = index priority
    int32_t n;
    int32_t s_max, m_max;               // length bin limits
    int32_t max_rounds;
    int32_t tail_volume;                // rounds reading <= this many entries run in block 0 alone (< 0: never)
    uint32_t barrier_polls;             // the grid barrier gives up after this many polls
    uint32_t color_limit;               // a color >= this overflows (16-bit state)
    T* X0;
    T* X1;
    int32_t* colors_out;
    int32_t* settle_round;              // NULL, or receives the round in which each vertex settled
    int32_t* act0;                      // active lists (row starts as in colidx)
    int32_t* act1;
    uint32_t* stat;                     // static masks, 8 words per vertex
    // worklists per parity (A: even k, B: odd k): S, M, H entries
    // {vertex, row start, active length, degree}, first chunk of each H
    // entry, owner position of each chunk
    int4* SA; int4* MA; int4* HA; int32_t* HcA; int32_t* OA;
    int4* SB; int4* MB; int4* HB; int32_t* HcB; int32_t* OB;
    int32_t* defer;                     // pass 1: rows longer than kPass1Flat
    HubRecord* hubs;
    RoundState* st;
    int32_t* round_sizes;               // device telemetry, round_sizes[k-1] = |U_k|
    unsigned long long* round_vol;      // device telemetry, round_vol[k-1] = entries round k reads
    unsigned long long* round_ns;       // NULL, or device telemetry: round_ns[k-1] = %globaltimer when
                                        // round k's pass starts (persistent launch; round_cap + 1 entries)
    int32_t round_cap;
};

// ------------------------------------------------------------ helpers

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// L2 eviction policies: adjacency is streamed and should not push the color
// arrays (gathered at random) out of L2.
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

#ifndef GC_L1_COLORS
#define GC_L1_COLORS 1
#endif

// Adjacency / active-list entry.  colidx is read-only for the whole call;
// an active list is written in one round and read in the next.  Rounds are
// separated by kernel boundaries or by grid_barrier, whose fences make
// earlier rounds' writes visible to cached loads after it (the ordering a
// grid-wide synchronisation gives), so these loads may use L1.
__device__ __forceinline__ int32_t ld_row(const int32_t* a, uint64_t pol) {
    int32_t r;
#if GC_L1_COLORS
    asm volatile("ld.global.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(a), "l"(pol));
#else
    asm volatile("ld.global.cg.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(a), "l"(pol));
#endif
    return r;
}
__device__ __forceinline__ int32_t ld_adj(const int32_t* a, uint64_t pol) {
    int32_t r;
    asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(a), "l"(pol));
    return r;
}

// Color word: written in earlier rounds (visible after the round boundary,
// as above) and kept in L2 (evict_last); the few high-degree vertices that
// most gathers hit stay in each SM's L1.  Within a round a word may gain its
// settled flag while others read it; a copy without the flag is still the
// right color, and the flag is seen a round later.
__device__ __forceinline__ uint16_t ld_color(const uint16_t* a, uint64_t pol) {
    uint16_t r;
#if GC_L1_COLORS
    asm volatile("ld.global.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(r) : "l"(a), "l"(pol));
#else
    asm volatile("ld.global.cg.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(r) : "l"(a), "l"(pol));
#endif
    return r;
}
__device__ __forceinline__ int32_t ld_color(const int32_t* a, uint64_t pol) {
    int32_t r;
#if GC_L1_COLORS
    asm volatile("ld.global.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(a), "l"(pol));
#else
    asm volatile("ld.global.cg.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(a), "l"(pol));
#endif
    return r;
}

// With a priority array, active lists written from round 2 on carry, in bit
// 31 of each entry (ids are below 2^31), whether that neighbour precedes the
// list's vertex.  The order never changes, so it is computed once (round 2)
// and later rounds test a bit instead of gathering two priority keys per
// equally colored neighbour.  Under index priority the test is one compare
// and the lists carry plain ids.
constexpr uint32_t kPrecBit = 0x80000000u;
__device__ __forceinline__ int32_t entry_id(int32_t x) { return x & 0x7fffffff; }

// w precedes v: (prio[w], w) < (prio[v], v); pv = prio[v] (ignored if no prio).
__device__ __forceinline__ bool precedes(const uint32_t* __restrict__ prio, int32_t w, int32_t v,
                                         uint32_t pv) {
    if (prio) {
        const uint32_t pw = __ldg(prio + w);
        if (pw != pv) return pw < pv;
    }
    return w < v;
}

// Append a worklist entry (if flag) with one atomic per warp.  All lanes call it.
__device__ __forceinline__ void warp_append(bool flag, int4 e, int4* list, unsigned* cnt) {
    const unsigned ballot = __ballot_sync(kFull, flag);
    if (ballot == 0) return;
    const unsigned lane = lane_id();
    const int leader = __ffs(ballot) - 1;
    unsigned base = 0;
    if ((int)lane == leader) base = atomicAdd(cnt, (unsigned)__popc(ballot));
    base = __shfl_sync(kFull, base, leader);
    if (flag) list[base + __popc(ballot & ((1u << lane) - 1u))] = e;
}

__device__ __forceinline__ void warp_append_i32(bool flag, int32_t v, int32_t* list, unsigned* cnt) {
    const unsigned ballot = __ballot_sync(kFull, flag);
    if (ballot == 0) return;
    const unsigned lane = lane_id();
    const int leader = __ffs(ballot) - 1;
    unsigned base = 0;
    if ((int)lane == leader) base = atomicAdd(cnt, (unsigned)__popc(ballot));
    base = __shfl_sync(kFull, base, leader);
    if (flag) list[base + __popc(ballot & ((1u << lane) - 1u))] = v;
}

// Where the next round's worklists go.
struct NextLists {
    int4* S; int4* M; int4* H; int32_t* Hc; int32_t* O;
    RoundCounts* cnt;  // the next round's counts
    int32_t s_max, m_max;
};

__device__ __forceinline__ int bin_of(int32_t len, int32_t s_max, int32_t m_max) {
    return len <= s_max ? kBinS : (len <= m_max ? kBinM : kBinH);
}

// Append H-bin entry e (lane 0's copy) to the next round and hand it its
// chunks.  Called by all lanes of a warp.
__device__ __forceinline__ void warp_append_hub(const NextLists& nl, int4 e) {
    const unsigned nch = (unsigned)(e.z + kChunk - 1) / kChunk;
    unsigned pos = 0, c0 = 0;
    if (lane_id() == 0) {
        const unsigned long long old = atomicAdd(&nl.cnt->hc, ((unsigned long long)nch << 32) | 1ull);
        pos = hub_count(old);
        c0 = hub_chunks(old);
        nl.H[pos] = e;
        nl.Hc[pos] = (int32_t)c0;
    }
    pos = __shfl_sync(kFull, pos, 0);
    c0 = __shfl_sync(kFull, c0, 0);
    for (unsigned j = lane_id(); j < nch; j += 32) nl.O[c0 + j] = (int32_t)pos;
}

// Append the H-bin entries of the lanes whose flag is set, with one atomic for
// all of them (their chunks get consecutive ranges).  Called by all lanes.
__device__ __forceinline__ void warp_append_hubs(const NextLists& nl, bool flag, int4 e) {
    const unsigned ballot = __ballot_sync(kFull, flag);
    if (ballot == 0) return;
    const unsigned lane = lane_id();
    const unsigned nch = flag ? (unsigned)(e.z + kChunk - 1) / kChunk : 0u;
    unsigned incl = nch;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned x = __shfl_up_sync(kFull, incl, o);
        if ((int)lane >= o) incl += x;
    }
    const unsigned total = __shfl_sync(kFull, incl, 31);
    unsigned long long old = 0;
    if (lane == 0) old = atomicAdd(&nl.cnt->hc, ((unsigned long long)total << 32) | (unsigned long long)__popc(ballot));
    old = __shfl_sync(kFull, old, 0);
    if (flag) {
        const unsigned pos = hub_count(old) + (unsigned)__popc(ballot & ((1u << lane) - 1u));
        const unsigned c0 = hub_chunks(old) + incl - nch;
        nl.H[pos] = e;
        nl.Hc[pos] = (int32_t)c0;
        for (unsigned j = 0; j < nch; ++j) nl.O[c0 + j] = (int32_t)pos;
    }
}

// Append one entry held by lane 0 (any bin).  Called by all lanes of a warp.
__device__ __forceinline__ void warp_append_one(const NextLists& nl, int4 e) {
    const int bin = bin_of(e.z, nl.s_max, nl.m_max);
    if (bin == kBinH) {
        warp_append_hub(nl, e);
    } else if (lane_id() == 0) {
        int4* list = bin == kBinM ? nl.M : nl.S;
        list[atomicAdd(bin == kBinM ? &nl.cnt->m : &nl.cnt->s, 1u)] = e;
    }
}

// Bits of colors base+1 .. base+256 seen by one lane.
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
    // OR over the warp; every lane receives word `lane & 7` of the result.
    __device__ __forceinline__ uint32_t warp_reduce_word() const {
        const uint32_t r0 = __reduce_or_sync(kFull, (uint32_t)w0);
        const uint32_t r1 = __reduce_or_sync(kFull, (uint32_t)(w0 >> 32));
        const uint32_t r2 = __reduce_or_sync(kFull, (uint32_t)w1);
        const uint32_t r3 = __reduce_or_sync(kFull, (uint32_t)(w1 >> 32));
        const uint32_t r4 = __reduce_or_sync(kFull, (uint32_t)w2);
        const uint32_t r5 = __reduce_or_sync(kFull, (uint32_t)(w2 >> 32));
        const uint32_t r6 = __reduce_or_sync(kFull, (uint32_t)w3);
        const uint32_t r7 = __reduce_or_sync(kFull, (uint32_t)(w3 >> 32));
        const unsigned q = lane_id() & 7u;
        uint32_t r = r0;
        r = q == 1u ? r1 : r;
        r = q == 2u ? r2 : r;
        r = q == 3u ? r3 : r;
        r = q == 4u ? r4 : r;
        r = q == 5u ? r5 : r;
        r = q == 6u ? r6 : r;
        r = q == 7u ? r7 : r;
        return r;
    }
};

// First clear bit of the 256-bit window whose word q sits in lanes with
// (lane & 7) == q; -1 if all set.  All lanes call it and get the same value.
__device__ __forceinline__ int window_first_clear(uint32_t word) {
    const unsigned notfull = __ballot_sync(kFull, lane_id() < 8u && word != 0xffffffffu);
    if (notfull == 0) return -1;
    const int q = __ffs(notfull) - 1;
    const uint32_t wq = __shfl_sync(kFull, word, q);
    return q * 32 + __ffs(~wq) - 1;
}

// First fit beyond the first window: rescan v's whole original row (settled
// neighbours were dropped from the active list) for windows base+1 .. until
// one has a free color.  Terminates: a full window of 256 colors needs 256
// more neighbours, and first fit never exceeds degree + 1.
template <typename T>
__device__ __forceinline__ unsigned rescan_first_fit(const int32_t* __restrict__ rowptr,
                                                     const int32_t* __restrict__ colidx, const T* Xc,
                                                     int32_t v) {
    const int32_t b = __ldg(rowptr + v), e = __ldg(rowptr + v + 1);
    for (unsigned base = 256u;; base += 256u) {
        Mask256 m;
        m.clear();
        for (int32_t i = b + (int32_t)lane_id(); i < e; i += 32)
            m.set(word_color(__ldcg(Xc + __ldg(colidx + i))) - 1u - base);
        const int ff = window_first_clear(m.warp_reduce_word());
        if (ff >= 0) return base + (unsigned)ff + 1u;
    }
}

// --------------------------------------------------- bounded grid barrier

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// All blocks of a cooperative launch meet here.  Returns false (and sets
// status = timeout) if the wait gave up; the caller then leaves the loop.
__device__ __forceinline__ bool grid_barrier(RoundState* st, unsigned max_polls) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned* vgen = &st->bar_gen;
        const unsigned gen = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(&st->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            // every block's writes of this round are in: the status they leave
            // is the one all blocks act on after the barrier (a block that is
            // already in the next round may change st->status meanwhile)
            __threadfence();
            st->status_at_barrier = *((volatile int*)&st->status);
            atomicExch(&st->bar_count, 0u);
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            const unsigned long long t0 = globaltimer_ns();
            unsigned polls = 0, nap = 32;
            while (*vgen == gen) {
                __nanosleep(nap);
                nap = nap < 256 ? nap * 2 : 256;
                if (++polls >= max_polls || globaltimer_ns() - t0 > kBarrierTimeoutNs) {
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
    const int m = __reduce_max_sync(kFull, maxc);
    if (lane_id() == 0 && m > 0) atomicMax(&st->max_color, m);
}

// Add a warp's share of round r's read volume to the round counter
// (rc[r % 3].vol) and to the telemetry (round_vol[r-1]).
__device__ __forceinline__ void fold_volume(RoundState* st, unsigned long long* round_vol, int32_t cap, int r,
                                            unsigned vol) {
    const unsigned s = __reduce_add_sync(kFull, vol);
    if (lane_id() == 0 && s) {
        atomicAdd(&st->rc[r % 3].vol, s);
        if (r - 1 < cap) atomicAdd(&round_vol[r - 1], (unsigned long long)s);
    }
}

// ------------------------------------------------------------ setup scan

// Degree statistics: max degree, list capacities, hub chunks, rowptr checks.
__global__ void stats_kernel(const int32_t* __restrict__ rowptr, int32_t n, int32_t s_max,
                             int32_t m_max, Stats* s) {
    int mx = 0, bad = 0;
    unsigned c0 = 0, c1 = 0, c2 = 0, df = 0;
    unsigned long long ch = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = __ldg(rowptr + v + 1) - __ldg(rowptr + v);
        if (d < 0) { bad = 1; continue; }
        mx = max(mx, d);
        c0 += d >= 1;
        c1 += d > s_max;
        c2 += d > m_max;
        df += d > kPass1Flat;
        if (d > m_max) ch += (unsigned long long)((d + kChunk - 1) / kChunk);
    }
    mx = __reduce_max_sync(kFull, mx);
    bad = __reduce_or_sync(kFull, (unsigned)bad);
    c0 = __reduce_add_sync(kFull, c0);
    c1 = __reduce_add_sync(kFull, c1);
    c2 = __reduce_add_sync(kFull, c2);
    df = __reduce_add_sync(kFull, df);
    if (lane_id() == 0) {
        atomicMax(&s->max_degree, mx);
        if (bad) s->bad = 1;
        if (c0) atomicAdd(&s->cap[0], c0);
        if (c1) atomicAdd(&s->cap[1], c1);
        if (c2) atomicAdd(&s->cap[2], c2);
        if (df) atomicAdd(&s->defer, df);
    }
    for (int o = 16; o > 0; o >>= 1) ch += __shfl_xor_sync(kFull, ch, o);
    if (lane_id() == 0 && ch) atomicAdd(&s->hub_chunks, ch);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (__ldg(rowptr) != 0) s->bad = 1;
        s->nnz = __ldg(rowptr + n);
    }
}

// ------------------------------------------------------------- pass 1

// Outcome of round 1 for v: C_2[v] = 2 if it conflicts (then it joins U_2),
// else v keeps color 1 for good (flagged in both buffers).
template <typename T>
__device__ __forceinline__ void pass1_write(const Params<T>& p, int32_t v, bool conflict, int& maxc) {
    if (conflict) {
        p.X0[v] = (T)2;
    } else {
        const T one = (T)(1u | Word<T>::kFlag);
        p.X0[v] = one;
        p.X1[v] = one;
        p.colors_out[v] = 1;
        if (p.settle_round) p.settle_round[v] = 1;
        maxc = 1;
    }
}

template <typename T>
__device__ __forceinline__ NextLists pass1_next(const Params<T>& p) {
    NextLists nl;
    nl.S = p.SA; nl.M = p.MA; nl.H = p.HA; nl.Hc = p.HcA; nl.O = p.OA;
    nl.cnt = &p.st->rc[2];
    nl.s_max = p.s_max;
    nl.m_max = p.m_max;
    return nl;
}

// Round 1 on 32 consecutive vertices per task, over vertices [v_begin, v_end)
// (v_begin a multiple of 32; the host may launch it per range as the input
// arrives).  Their adjacency entries
// (rows of degree <= kPass1Flat) are read as one flat, coalesced range;
// lane l of batch u handles flat entry F0 + 32u + l, finds its row from the
// batch's row starts (an OR-reduction over the warp and a table of the
// non-empty rows' lanes), and marks the row in shared memory when the entry
// precedes it.  Longer rows go to pass1_long_kernel.
template <typename T>
__global__ void __launch_bounds__(256, 5) pass1_kernel(Params<T> p, int32_t v_begin, int32_t v_end) {
    // a warp takes two tasks (t, t + W) at a time and appends their S and M
    // entries with one atomic per bin: every task appends to both, and the
    // counters' lines were the busiest of the L2 in this kernel
    constexpr int NT = 2;
    struct P1Smem {
        uint8_t lane_of[32];  // lane of the i-th non-empty row
        unsigned hit[32];     // row r has a preceding neighbour
    };
    __shared__ P1Smem s_p1[8];
    const unsigned wib = threadIdx.x >> 5;
    const unsigned lane = lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t ntasks = ((int64_t)v_end - v_begin + 31) / 32;
    const NextLists nl = pass1_next(p);
    const uint64_t pol_adj = policy_evict_first();
    int maxc = 0;
    unsigned vol = 0;
    for (int64_t t0 = gw; t0 < ntasks; t0 += W * NT) {
        int4 ev[NT];
        bool fS[NT], fM[NT];
#pragma unroll
        for (int jt = 0; jt < NT; ++jt) {
            const int64_t t = t0 + (int64_t)jt * W;
            const int64_t vv = (int64_t)v_begin + t * 32 + lane;
            const bool valid = t < ntasks && vv < v_end;
            const int32_t v = valid ? (int32_t)vv : 0;
            const int32_t b = valid ? __ldg(p.rowptr + v) : 0;
            const int32_t d = valid ? __ldg(p.rowptr + v + 1) - b : 0;
            const bool longrow = d > kPass1Flat;
            const int32_t eff = longrow ? 0 : d;
            const uint32_t pv = (p.prio && valid) ? __ldg(p.prio + v) : 0u;
            int32_t incl = eff;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t x = __shfl_up_sync(kFull, incl, o);
                if ((int)lane >= o) incl += x;
            }
            const int32_t off = incl - eff;
            const int32_t D = __shfl_sync(kFull, incl, 31);
            // entry f's row: the last non-empty row starting at or before f, found
            // from the batch's row starts (one OR-reduction) and a lane table
            const unsigned nz = __ballot_sync(kFull, eff > 0);
            if (eff > 0) s_p1[wib].lane_of[__popc(nz & ((1u << lane) - 1u))] = (uint8_t)lane;
            s_p1[wib].hit[lane] = 0u;
            const int32_t b_off = b - off;  // entry f of this row sits at colidx[b_off + f]
            __syncwarp();
            for (int32_t F0 = 0; F0 < D; F0 += 32 * 4) {
                int32_t w[4], own[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int32_t base = F0 + 32 * u;
                    const int32_t f = base + (int32_t)lane;
                    const int32_t rel = off - base;
                    const unsigned before = __popc(__ballot_sync(kFull, eff > 0 && rel < 0));
                    const unsigned starts = __reduce_or_sync(kFull, (eff > 0 && rel >= 0 && rel < 32) ? (1u << rel) : 0u);
                    const unsigned rank = before + __popc(starts & (0xffffffffu >> (31 - lane)));
                    const int o = (f < D && rank > 0) ? (int)s_p1[wib].lane_of[rank - 1] : 0;
                    own[u] = o;
                    const int32_t rb = __shfl_sync(kFull, b_off, o);
                    w[u] = f < D ? ld_adj(p.colidx + rb + f, pol_adj) : 0;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int32_t f = F0 + 32 * u + (int32_t)lane;
                    const uint32_t opv = __shfl_sync(kFull, pv, own[u]);
                    if (f < D && precedes(p.prio, w[u], (int32_t)(v_begin + t * 32 + own[u]), opv))
                        s_p1[wib].hit[own[u]] = 1u;
                }
            }
            __syncwarp();
            const bool hit = s_p1[wib].hit[lane] != 0u;
            if (valid && !longrow) {
                pass1_write(p, v, hit, maxc);
                if (hit) vol += (unsigned)d;
            }
            const int bin = bin_of(d, p.s_max, p.m_max);
            const bool go = valid && !longrow && hit;
            ev[jt] = make_int4(v, b, d, d);
            fS[jt] = go && bin == kBinS;
            fM[jt] = go && bin == kBinM;
            // hubs that stayed in the flat range (m_max < d <= kPass1Flat)
            unsigned hubs = __ballot_sync(kFull, go && bin == kBinH);
            while (hubs) {
                const int j = __ffs(hubs) - 1;
                hubs &= hubs - 1;
                const int32_t dj = __shfl_sync(kFull, d, j);
                warp_append_hub(nl, make_int4(__shfl_sync(kFull, v, j), __shfl_sync(kFull, b, j), dj, dj));
            }
            warp_append_i32(valid && longrow, v, p.defer, &p.st->defer_cnt);
        }
        // the S and M entries of these NT tasks, one atomic per bin
#pragma unroll
        for (int bin = 0; bin < 2; ++bin) {
            unsigned bal[NT], n = 0;
#pragma unroll
            for (int jt = 0; jt < NT; ++jt) {
                bal[jt] = __ballot_sync(kFull, bin == 0 ? fS[jt] : fM[jt]);
                n += __popc(bal[jt]);
            }
            if (n == 0) continue;
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(bin == 0 ? &nl.cnt->s : &nl.cnt->m, n);
            base = __shfl_sync(kFull, base, 0);
            int4* const list = bin == 0 ? nl.S : nl.M;
#pragma unroll
            for (int jt = 0; jt < NT; ++jt) {
                if ((bal[jt] >> lane) & 1u) list[base + __popc(bal[jt] & ((1u << lane) - 1u))] = ev[jt];
                base += __popc(bal[jt]);
            }
        }
    }
    fold_max_color(p.st, maxc);
    fold_volume(p.st, p.round_vol, p.round_cap, 2, vol);
}

// Round 1 for rows longer than kPass1Flat: a warp takes up to 32 of them (one
// per lane; fewer when there are not many, so that every warp has some),
// reads them one after another, 128 entries per step, stopping at the first
// preceding neighbour, and appends the conflicting ones (all H bin: longer
// than kPass1Flat >= m_max) with one atomic.
template <typename T>
__global__ void __launch_bounds__(256) pass1_long_kernel(Params<T> p) {
    const unsigned lane = lane_id();
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const unsigned nd = __ldcg(&p.st->defer_cnt);
    const NextLists nl = pass1_next(p);
    const uint64_t pol_adj = policy_evict_first();
    int maxc = 0;
    unsigned vol = 0;
    const int64_t R = max((int64_t)1, min((int64_t)32, ((int64_t)nd + W - 1) / W));  // rows per warp
    for (int64_t t0 = gw * R; t0 < nd; t0 += W * R) {
        const int64_t i = t0 + lane;
        const bool valid = lane < R && i < nd;
        const int32_t v = valid ? __ldcg(p.defer + i) : 0;
        const int32_t b = valid ? __ldg(p.rowptr + v) : 0, e = valid ? __ldg(p.rowptr + v + 1) : 0;
        const uint32_t pv = (p.prio && valid) ? __ldg(p.prio + v) : 0u;
        bool mine = false;
        const int rows = (int)min(R, (int64_t)nd - t0);
        for (int j = 0; j < rows; ++j) {
            const int32_t vj = __shfl_sync(kFull, v, j), bj = __shfl_sync(kFull, b, j), ej = __shfl_sync(kFull, e, j);
            const uint32_t pvj = __shfl_sync(kFull, pv, j);
            bool conflict = false;
            for (int32_t c = bj; c < ej && !conflict; c += 128) {
                int32_t w[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int32_t x = c + 32 * u + (int32_t)lane;
                    w[u] = x < ej ? ld_adj(p.colidx + x, pol_adj) : -1;
                }
                bool h = false;
#pragma unroll
                for (int u = 0; u < 4; ++u) h |= w[u] >= 0 && precedes(p.prio, w[u], vj, pvj);
                conflict = __any_sync(kFull, h);
            }
            if ((int)lane == j) mine = conflict;
        }
        if (valid) {
            pass1_write(p, v, mine, maxc);
            if (mine) vol += (unsigned)(e - b);
        }
        warp_append_hubs(nl, valid && mine, make_int4(v, b, e - b, e - b));
    }
    fold_max_color(p.st, maxc);
    fold_volume(p.st, p.round_vol, p.round_cap, 2, vol);
}

// ------------------------------------------------- fused pass, k >= 2

template <typename T>
struct PassIO {
    const T* Xc;            // C_k (flagged once settled)
    T* Xcw;                 // the same array, for setting the settled flag
    T* Xn;                  // receives C_{k+1}
    int k;                  // the round whose Phase 2 this pass runs
    const int32_t* rin;     // active lists read this round (colidx in round 2)
    int32_t* rout;          // active lists written for the next round
    bool first;             // round 2: no static masks yet
    const int4* S; const int4* M; const int4* H; const int32_t* Hc; const int32_t* O;
    NextLists next;
    uint64_t pol_row, pol_col;
};

template <typename T>
__device__ __forceinline__ PassIO<T> pass_io(const Params<T>& p, int k) {
    PassIO<T> io;
    const bool odd = (k & 1) != 0;
    io.Xc = odd ? p.X1 : p.X0;
    io.Xcw = odd ? p.X1 : p.X0;
    io.Xn = odd ? p.X0 : p.X1;
    io.first = k == 2;
    io.k = k;
    io.rin = k == 2 ? p.colidx : (odd ? p.act1 : p.act0);
    io.rout = odd ? p.act0 : p.act1;
    io.S = odd ? p.SB : p.SA;
    io.M = odd ? p.MB : p.MA;
    io.H = odd ? p.HB : p.HA;
    io.Hc = odd ? p.HcB : p.HcA;
    io.O = odd ? p.OB : p.OA;
    io.next.S = odd ? p.SA : p.SB;
    io.next.M = odd ? p.MA : p.MB;
    io.next.H = odd ? p.HA : p.HB;
    io.next.Hc = odd ? p.HcA : p.HcB;
    io.next.O = odd ? p.OA : p.OB;
    io.next.cnt = &p.st->rc[(k + 1) % 3];
    io.next.s_max = p.s_max;
    io.next.m_max = p.m_max;
    io.pol_row = policy_evict_first();
    io.pol_col = policy_evict_last();
    return io;
}

// v settles with color cv: flag it in both buffers, publish it.
template <typename T>
__device__ __forceinline__ void settle(const Params<T>& p, const PassIO<T>& io, int32_t v, uint32_t cv) {
    const T word = (T)(cv | Word<T>::kFlag);
    io.Xn[v] = word;
    io.Xcw[v] = word;
    p.colors_out[v] = (int32_t)cv;
    if (p.settle_round) p.settle_round[v] = io.k;
}

// v takes color c in round k+1.
template <typename T>
__device__ __forceinline__ void recolor(const Params<T>& p, const PassIO<T>& io, int32_t v, uint32_t c) {
    if (c >= p.color_limit) atomicExch(&p.st->status, kStatusColorOverflow);
    io.Xn[v] = (T)(c & (Word<T>::kFlag - 1u));
}

// What a warp needs to start a task.  Loaded one task ahead.
struct TaskHead {
    int4 e;       // {vertex, row start, active length, degree}; x < 0 marks an empty slot
    int32_t pos;  // H chunk: worklist position of its vertex
    int32_t lo;   // H chunk: first entry of the chunk
};

template <typename T>
__device__ __forceinline__ TaskHead load_head(const PassIO<T>& io, unsigned t, unsigned nS,
                                              unsigned nM, unsigned nHC, unsigned tM, unsigned mpt,
                                              unsigned spt) {
    TaskHead h;
    h.pos = 0;
    h.lo = 0;
    if (t < nHC) {
        h.pos = __ldcg(io.O + t);
        h.e = __ldcg(io.H + h.pos);
        h.lo = h.e.y + ((int32_t)t - __ldcg(io.Hc + h.pos)) * kChunk;
    } else if (t - nHC < tM) {
        const unsigned i = (t - nHC) * mpt + lane_id();
        h.e = (lane_id() < mpt && i < nM) ? __ldcg(io.M + i) : make_int4(-1, 0, 0, 0);
    } else {
        const unsigned i = (t - nHC - tM) * spt + lane_id();
        h.e = (lane_id() < spt && i < nS) ? __ldcg(io.S + i) : make_int4(-1, 0, 0, 0);
    }
    return h;
}

// Shared memory of one warp for a flat task.
// The color windows are stored word-major ([word q][lane]), so the 32 lanes
// touching word q of their own vertex's window hit 32 different banks.
struct FlatSmem {
    uint32_t stat[8 * 32];  // per entry vertex: static mask (+ colors settled this round)
    uint32_t dyn[8 * 32];   // per entry vertex: colors of unsettled neighbours this round
    uint32_t conf;          // per entry vertex: conflict flag
    uint32_t lane_of[32];   // lane of the i-th non-empty row
    int32_t vid[32];        // vertex of each lane
};

// Ask L1 for the line holding a (list entries read soon by this warp).
__device__ __forceinline__ void prefetch_l1(const void* a) {
    asm volatile("prefetch.global.L1 [%0];" :: "l"(a));
}

// Stores of the next round's active lists and static masks: read once, in
// the next round, so evicted first.
__device__ __forceinline__ void st_stream(int32_t* a, int32_t x, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.s32 [%0], %1, %2;" :: "l"(a), "r"(x), "l"(pol) : "memory");
}

// S and M bins: up to 32 worklist entries per task, one per lane.  Their
// active lists are walked as one flat range in batches of 32 entries (lane
// l of batch u takes flat entry F0 + 32u + l), so every lane has an entry in
// every batch whatever the lengths are.  The row owning an entry is found
// from the batch's row starts: a row that starts inside the batch sets the
// bit of its first lane (one OR-reduction over the warp), and an entry's
// row is the last one started at or before it, counted among the non-empty
// rows (a 32-entry table maps that count to the row's lane).  Each entry ORs its neighbour's color into
// its vertex's window in shared memory, flags a conflict, and, if the
// neighbour has not settled, is copied to the next round's list at the
// vertex's running write position.  Afterwards each lane decides its own
// vertex.
template <typename T, bool P>  // P: a priority array is given
__device__ __forceinline__ void flat_task(const Params<T>& p, const PassIO<T>& io, int4 en,
                                          FlatSmem& sm, int& maxc, unsigned& vol) {
    const unsigned lane = lane_id();
    const bool valid = en.x >= 0;
    const int32_t v = valid ? en.x : 0;
    const int32_t b = en.y;
    const int32_t len = valid ? en.z : 0;
    const uint32_t cv = valid ? word_color(ld_color(io.Xc + v, io.pol_col)) : 0u;
    // static mask of v (none yet in round 2)
    if (valid && !io.first) {
        const uint4* src = reinterpret_cast<const uint4*>(p.stat + (size_t)v * 8);
        const uint4 a = __ldcg(src), c = __ldcg(src + 1);
        sm.stat[0 * 32 + lane] = a.x; sm.stat[1 * 32 + lane] = a.y;
        sm.stat[2 * 32 + lane] = a.z; sm.stat[3 * 32 + lane] = a.w;
        sm.stat[4 * 32 + lane] = c.x; sm.stat[5 * 32 + lane] = c.y;
        sm.stat[6 * 32 + lane] = c.z; sm.stat[7 * 32 + lane] = c.w;
    } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) sm.stat[q * 32 + lane] = 0u;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) sm.dyn[q * 32 + lane] = 0u;
    if (lane == 0) sm.conf = 0u;
    int32_t incl = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t x = __shfl_up_sync(kFull, incl, o);
        if ((int)lane >= o) incl += x;
    }
    const int32_t off = incl - len;
    const int32_t D = __shfl_sync(kFull, incl, 31);
    const unsigned nz = __ballot_sync(kFull, len > 0);  // rows that own entries
    if (len > 0) sm.lane_of[__popc(nz & ((1u << lane) - 1u))] = lane;
    sm.vid[lane] = v;
    int32_t kept = 0;  // entries of this lane's vertex written for the next round
    __syncwarp();
    const int32_t b_off = b - off;  // row start minus flat offset: entry f of this row is at b_off + f
    for (int32_t F0 = 0; F0 < D; F0 += 32 * kFlatBatches) {
        int32_t w[kFlatBatches], own[kFlatBatches], seglo[kFlatBatches];
#pragma unroll
        for (int u = 0; u < kFlatBatches; ++u) {
            const int32_t base = F0 + 32 * u;
            const int32_t f = base + (int32_t)lane;
            // rows started before this batch, and the starts inside it
            const int32_t rel = off - base;
            const unsigned before = __popc(__ballot_sync(kFull, len > 0 && rel < 0));
            const unsigned starts = __reduce_or_sync(kFull, (len > 0 && rel >= 0 && rel < 32) ? (1u << rel) : 0u);
            const unsigned upto = starts & (0xffffffffu >> (31 - lane));
            const unsigned rank = before + __popc(upto);
            const int o = (f < D && rank > 0) ? (int)sm.lane_of[rank - 1] : 0;
            own[u] = o;
            // first lane of my owner's entries in this batch: the last row start at or
            // before this lane, or 0 if the row began in an earlier batch
            seglo[u] = upto ? 31 - __clz(upto) : 0;
            const int32_t rb = __shfl_sync(kFull, b_off, o);
            w[u] = f < D ? ld_row(io.rin + rb + f, io.pol_row) : 0;
        }
        T c[kFlatBatches];
#pragma unroll
        for (int u = 0; u < kFlatBatches; ++u) {
            const int32_t f = F0 + 32 * u + (int32_t)lane;
            c[u] = f < D ? ld_color(io.Xc + (P ? entry_id(w[u]) : w[u]), io.pol_col) : (T)0;
        }
#pragma unroll
        for (int u = 0; u < kFlatBatches; ++u) {
            const int32_t base = F0 + 32 * u;
            const int32_t f = base + (int32_t)lane;
            const int o = own[u];
            const uint32_t ocv = __shfl_sync(kFull, cv, o);
            const int32_t wbase = __shfl_sync(kFull, b + kept, o);  // next free slot of the owner's list
            const bool in = f < D;
            const uint32_t col = word_color(c[u]);
            const bool settled = in && word_settled(c[u]);
            // does this neighbour precede its owner?  Round 2 works it out (for the
            // conflict test and for the bit of every entry it keeps); later rounds read
            // the bit.
            const int32_t wid = P ? entry_id(w[u]) : w[u];
            bool pre = false;
            if constexpr (!P) {
                if (in && col == ocv) pre = wid < sm.vid[o];
            } else if (in && (col == ocv || (io.first && !settled))) {
                if (io.first) {
                    const int32_t ov = sm.vid[o];
                    pre = precedes(p.prio, wid, ov, __ldg(p.prio + ov));
                } else {
                    pre = w[u] < 0;
                }
            }
            if (in && col == ocv && pre) atomicOr(&sm.conf, 1u << o);
            {
                const unsigned idx = col - 1u;
                if (in && idx < 256u)
                    atomicOr(settled ? &sm.stat[(idx >> 5) * 32 + o] : &sm.dyn[(idx >> 5) * 32 + o],
                             1u << (idx & 31u));
            }
            // survivors: copy to the next round's list, in order within each vertex
            const bool keep = in && !settled;
            const unsigned kb = __ballot_sync(kFull, keep);
            const unsigned below = kb & ((1u << lane) - 1u) & ~((1u << seglo[u]) - 1u);
            if (keep)
                st_stream(io.rout + wbase + __popc(below),
                          (P && io.first) ? (int32_t)((uint32_t)wid | (pre ? kPrecBit : 0u)) : w[u],
                          io.pol_row);
            // my vertex's lanes in this batch: [lo, hi)
            const int32_t lo = max(0, min(32, off - base));
            const int32_t hi = max(0, min(32, off + len - base));
            if (hi > lo) {
                const unsigned bits = hi - lo == 32 ? kFull : ((1u << (hi - lo)) - 1u);
                kept += __popc((kb >> lo) & bits);
            }
        }
    }
    __syncwarp();
    const bool conflict = valid && ((sm.conf >> lane) & 1u);
    uint32_t color = 0;
    bool rescan = false;
    if (conflict) {
        int ff = -1;
#pragma unroll
        for (int q = 7; q >= 0; --q) {
            const uint32_t word = sm.stat[q * 32 + lane] | sm.dyn[q * 32 + lane];
            if (word != 0xffffffffu) ff = q * 32 + __ffs(~word) - 1;
        }
        if (ff >= 0) color = (uint32_t)ff + 1u;
        else rescan = true;
    }
    unsigned need = __ballot_sync(kFull, rescan);
    while (need) {
        const int j = __ffs(need) - 1;
        need &= need - 1;
        const uint32_t cj = rescan_first_fit(p.rowptr, p.colidx, io.Xc, __shfl_sync(kFull, v, j));
        if ((int)lane == j) color = cj;
    }
    if (valid) {
        if (conflict) {
            recolor(p, io, v, color);
            vol += (unsigned)kept;
            uint4* dst = reinterpret_cast<uint4*>(p.stat + (size_t)v * 8);
            dst[0] = make_uint4(sm.stat[0 * 32 + lane], sm.stat[1 * 32 + lane],
                                sm.stat[2 * 32 + lane], sm.stat[3 * 32 + lane]);
            dst[1] = make_uint4(sm.stat[4 * 32 + lane], sm.stat[5 * 32 + lane],
                                sm.stat[6 * 32 + lane], sm.stat[7 * 32 + lane]);
        } else {
            settle(p, io, v, cv);
            maxc = max(maxc, (int)cv);
        }
    }
    // next round: same row start, `kept` active entries; the bin may shrink
    const int4 ne = make_int4(v, b, kept, en.w);
    const int nb = bin_of(kept, p.s_max, p.m_max);
    warp_append(conflict && nb == kBinS, ne, io.next.S, &io.next.cnt->s);
    warp_append(conflict && nb == kBinM, ne, io.next.M, &io.next.cnt->m);
    __syncwarp();
}

// M bin: up to kMedPerTask worklist entries per task (lane i holds entry i), taken
// one vertex at a time by the whole warp: lane l reads entries l, l + 32, ...
// of the vertex's active list, four batches of 32 in flight.  Colors 1..64
// collect in per-lane registers (all neighbours, and those found settled)
// and are OR-reduced once per vertex; colors 65..256 go to the warp's shared
// windows, where no two vertices meet.  So the lanes never contend on one
// shared word, which the flat walk does when most of a batch belongs to one
// long list.  The decisions stay in the lane of their entry, and the task
// appends its conflicting vertices to the next round with one atomic per
// bin.
template <typename T, bool P>  // P: a priority array is given
__device__ __forceinline__ void vertex_task(const Params<T>& p, const PassIO<T>& io, int4 en,
                                            FlatSmem& sm, int& maxc, unsigned& vol) {
    constexpr int kB = 4;  // batches in flight
    const unsigned lane = lane_id();
    const bool first = io.first;
    bool my_conflict = false;
    int32_t my_kept = 0;
    unsigned todo = __ballot_sync(kFull, en.x >= 0);
    while (todo) {
        const int j = __ffs(todo) - 1;
        todo &= todo - 1;
        const int32_t v = __shfl_sync(kFull, en.x, j);
        const int32_t b = __shfl_sync(kFull, en.y, j);
        const int32_t len = __shfl_sync(kFull, en.z, j);
        // the next vertex's list comes into L1 while this one is read (lanes 0..8:
        // one 128-byte line each, the last one for the end of the list)
        if (todo) {
            const int jn = __ffs(todo) - 1;
            const int32_t bn = __shfl_sync(kFull, en.y, jn), ln = __shfl_sync(kFull, en.z, jn);
            if (lane < 8u && (int32_t)lane * 32 < ln) prefetch_l1(io.rin + bn + 32 * lane);
            else if (lane == 8u) prefetch_l1(io.rin + bn + ln - 1);
        }
        const uint32_t cv = word_color(ld_color(io.Xc + v, io.pol_col));
        const uint32_t pv = (P && first) ? __ldg(p.prio + v) : 0u;
        // v's static mask, word `lane` (read now, used after the list)
        const uint32_t old = (lane < 8u && !first) ? __ldcg(p.stat + (size_t)v * 8 + lane) : 0u;
        if (lane < 8u) { sm.dyn[lane] = 0u; sm.stat[lane] = 0u; }
        __syncwarp();
        uint32_t rd0 = 0u, rs0 = 0u, rd1 = 0u, rs1 = 0u;  // this lane's colors 1..64 (all, settled)
        bool conflict = false;
        int32_t kept = 0;
        for (int32_t base = 0; base < len; base += 32 * kB) {
            int32_t w[kB];
            T c[kB];
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int32_t i = base + 32 * u + (int32_t)lane;
                w[u] = i < len ? ld_row(io.rin + b + i, io.pol_row) : 0;
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int32_t i = base + 32 * u + (int32_t)lane;
                c[u] = i < len ? ld_color(io.Xc + (P ? entry_id(w[u]) : w[u]), io.pol_col) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int32_t i = base + 32 * u + (int32_t)lane;
                const bool in = i < len;
                const uint32_t col = word_color(c[u]);
                const bool settled = in && word_settled(c[u]);
                const int32_t wid = P ? entry_id(w[u]) : w[u];
                bool pre = false;
                if constexpr (!P) {
                    pre = in && col == cv && wid < v;
                } else if (in && (col == cv || (first && !settled))) {
                    pre = first ? precedes(p.prio, wid, v, pv) : w[u] < 0;
                    if (first) w[u] = (int32_t)((uint32_t)wid | (pre ? kPrecBit : 0u));  // the entry kept
                }
                if (in) {
                    if (col == cv && pre) conflict = true;
                    const unsigned idx = col - 1u;
                    const uint32_t bit = 1u << (idx & 31u);
                    if (idx < 32u) {
                        rd0 |= bit;
                        rs0 |= settled ? bit : 0u;
                    } else if (idx < 64u) {
                        rd1 |= bit;
                        rs1 |= settled ? bit : 0u;
                    } else if (idx < 256u) {
                        atomicOr(&sm.dyn[idx >> 5], bit);
                        if (settled) atomicOr(&sm.stat[idx >> 5], bit);
                    }
                }
                // survivors, in order, to the next round's list
                const unsigned kb = __ballot_sync(kFull, in && !settled);
                if (in && !settled)
                    st_stream(io.rout + b + kept + __popc(kb & ((1u << lane) - 1u)), w[u], io.pol_row);
                kept += __popc(kb);
            }
        }
        const bool conf = __any_sync(kFull, conflict);
        rd0 = __reduce_or_sync(kFull, rd0);
        rs0 = __reduce_or_sync(kFull, rs0);
        rd1 = __reduce_or_sync(kFull, rd1);
        rs1 = __reduce_or_sync(kFull, rs1);
        __syncwarp();
        const unsigned q7 = lane & 7u;
        uint32_t stat = 0u, all = 0u;
        if (lane < 8u) {
            stat = old | sm.stat[q7] | (q7 == 0u ? rs0 : (q7 == 1u ? rs1 : 0u));
            all = stat | sm.dyn[q7] | (q7 == 0u ? rd0 : (q7 == 1u ? rd1 : 0u));
        }
        __syncwarp();
        if (!conf) {
            if (lane == 0) settle(p, io, v, cv);
            maxc = max(maxc, (int)cv);
        } else {
            const int ff = window_first_clear(all);
            const uint32_t color = ff >= 0 ? (uint32_t)ff + 1u : rescan_first_fit(p.rowptr, p.colidx, io.Xc, v);
            if (lane < 8u) p.stat[(size_t)v * 8 + lane] = stat;
            if (lane == 0) {
                recolor(p, io, v, color);
                vol += (unsigned)kept;
            }
        }
        if ((int)lane == j) {
            my_conflict = conf;
            my_kept = kept;
        }
    }
    // next round: same row start, the kept entries; the bin may shrink (never grow)
    const int4 ne = make_int4(en.x, en.y, my_kept, en.w);
    const int nb = bin_of(my_kept, p.s_max, p.m_max);
    warp_append(my_conflict && nb == kBinS, ne, io.next.S, &io.next.cnt->s);
    warp_append(my_conflict && nb == kBinM, ne, io.next.M, &io.next.cnt->m);
    __syncwarp();
}

// H bin: one chunk of up to 1024 entries of the vertex at worklist position
// h.pos, read in sub-blocks of 256 (two halves of 4 entries per lane).  A
// vertex whose active list fits one chunk is decided by this warp at once;
// otherwise the chunks OR their results into the vertex's record, and the
// warp that completes the last chunk decides it and clears the record.
template <typename T, bool P>  // P: a priority array is given
__device__ __forceinline__ void hub_chunk(const Params<T>& p, const PassIO<T>& io, TaskHead h,
                                          FlatSmem& sm, int& maxc, unsigned& vol) {
    constexpr int kHalf = kPerLane / 2;
    const unsigned lane = lane_id();
    const int32_t v = h.e.x, b = h.e.y, len = h.e.z;
    const int32_t e = b + len;
    const int32_t lo = h.lo, hi = min(e, lo + kChunk);
    const unsigned nch = (unsigned)(len + kChunk - 1) / kChunk;
    const bool single = nch == 1;
    const uint32_t cv = word_color(ld_color(io.Xc + v, io.pol_col));
    const uint32_t pv = p.prio ? __ldg(p.prio + v) : 0u;
    // a vertex decided by this warp: its static mask word `lane`, read now
    const uint32_t old_single = (single && lane < 8u && !io.first) ? __ldcg(p.stat + (size_t)v * 8 + lane) : 0u;
    bool conflict = false;
    // this chunk's color windows: all colors in sm.dyn[0..8), settled ones in sm.stat[0..8)
    if (lane < 8u) { sm.dyn[lane] = 0u; sm.stat[lane] = 0u; }
    __syncwarp();
    HubRecord* rec = p.hubs + h.pos;
    unsigned local = 0;  // survivors written so far (single-chunk vertex)
    uint32_t rd0 = 0u, rs0 = 0u, rd1 = 0u, rs1 = 0u;  // this lane's colors 1..64 (all, settled)
    for (int32_t sb = lo; sb < hi; sb += kHubSub) {
        // the next sub-block (eight 128-byte lines) comes into L1 meanwhile
        if (lane < 8u && sb + kHubSub + 32 * (int32_t)lane < hi) prefetch_l1(io.rin + sb + kHubSub + 32 * lane);
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            int32_t w[kHalf];
            T c[kHalf];
            unsigned keepbits[kHalf];
#pragma unroll
            for (int u = 0; u < kHalf; ++u) {
                const int32_t j = sb + (int32_t)lane + 32 * (half * kHalf + u);
                w[u] = j < hi ? ld_row(io.rin + j, io.pol_row) : 0;
            }
#pragma unroll
            for (int u = 0; u < kHalf; ++u) {
                const int32_t j = sb + (int32_t)lane + 32 * (half * kHalf + u);
                c[u] = j < hi ? ld_color(io.Xc + (P ? entry_id(w[u]) : w[u]), io.pol_col) : (T)0;
            }
            unsigned nkeep = 0;
#pragma unroll
            for (int u = 0; u < kHalf; ++u) {
                const int32_t j = sb + (int32_t)lane + 32 * (half * kHalf + u);
                const bool in = j < hi;
                const uint32_t col = word_color(c[u]);
                const bool settled = in && word_settled(c[u]);
                const int32_t wid = P ? entry_id(w[u]) : w[u];
                bool pre = false;
                if constexpr (!P) {
                    pre = in && col == cv && wid < v;
                } else if (in && (col == cv || (io.first && !settled))) {
                    pre = io.first ? precedes(p.prio, wid, v, pv) : w[u] < 0;
                    if (io.first) w[u] = (int32_t)((uint32_t)wid | (pre ? kPrecBit : 0u));  // the entry kept
                }
                if (in) {
                    if (col == cv && pre) conflict = true;
                    const unsigned idx = col - 1u;
                    // colors 1..64 gather in registers (one warp reduction per chunk); the
                    // rest go to the shared windows, where every lane of the warp would
                    // otherwise hit the same few words
                    const uint32_t bit = 1u << (idx & 31u);
                    if (idx < 32u) {
                        rd0 |= bit;
                        rs0 |= settled ? bit : 0u;
                    } else if (idx < 64u) {
                        rd1 |= bit;
                        rs1 |= settled ? bit : 0u;
                    } else if (idx < 256u) {
                        atomicOr(&sm.dyn[idx >> 5], bit);
                        if (settled) atomicOr(&sm.stat[idx >> 5], bit);
                    }
                }
                keepbits[u] = __ballot_sync(kFull, in && !settled);
                nkeep += __popc(keepbits[u]);
            }
            // survivors go to [b + slot, b + slot + nkeep) of the next round's list
            unsigned slot = local;
            if (!single) {
                if (lane == 0 && nkeep) slot = atomicAdd(&rec->kept, nkeep);
                slot = __shfl_sync(kFull, slot, 0);
            }
            local += nkeep;
#pragma unroll
            for (int u = 0; u < kHalf; ++u) {
                if ((keepbits[u] >> lane) & 1u)
                    st_stream(io.rout + b + slot + __popc(keepbits[u] & ((1u << lane) - 1u)), w[u], io.pol_row);
                slot += __popc(keepbits[u]);
            }
        }
    }
    const bool any_conflict = __any_sync(kFull, conflict);
    __syncwarp();
    rd0 = __reduce_or_sync(kFull, rd0);
    rs0 = __reduce_or_sync(kFull, rs0);
    rd1 = __reduce_or_sync(kFull, rd1);
    rs1 = __reduce_or_sync(kFull, rs1);
    const unsigned q7 = lane & 7u;
    const uint32_t word = sm.dyn[q7] | (q7 == 0u ? rd0 : (q7 == 1u ? rd1 : 0u));
    const uint32_t sword = sm.stat[q7] | (q7 == 0u ? rs0 : (q7 == 1u ? rs1 : 0u));
    __syncwarp();
    bool conf;
    int32_t kept;
    uint32_t all = 0, stat = 0;
    if (single) {
        conf = any_conflict;
        kept = (int32_t)local;
        if (lane < 8u) {
            stat = old_single | sword;
            all = stat | word;
        }
    } else {
        if (lane < 8u && word) atomicOr(&rec->mask[lane], word);
        if (lane < 8u && sword) atomicOr(&rec->stat[lane], sword);
        if (lane == 0 && any_conflict) atomicOr(&rec->conflict, 1u);
        __threadfence();
        unsigned done = 0;
        if (lane == 0) done = atomicAdd(&rec->done, 1u);
        done = __shfl_sync(kFull, done, 0);
        if (done != nch - 1) return;
        // last chunk of v: decide
        __threadfence();
        conf = __ldcg(&rec->conflict) != 0u;
        kept = (int32_t)__ldcg(&rec->kept);
        if (lane < 8u) {
            const uint32_t old = io.first ? 0u : __ldcg(p.stat + (size_t)v * 8 + lane);
            stat = old | __ldcg(&rec->stat[lane]);
            all = stat | __ldcg(&rec->mask[lane]);
        }
        ((unsigned*)rec)[lane] = 0u;  // reset for the next round (32 words)
    }
    if (!conf) {
        if (lane == 0) settle(p, io, v, cv);
        maxc = max(maxc, (int)cv);
        return;
    }
    const int ff = window_first_clear(all);
    const uint32_t color = ff >= 0 ? (uint32_t)ff + 1u : rescan_first_fit(p.rowptr, p.colidx, io.Xc, v);
    if (lane < 8u) p.stat[(size_t)v * 8 + lane] = stat;
    if (lane == 0) {
        recolor(p, io, v, color);
        vol += (unsigned)kept;
    }
    warp_append_one(io.next, make_int4(v, b, kept, h.e.w));
}

// One fused pass over U_k, shared among W warps (this warp is number gw).
// Task t: first the H-bin chunks, then the M-bin entries, up to kMedPerTask
// per task (fewer as the round shrinks), then the S-bin entries, 32 per task
// (down to kShortPerTaskMin as the round shrinks); an S or H task reads at
// most 1024 entries.  Warp gw takes tasks gw, gw + W, ... for half of its even
// share (at least two); then, with a counter (ctr), it claims one task at a
// time (nstat W + the counter's old value), so that warps that drew cheap
// tasks take more and the round ends when the work does, not when the
// unluckiest warp's fixed share does, while only about half the tasks cost an
// atomic on the counter's line; without a counter it keeps taking every W-th
// task.  The next task's head is loaded, and the claim after it issued,
// before the current task runs, so neither waits on memory.
template <typename T, bool P>  // P: a priority array is given
__device__ __forceinline__ void run_pass(const Params<T>& p, int k, unsigned nS, unsigned nM,
                                         unsigned nHC, int& maxc, unsigned gw, unsigned W, unsigned* ctr) {
    __shared__ FlatSmem s_flat[kWarpsPerBlockMax];
    const PassIO<T> io = pass_io(p, k);
    const unsigned wib = threadIdx.x >> 5;
    // S vertices per task: 32 in a large round, down to kShortPerTaskMin as it
    // shrinks; a task of 32 short lists walks up to 1024 entries in sequence,
    // which in the last rounds was the longest chain of the round
    const unsigned spt = max((unsigned)kShortPerTaskMin, min(32u, nS / (4u * W)));
    const unsigned tS = (nS + spt - 1) / spt;
    // M vertices per task: up to kMedPerTask when the round has enough of them
    // for several tasks per warp, fewer (down to 1) as the round shrinks, so
    // that a task's chain of per-vertex reads does not set the round's length
    const unsigned mpt = max(1u, min((unsigned)kMedPerTask, nM / (4u * W)));
    const unsigned tM = (nM + mpt - 1) / mpt;
    const unsigned total = nHC + tM + tS;
    unsigned vol = 0;  // this lane's share of the next round's read volume
    // this warp's tasks: gw + jW for j < nstat, then claimed ones from nstat W on
    const unsigned nstat = ctr ? max(2u, total / W / 2) : 0xffffffffu;
    TaskHead cur;
    if (gw < total) cur = load_head(io, gw, nS, nM, nHC, tM, mpt, spt);
    unsigned tn = gw + W;
    unsigned j = 0;  // position of the current task in that sequence
    for (unsigned t = gw; t < total; ++j) {
        TaskHead nxt;
        if (tn < total) nxt = load_head(io, tn, nS, nM, nHC, tM, mpt, spt);
        // the task after next: fixed, or claimed now (its number is needed after this task)
        const bool fixed = j + 2u < nstat;
        unsigned claim = 0;
        if (!fixed && tn < total && lane_id() == 0) claim = atomicAdd(ctr, 1u);
        if (t < nHC) {
            hub_chunk<T, P>(p, io, cur, s_flat[wib], maxc, vol);
        } else if (t - nHC < tM) {
            vertex_task<T, P>(p, io, cur.e, s_flat[wib], maxc, vol);
        } else {
            flat_task<T, P>(p, io, cur.e, s_flat[wib], maxc, vol);
        }
        const unsigned tnn = fixed ? tn + W : nstat * W + __shfl_sync(kFull, claim, 0);
        t = tn;
        cur = nxt;
        tn = tn < total ? tnn : total;
    }
    fold_volume(p.st, p.round_vol, p.round_cap, k + 1, vol);
}

// All rounds k >= 2 in one cooperative launch; a bounded grid barrier
// separates the rounds.  Every block reads the same counts and status after
// a barrier, so all blocks take the same decisions in the same round.  Once a
// round reads at most p.tail_volume entries, block 0 runs the remaining rounds
// alone, separated by block barriers (the other blocks leave): the same
// synchronous rounds, without the cost of a grid barrier per round.
template <typename T, bool P>  // P: a priority array is given
__global__ void __launch_bounds__(256, kMinBlocks) rounds_persistent_kernel(Params<T> p) {
    RoundState* st = p.st;
    int maxc = 0;
    unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    unsigned W = (gridDim.x * blockDim.x) >> 5;
    bool tail = false;
    for (int k = 2;; ++k) {
        const RoundCounts& c = st->rc[k % 3];
        const unsigned long long hc = __ldcg(&c.hc);
        const unsigned nS = __ldcg(&c.s), nM = __ldcg(&c.m), nH = hub_count(hc), nHC = hub_chunks(hc);
        const unsigned size = nS + nM + nH;
        // start of this pass (the last record, for the empty round, marks the end)
        if (p.round_ns && blockIdx.x == 0 && threadIdx.x == 0 && k - 1 <= p.round_cap)
            p.round_ns[k - 1] = globaltimer_ns();
        if (size == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) st->rounds = k - 1;
            break;
        }
        // (not st->status itself: a block already working on this round may set it)
        if (__ldcg(&st->status_at_barrier) == kStatusColorOverflow) break;
        if (k > p.max_rounds) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                st->rounds = k - 1;
                st->status = kStatusMaxRounds;
            }
            break;
        }
        if (!tail && p.tail_volume >= 0 && __ldcg(&st->rc[k % 3].vol) <= (unsigned)p.tail_volume) {
            if (blockIdx.x != 0) break;
            tail = true;
            gw = threadIdx.x >> 5;
            W = blockDim.x >> 5;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            RoundCounts& z = st->rc[(k + 2) % 3];
            z.s = z.m = z.vol = 0u;
            z.hc = 0ull;
            st->task_next[(k + 1) % 3] = 0u;  // round k + 1's claims (no one touches it in round k)
            if (k - 1 < p.round_cap) p.round_sizes[k - 1] = (int32_t)size;
        }
        run_pass<T, P>(p, k, nS, nM, nHC, maxc, gw, W, &st->task_next[k % 3]);
        if (tail) {
            __syncthreads();
            if (threadIdx.x == 0) {
                __threadfence();
                st->status_at_barrier = *((volatile int*)&st->status);
            }
            __syncthreads();
        } else if (!grid_barrier(st, p.barrier_polls)) {
            break;
        }
    }
    fold_max_color(st, maxc);
}

// One pass per launch (loop mode 1): counts come from the host.
template <typename T, bool P>  // P: a priority array is given
__global__ void __launch_bounds__(256, kMinBlocks) round_kernel(Params<T> p, int k, unsigned nS, unsigned nM,
                                                       unsigned nHC) {
    int maxc = 0;
    run_pass<T, P>(p, k, nS, nM, nHC, maxc, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
             (gridDim.x * blockDim.x) >> 5, nullptr);
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

// Loop mode 2: the rounds as a CUDA graph whose while node repeats
// graph_round_kernel + graph_cond_kernel on the device.  graph_round_kernel
// runs round st->graph_round over the counts that the previous pass left.
template <typename T, bool P>  // P: a priority array is given
__global__ void __launch_bounds__(256, kMinBlocks) graph_round_kernel(Params<T> p) {
    RoundState* st = p.st;
    const int k = __ldcg(&st->graph_round);
    const RoundCounts& c = st->rc[k % 3];
    const unsigned nS = __ldcg(&c.s), nM = __ldcg(&c.m), nHC = hub_chunks(__ldcg(&c.hc));
    int maxc = 0;
    run_pass<T, P>(p, k, nS, nM, nHC, maxc, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
             (gridDim.x * blockDim.x) >> 5, nullptr);
    fold_max_color(st, maxc);
}

// One thread, after round k (k = 1 before the loop): decide whether round k + 1
// runs, clear the counters it will append to, and set the while condition.
template <typename T>
__global__ void graph_cond_kernel(Params<T> p, int before_loop, cudaGraphConditionalHandle handle) {
    RoundState* st = p.st;
    const int k = before_loop ? 1 : st->graph_round;
    const int kn = k + 1;
    const RoundCounts& c = st->rc[kn % 3];
    const unsigned size = c.s + c.m + hub_count(c.hc);
    unsigned go = 0u;
    if (size == 0u) {
        st->rounds = k;
    } else if (st->status == kStatusColorOverflow) {
        st->rounds = k;
    } else if (kn > p.max_rounds) {
        st->rounds = k;
        st->status = kStatusMaxRounds;
    } else {
        RoundCounts& z = st->rc[(kn + 1) % 3];
        z.s = z.m = z.vol = 0u;
        z.hc = 0ull;
        if (kn - 1 < p.round_cap) p.round_sizes[kn - 1] = (int32_t)size;
        st->graph_round = kn;
        go = 1u;
    }
    __threadfence();
    cudaGraphSetConditional(handle, go);
}

struct ValidateOut {
    unsigned long long sum_fwd, sum_bwd;
    int bad_index, self_loop;
};

// Range and self-loop checks per entry; symmetry via hash sums of the entry
// multiset E and of its transpose (equal when E is symmetric).
__global__ void validate_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                int32_t n, ValidateOut* out) {
    const unsigned lane = lane_id();
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
