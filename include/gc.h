/*
 * gc.h - C ABI of the GB300 speculative distance-1 graph coloring library
 * (libgc.so).
 *
 * Method: Algorithm 2 ("Iterative", Sec. 3.2) of Catalyurek, Feo,
 * Gebremedhin, Halappanavar and Pothen, "Graph coloring algorithms for
 * multi-core and massively multithreaded architectures" (arXiv 1205.3809),
 * run in synchronous rounds over a worklist U (initially all vertices):
 *   Phase 1 (tentative coloring): every v in U takes the smallest color > 0
 *     that none of its neighbours held at the end of the previous round
 *     (first fit, Algorithm 1 / Sec. 3.1);
 *   Phase 2 (conflict detection): v in U goes back to U if a neighbour w
 *     with the same color precedes it, where w precedes v iff
 *     (priority[w], w) < (priority[v], v); with no priority array this is the
 *     paper's rule that the higher index recolors;
 * until U is empty.  Because each round reads only the previous round's
 * colors, the result is a pure function of the graph and the priority.
 *
 * Conventions for every entry point:
 *  - Graph: simple undirected graph as a symmetric CSR of int32: rowptr has
 *    n+1 entries, rowptr[0] = 0, non-decreasing, nnz = rowptr[n] < 2^31;
 *    colidx has nnz entries, each in [0, n); adjacency must be symmetric (a
 *    one-directional entry could hide a conflict) and free of self loops.
 *    Rows need not be sorted.  Duplicate entries are harmless.
 *  - Device pointers are global-memory pointers of the current CUDA device;
 *    the caller owns them; inputs are never modified.
 *  - Colors are written as int32 in 1..ncolors.
 *  - Calls are stream-ordered on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream) and return after the host outputs are known, i.e. they
 *    synchronise that stream once at the end (and once after the setup scan).
 *  - Errors are returned as a gc_status code; nothing is thrown or aborted.
 *    After GC_ERR_CUDA the CUDA error is available from gc_last_cuda_error().
 *  - The library keeps a per-device workspace (grow only) between calls;
 *    gc_release() frees it.  Calls from several host threads are serialised.
 */
#ifndef GC_H
#define GC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gc_status {
    GC_OK = 0,
    GC_ERR_INVALID = -1,    /* bad argument (null pointer, n < 0, bad option) */
    GC_ERR_CUDA = -2,       /* a CUDA runtime call failed */
    GC_ERR_OOM = -3,        /* workspace allocation failed */
    GC_ERR_MAX_ROUNDS = -4, /* U not empty after max_rounds rounds */
    GC_ERR_TIMEOUT = -5,    /* a bounded device-side wait gave up */
    GC_ERR_BAD_GRAPH = -6,  /* CSR rejected by the setup scan or validation */
    GC_ERR_TOO_LARGE = -7   /* gc_color_noalloc: graph needs more scratch than it has */
} gc_status;

/*
 * Options.  Zero-initialise and set what you need; 0 selects the default.
 */
typedef struct gc_options {
    int32_t small_max_degree;  /* worklist vertices whose active list has at
                                  most this many entries go 32 to a warp task
                                  (1..32, default 32) */
    int32_t medium_max_degree; /* active lists up to this length (and above
                                  the small limit) go up to 16 to a warp task
                                  (fewer in rounds with few of them), each list
                                  read by the whole warp in turn; longer lists are
                                  split into chunks of 1024 entries, one warp
                                  each (small_max_degree..256, default 256) */
    int32_t max_rounds;        /* stop with GC_ERR_MAX_ROUNDS after this many
                                  rounds (default n; rounds <= n always holds,
                                  since the first vertex of U in precedence
                                  order settles in every round) */
    int32_t validate;          /* 1: check colidx range, self loops and
                                  symmetry on the device before coloring */
    int32_t loop_mode;         /* 0: all rounds in one persistent cooperative
                                  launch (default); 1: one launch per round,
                                  the host reads |U| after each; 2: a CUDA
                                  graph whose while node runs one round
                                  kernel per round and decides on the device
                                  whether to go on */
    int32_t color_bits;        /* 0 or 16: 16-bit color state (a flag bit and
                                  colors below 2^15), and if a color does not
                                  fit, the call starts over with 32-bit state;
                                  32: 32-bit state from the start */
    int32_t block_threads;     /* threads per block: 128 or 256 (default) */
    int32_t telemetry;         /* 1: time the phases with CUDA events on the
                                  call's stream (see gc_last_phase_ms) */
    int32_t narrow_color_limit; /* testing: with 16-bit state, treat colors >=
                                  this as not fitting (0: 2^15), to exercise
                                  the 32-bit restart */
    int32_t tail_volume;       /* persistent launch: once a round reads at
                                  most this many adjacency entries, one thread
                                  block runs the remaining rounds alone, with
                                  block barriers instead of grid barriers
                                  (0 or negative: never, the default: the
                                  last rounds are bound by their longest
                                  task, not by the barrier) */
    int32_t batch_mode;        /* gc_batch_create only.  0: choose (default:
                                  2 when no graph holds more than 2/SMs of
                                  the batch's vertices + entries, else 1);
                                  1: all graphs share one persistent grid and
                                  its rounds (the single-graph kernels on the
                                  union); 2: one thread block per graph, its
                                  colors in shared memory (one byte each, up
                                  to the block's shared memory; larger graphs
                                  keep them in global memory), graphs taken
                                  largest first from a queue */
    int32_t local_thread_degree; /* batch_mode 2: graphs whose average degree
                                  is at most this take one thread per vertex
                                  (default 0 means 32; negative: never); the
                                  others a group of 4..32 lanes per vertex,
                                  about half their average degree */
    int32_t local_shared_bytes; /* batch_mode 2: shared memory per block for
                                  colors, at least 16384 and at most what a
                                  block can have (0: 167936, which leaves L1
                                  cache for the rows; a graph with more
                                  vertices keeps the rest of its colors in
                                  global memory) */
    int32_t barrier_poll_limit; /* testing, loop_mode 0: the grid barrier
                                  between rounds gives up after this many
                                  polls (0: after 2^26 polls or 4 s), sets
                                  GC_ERR_TIMEOUT and every block leaves; the
                                  next call starts from a clean state */
    int32_t workspace_limit_mb; /* testing: a call that would have to grow
                                  the device workspace beyond this many MiB
                                  fails with GC_ERR_OOM without allocating
                                  (as if cudaMalloc had refused), keeping the
                                  workspace it already has (0: no limit) */
    int32_t reserved[1];
} gc_options;

/*
 * gc_color - color the graph (Algorithm 2, synchronous rounds).
 *   rowptr, colidx : device, CSR as above.
 *   n              : vertex count (>= 0).
 *   priority       : device, n uint32 keys, or NULL for index priority.
 *                    Smaller key = higher precedence; ties go by index.
 *   colors_out     : device, n int32 (caller-allocated), receives 1-based colors.
 *   ncolors        : host, receives the largest color (0 when n == 0).
 *   rounds         : host, receives the number of rounds (0 iff n == 0).
 * Returns GC_OK or a gc_status code.  On an error colors_out is unspecified.
 */
int gc_color(const int32_t* rowptr, const int32_t* colidx, int32_t n, const uint32_t* priority,
             int32_t* colors_out, int32_t* ncolors, int32_t* rounds);

/*
 * gc_color_ex - gc_color with a stream, options and per-round telemetry.
 *   stream          : cudaStream_t to run on (NULL = default stream).
 *   opt             : options or NULL for defaults.
 *   round_sizes     : host, optional (NULL): round_sizes[r-1] = |U| at the
 *                     start of round r, for r = 1..min(rounds, round_sizes_cap,
 *                     2^20).
 */
int gc_color_ex(const int32_t* rowptr, const int32_t* colidx, int32_t n, const uint32_t* priority,
                int32_t* colors_out, int32_t* ncolors, int32_t* rounds, void* stream,
                const gc_options* opt, int32_t* round_sizes, int32_t round_sizes_cap);

/*
 * gc_color_host - the same computation on a graph held in HOST memory.
 *   rowptr, colidx, priority (or NULL): host arrays, as above.
 *   colors_out : host, n int32.
 * The library copies the inputs into its device workspace on `stream`,
 * colors, and copies the colors back; pinned host buffers copy fastest.
 */
int gc_color_host(const int32_t* rowptr, const int32_t* colidx, int32_t n,
                  const uint32_t* priority, int32_t* colors_out, int32_t* ncolors,
                  int32_t* rounds, void* stream, const gc_options* opt);

/*
 * gc_validate_csr - device check of a CSR graph (rowptr shape, colidx range,
 * no self loops, symmetric adjacency).  Symmetry is tested by comparing two
 * 64-bit hash sums of the entry multiset and of its transpose, so an
 * asymmetric graph passes with probability about 2^-64.
 * Returns GC_OK, GC_ERR_BAD_GRAPH, or another gc_status code.
 */
int gc_validate_csr(const int32_t* rowptr, const int32_t* colidx, int32_t n, void* stream);

/*
 * gc_last_round_stats - per-round telemetry of the last successful coloring
 * call on the current device: sizes[r-1] = |U_r| and volumes[r-1] = the sum of
 * the degrees of the vertices of U_r (the adjacency entries round r's Phase 1
 * reads), for r = 1..min(rounds, cap, 4096 or the round_sizes_cap of that
 * call).  Either output may be NULL.  Returns the number of rounds written,
 * or a negative gc_status (GC_ERR_INVALID if there is no such call).
 */
int gc_last_round_stats(int32_t* sizes, int64_t* volumes, int32_t cap);

/*
 * gc_last_phase_ms - phase timings, in milliseconds from CUDA events recorded
 * on the call's stream, of the last call made with opt->telemetry = 1:
 * ms[0] setup scan kernel, ms[1] round 1 (the two pass-1 kernels), ms[2]
 * every later round (the persistent kernel, or all per-round launches with
 * their host round trips in loop_mode 1), ms[3] the whole call.
 * Returns the number of values written (<= cap, at most 4) or GC_ERR_INVALID.
 */
int gc_last_phase_ms(float* ms, int32_t cap);

/*
 * gc_last_round_ns - how long each round took in the last call made with
 * opt->telemetry = 1 and loop_mode 0 (one persistent launch): ns[0] = 0
 * (round 1 and its conflict test run before that launch; gc_last_phase_ms
 * times them), ns[k-1] = nanoseconds from the start of the pass that runs
 * round k's conflict test (and round k+1's tentative coloring) to the start
 * of the next, for k = 2..min(rounds, cap, 4096 or that call's
 * round_sizes_cap), read from the device's %globaltimer by one thread after
 * each grid barrier (its resolution is the device's, typically 32 ns to
 * 1 us).  Returns the number of values written, or GC_ERR_INVALID when the
 * last call kept no such record.
 */
int gc_last_round_ns(int64_t* ns, int32_t cap);

/* Text for a gc_status code (static storage). */
const char* gc_strerror(int code);

/* The CUDA error code (cudaError_t) behind the last GC_ERR_CUDA, or 0. */
int gc_last_cuda_error(void);

/* Free the workspace of every device this process used.  Returns GC_OK. */
int gc_release(void);

/* Bytes of device workspace currently held on the current device. */
size_t gc_workspace_bytes(void);

/* Number of kernel launches made by the last successful call on this
 * process (for launch accounting). */
int64_t gc_last_launch_count(void);

/*
 * gc_color_noalloc - gc_color for callers that cannot allocate memory while
 * they run: for example inside a framework whose caching allocator has
 * already reserved the device's memory, in a service with a fixed memory
 * plan that allocates nothing after start-up, or where cudaMalloc / cudaFree
 * must not synchronise the device.  The paper has no counterpart; this is an
 * interface of this library only.
 *
 * Same arguments and results as gc_color (device inputs and colors_out,
 * host ncolors and rounds, index priority when priority is NULL), on
 * `stream` (a cudaStream_t, NULL = legacy default stream), always with the
 * default options.  It calls no cudaMalloc, cudaMallocHost, cudaFree or any
 * other allocating routine: its workspace is one file-scope device array of
 * gc_noalloc_capacity_bytes() bytes (64 MiB), which every GPU that loads the
 * library holds until the process exits, and its host staging is on the
 * stack.  The first call on each device looks up that array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  Every call shares the array and it keeps the last call's
 * contents; each call clears what must start at zero.  Two calls that ran
 * on the GPU at the same time would race on the array; that cannot happen
 * here, because the call synchronises `stream` before it returns (it reads
 * the round count back) and calls from several host threads are serialised.
 * gc_last_round_stats, gc_last_round_ns and gc_last_phase_ms report nothing
 * after this call (GC_ERR_INVALID); gc_last_launch_count counts its kernel
 * launches.
 * Returns GC_ERR_TOO_LARGE when the graph needs more workspace than the
 * array holds (roughly 70 bytes per vertex plus 8 per adjacency entry), and
 * otherwise the codes gc_color returns.
 */
int gc_color_noalloc(const int32_t* rowptr, const int32_t* colidx, int32_t n,
                     const uint32_t* priority, int32_t* colors_out, int32_t* ncolors,
                     int32_t* rounds, void* stream);

/* Size in bytes of the fixed workspace gc_color_noalloc uses. */
size_t gc_noalloc_capacity_bytes(void);

/*
 * gc_color_async - Algorithm 2 (Sec. 3.2) as the paper runs it on shared
 * memory: Phase 1 reads the one shared color array while other threads
 * write it (each vertex sees some of this round's tentative colors), Phase 2
 * sends the later (by priority, then index) of two equally colored
 * neighbours back.  The colors depend on the schedule: the result is a
 * proper coloring with every color <= degree + 1, not a fixed one.  Same
 * arguments as gc_color plus max_rounds (<= 0: n) and stream; device arrays;
 * synchronises `stream` once per round.  Returns GC_OK, GC_ERR_INVALID,
 * GC_ERR_OOM, GC_ERR_CUDA or GC_ERR_MAX_ROUNDS.
 */
int gc_color_async(const int32_t* rowptr, const int32_t* colidx, int32_t n, const uint32_t* priority,
                   int32_t* colors_out, int32_t* ncolors, int32_t* rounds, int32_t max_rounds, void* stream);

/*
 * Batched coloring: many independent graphs in one persistent launch.
 *
 * Algorithm 2 (Sec. 3.2) in synchronous rounds on each graph of a batch, so
 * that each graph gets exactly the colors, color count and round count that
 * gc_color gives it alone, in one of two ways (gc_options.batch_mode):
 *   2: persistent thread blocks, one per SM, each taking whole graphs from a
 *      queue (largest first) and running all of a graph's rounds with its
 *      colors in shared memory (the default when no graph is a large share
 *      of the batch);
 *   1: all graphs advancing together in one cooperative launch over their
 *      disjoint union (vertex i of graph g = union vertex voff[g] + i, which
 *      keeps the order of indices inside every graph).
 *
 * Input layout (device arrays owned by the caller), for G graphs:
 *   vertex_offsets[G+1], edge_offsets[G+1] (HOST int64 arrays): graph g has
 *     n_g = voff[g+1] - voff[g] vertices and nnz_g = eoff[g+1] - eoff[g]
 *     adjacency entries; voff[0] = eoff[0] = 0, both nondecreasing,
 *     voff[G] < 2^31 and eoff[G] < 2^31;
 *   rowptr_cat[voff[G] + G]: graph g's own rowptr (n_g + 1 entries, from 0 to
 *     nnz_g) at rowptr_cat[voff[g] + g ..];
 *   colidx_cat[eoff[G]]: graph g's neighbour ids (local, 0 <= id < n_g) at
 *     colidx_cat[eoff[g] ..]; each graph symmetric with no self loops;
 *   priority: NULL (index order) or voff[G] uint32 keys (graph g's at
 *     priority[voff[g] ..]);
 * Outputs (device): colors_out[voff[G]] (colors >= 1), ncolors_out[G],
 *   rounds_out[G] (0 for an empty graph).
 *
 * gc_batch_create plans the batch: it checks the offsets and every graph's
 * rowptr, builds the union rowptr, scans degrees, allocates the plan's
 * workspace (mode 1: roughly 80 bytes per vertex plus 12 per adjacency entry;
 * mode 2: roughly 45 bytes per vertex) and, with opt->validate, checks ids,
 * self loops and symmetry.  It synchronises
 * `stream`.  The plan keeps the array pointers: later runs read the caller's
 * colidx_cat and priority and write the outputs, so their contents may change
 * between runs, but rowptr_cat is read only here (the degrees are fixed).
 * opt: as for gc_color_ex; loop_mode must be 0; telemetry is ignored.
 * Returns GC_OK, GC_ERR_INVALID, GC_ERR_BAD_GRAPH, GC_ERR_OOM or GC_ERR_CUDA;
 * on failure *plan is NULL.
 */
typedef struct gc_batch gc_batch;

int gc_batch_create(const int32_t* rowptr_cat, const int32_t* colidx_cat, const int64_t* vertex_offsets,
                    const int64_t* edge_offsets, int32_t num_graphs, const uint32_t* priority,
                    int32_t* colors_out, int32_t* ncolors_out, int32_t* rounds_out, const gc_options* opt,
                    void* stream, gc_batch** plan);

/* gc_batch_run - enqueue one coloring of the planned batch on `stream`:
 * memsets and kernels only (no allocation, no host synchronisation), so it
 * may be captured into a CUDA graph.  Read the status with gc_batch_status.
 * Runs of one plan use its one workspace: they must not overlap on the GPU
 * (issue them on one stream, or order the streams). */
int gc_batch_run(gc_batch* plan, void* stream);

/* gc_batch_launch_graph - the first call captures gc_batch_run into a CUDA
 * graph (on a private stream) and instantiates it; every call launches that
 * graph on `stream`. */
int gc_batch_launch_graph(gc_batch* plan, void* stream);

/* gc_batch_status - wait for `stream`, then report the last run: the largest
 * round count and color count over the batch, and GC_OK, GC_ERR_BAD_GRAPH (a
 * neighbour id outside its graph; it was replaced by 0), GC_ERR_MAX_ROUNDS
 * or GC_ERR_TIMEOUT. */
int gc_batch_status(gc_batch* plan, void* stream, int32_t* max_rounds, int32_t* max_colors);

/* gc_batch_features - the six gc_features features of every vertex of the
 * batch (features: voff[G] * 6 floats, device), from the plan's union graph
 * rebuilt from the current colidx_cat; graph g's rows at features[6*voff[g]..].
 * A vertex's features depend only on its own graph.  With gc_mlp_forward and
 * gc_priority_keys this gives the learned priority of every graph at once,
 * to be written into the priority array the plan was created with. */
int gc_batch_features(gc_batch* plan, float* features, void* stream);

/* gc_batch_round_stats - after a run (waits for `stream`): |U_r| over the whole
 * batch (sizes[r-1], host array of `cap`) and the adjacency entries round r
 * read (volumes[r-1]; round 1 reads every row; later rounds read the active
 * entries in batch_mode 1 and whole rows in batch_mode 2) for the first
 * min(rounds, cap, 4096) rounds, and the plan's color-state width in bits
 * (state_bits: 16 or 32 in mode 1, 8 in mode 2, whose graphs that need more
 * are recolored with 32-bit colors; the rounds of such a graph beyond the
 * 128th are counted twice).  Any output may be NULL.  Returns that round
 * count, or a gc_status (GC_ERR_INVALID for a NULL plan or cap < 0). */
int gc_batch_round_stats(gc_batch* plan, int32_t* sizes, int64_t* volumes, int32_t cap, int32_t* state_bits,
                         void* stream);

/* gc_batch_destroy - free the plan (waits for the device); NULL is a no-op. */
int gc_batch_destroy(gc_batch* plan);

/*
 * gc_color_batched - color a batch in one call: gc_batch_create, one
 * gc_batch_run and gc_batch_status on `stream`, then gc_batch_destroy.
 * Arguments as for gc_batch_create (offsets on the host, everything else on
 * the device, opt may be NULL).  Returns when the results are in colors_out,
 * ncolors_out and rounds_out, with the status of the run (GC_ERR_BAD_GRAPH
 * for an id outside its graph, GC_ERR_MAX_ROUNDS, ...).  For repeated runs on
 * the same batch, keep a plan instead: planning allocates and scans.
 */
int gc_color_batched(const int64_t* vertex_offsets, const int64_t* edge_offsets, int32_t num_graphs,
                     const int32_t* rowptr_cat, const int32_t* colidx_cat, const uint32_t* priority,
                     int32_t* colors_out, int32_t* ncolors_out, int32_t* rounds_out, void* stream,
                     const gc_options* opt);

/* Bytes of device memory the plan holds; kernels one run launches. */
size_t gc_batch_workspace_bytes(const gc_batch* plan);
int64_t gc_batch_launch_count(const gc_batch* plan);

/* gc_batch_mode - how the plan colors its graphs: 1 (one persistent grid over
 * the union) or 2 (one thread block per graph), as gc_options.batch_mode
 * describes; GC_ERR_INVALID for NULL. */
int gc_batch_mode(const gc_batch* plan);

/*
 * Autotuning.  Results never depend on the options (every option set gives
 * the same colors); only the time does.  These time a list of candidate
 * option sets on the caller's own input with CUDA events on `stream` (one
 * warm-up run, then `reps` timed runs each; the median goes to ms_out[c])
 * and return the index of the fastest in *best.  Candidates that change the
 * degree-bin limits or the block shape are the intended use.
 *
 * gc_tune: one graph, through gc_color_ex (colors_scratch: n int32, device).
 * gc_batch_tune: one batch, each candidate planned with gc_batch_create and
 * timed through gc_batch_launch_graph (arguments as for gc_batch_create).
 * Return GC_OK or the first error of a candidate's run.
 */
int gc_tune(const int32_t* rowptr, const int32_t* colidx, int32_t n, const uint32_t* priority,
            int32_t* colors_scratch, const gc_options* candidates, int32_t count, int32_t reps, void* stream,
            float* ms_out, int32_t* best);
int gc_batch_tune(const int32_t* rowptr_cat, const int32_t* colidx_cat, const int64_t* vertex_offsets,
                  const int64_t* edge_offsets, int32_t num_graphs, const uint32_t* priority, int32_t* colors_out,
                  int32_t* ncolors_out, int32_t* rounds_out, const gc_options* candidates, int32_t count,
                  int32_t reps, void* stream, float* ms_out, int32_t* best);

/*
 * Learned priority.  The paper colors in index order (Sec. 3.2) and cites
 * vertex-ordering heuristics for Algorithm 1 (smallest-last, largest-first;
 * Sec. 1, Sec. 3.1).  These entry points compute per-vertex features, run a
 * small MLP that scores where a vertex would sit in such an ordering, and turn
 * scores into gc_color priority keys.  All arrays are device arrays owned by
 * the caller; calls are asynchronous on `stream` and return after launching.
 * They return GC_OK, GC_ERR_INVALID or GC_ERR_CUDA.
 */

/* gc_features - features[6*v .. 6*v+5] of vertex v (fp32), deg = degree of v,
 * nbr = degrees of v's neighbours: log2(1+deg), floor(log2(1+deg)),
 * log2(1+mean nbr), log2(1+max nbr), log2(1+sum nbr), log2(1+min nbr)
 * (the last four 0 for an isolated vertex).  Graph as for gc_color. */
int gc_features(const int32_t* rowptr, const int32_t* colidx, int32_t n, float* features, void* stream);

/* Number of MLP parameters (1313): fp32 vector W1[32][6] | b1[32] |
 * W2[32][32] | b2[32] | W3[32] | b3.  Forward of features x: a0 = bf16(x),
 * a1 = bf16(relu(bf16(W1) a0 + b1)), a2 = bf16(relu(bf16(W2) a1 + b2)),
 * y = bf16(W3) . a2 + b3; products accumulate in fp32, bf16 rounds to
 * nearest even. */
int gc_mlp_param_count(void);

/* gc_mlp_forward - y[i] = MLP(x[6*i .. 6*i+5]) for i < n. */
int gc_mlp_forward(const float* params, const float* x, int64_t n, float* y, void* stream);

/* gc_mlp_grad - adds the gradient of scale * sum_i (y_i - t_i)^2 with respect
 * to params into grad (1313 floats) and sum_i (y_i - t_i)^2 into *sse
 * (device scalar).  Both accumulate: zero them first. */
int gc_mlp_grad(const float* params, const float* x, const float* t, int64_t n, float scale, float* grad,
                float* sse, void* stream);

/* gc_mlp_adam - one Adam step (Kingma & Ba) on params with moments m, v
 * (1313 floats each, zero before step 1); step counts from 1. */
int gc_mlp_adam(float* params, float* m, float* v, const float* grad, int32_t step, float lr, float beta1,
                float beta2, float eps, void* stream);

/* gc_mlp_train_step - one training step on the mean squared error of n
 * samples: zeroes grad (1313 floats) and *sse, adds the gradient of
 * (1/n) sum_i (y_i - t_i)^2 (gc_mlp_grad with scale 1/n), then takes
 * gc_mlp_adam step `step`.  Afterwards *sse holds sum_i (y_i - t_i)^2 under
 * the parameters before the update. */
int gc_mlp_train_step(float* params, float* m, float* v, float* grad, float* sse, const float* x, const float* t,
                      int64_t n, int32_t step, float lr, float beta1, float beta2, float eps, void* stream);

/* gc_priority_keys - keys[i] = a uint32 with the order of scores[i] (smaller
 * score, smaller key, higher precedence; -0 = +0; NaN last).  Equal scores
 * give equal keys, and gc_color then breaks the tie by index. */
int gc_priority_keys(const float* scores, int64_t n, uint32_t* keys, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GC_H */
