/*
 * The paper's own multicore form of Algorithm 2 ("Iterative", Sec. 3.2), as
 * its OpenMP implementations run it (Sec. 4): the worklist is split among
 * threads; in Phase 1 every worklist vertex takes the smallest color none of
 * its neighbours holds *at the moment it reads them* (other threads are
 * writing colors meanwhile), and in Phase 2, after all of Phase 1, a vertex
 * goes back to the worklist if a preceding neighbour holds its color.
 *
 * TEST AND BASELINE INFRASTRUCTURE ONLY: timed as the paper's CPU method on
 * the host cores beside the GPU path, never called by it.  The result depends
 * on the thread schedule, so it is checked for validity only (a proper
 * coloring, color(v) <= deg(v) + 1, rounds <= n); with one thread, Phase 1
 * visits U in order and reads every earlier color, which is Algorithm 1
 * (Greedy) in index order with no conflicts and one round (Sec. 3.2 notes
 * that one thread makes Phase 1 the serial algorithm) -- the pin in
 * tests/test_async_omp.py.
 *
 * Colors are read and written with relaxed atomics: the races the method
 * relies on are then defined behaviour.  Forbidden colors are marked with a
 * (round, vertex) stamp in a per-thread array, so marks of an earlier round
 * never count (the label reading of Algorithm 2's forbiddenColors).
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline int32_t load_color(const int32_t* c) { return __atomic_load_n(c, __ATOMIC_RELAXED); }
static inline void store_color(int32_t* c, int32_t x) { __atomic_store_n(c, x, __ATOMIC_RELAXED); }

/* w precedes v: smaller key first, ties by index (keys NULL: index order). */
static inline int precedes(int32_t w, int32_t v, const uint32_t* p) {
    if (p && p[w] != p[v]) return p[w] < p[v];
    return w < v;
}

/*
 * orc_async_omp - color with `threads` OpenMP threads (0: the runtime's
 * default).  colors[n] receives 1-based colors; returns 0, -1 for bad
 * arguments or memory, or -4 when the worklist is not empty after
 * max_rounds rounds (0: n).
 */
int orc_async_omp(int32_t n, const int32_t* rowptr, const int32_t* colidx, const uint32_t* prio,
                  int32_t threads, int32_t max_rounds, int32_t* color, int32_t* ncolors, int32_t* rounds) {
    if (n < 0 || !ncolors || !rounds || (n > 0 && (!rowptr || !color))) return -1;
    *ncolors = 0;
    *rounds = 0;
    if (n == 0) return 0;
    int32_t maxdeg = 0;
    for (int32_t v = 0; v < n; ++v)
        if (rowptr[v + 1] - rowptr[v] > maxdeg) maxdeg = rowptr[v + 1] - rowptr[v];
    const int nt = threads > 0 ? threads : omp_get_max_threads();
    const size_t width = (size_t)maxdeg + 2;  /* colors 0..maxdeg+1 */
    int32_t* U = malloc((size_t)n * sizeof(int32_t));
    int32_t* R = malloc((size_t)n * sizeof(int32_t));
    int64_t* marks = malloc((size_t)nt * width * sizeof(int64_t));
    if (!U || !R || !marks) {
        free(U);
        free(R);
        free(marks);
        return -1;
    }
    for (size_t i = 0; i < (size_t)nt * width; ++i) marks[i] = -1;
    for (int32_t v = 0; v < n; ++v) {
        U[v] = v;
        color[v] = 0;
    }
    const int32_t limit = max_rounds > 0 ? max_rounds : n;
    int32_t nu = n, r = 0;
    int rc = 0;
    while (nu > 0) {
        if (r >= limit) {
            rc = -4;
            break;
        }
        ++r;
        /* Phase 1: tentative colors from the neighbours' current colors */
#pragma omp parallel num_threads(nt)
        {
            int64_t* f = marks + (size_t)omp_get_thread_num() * width;
#pragma omp for schedule(dynamic, 512)
            for (int32_t i = 0; i < nu; ++i) {
                const int32_t v = U[i];
                const int64_t stamp = (int64_t)r * n + v;
                for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                    const int32_t c = load_color(color + colidx[e]);
                    if (c >= 0 && (size_t)c < width) f[c] = stamp;
                }
                int32_t c = 1;
                while (f[c] == stamp) ++c;
                store_color(color + v, c);
            }
        }
        /* Phase 2: the later of two equally colored neighbours goes back */
        int32_t nr = 0;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 512)
        for (int32_t i = 0; i < nu; ++i) {
            const int32_t v = U[i];
            const int32_t cv = load_color(color + v);
            for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                const int32_t w = colidx[e];
                if (load_color(color + w) == cv && precedes(w, v, prio)) {
                    R[__atomic_fetch_add(&nr, 1, __ATOMIC_RELAXED)] = v;
                    break;
                }
            }
        }
        int32_t* t = U;
        U = R;
        R = t;
        nu = nr;
    }
    int32_t mc = 0;
    for (int32_t v = 0; v < n; ++v)
        if (color[v] > mc) mc = color[v];
    *ncolors = mc;
    *rounds = r;
    free(U);
    free(R);
    free(marks);
    return rc;
}
