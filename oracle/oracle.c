/*
 * CPU oracle for speculative distance-1 graph coloring.  TEST INFRASTRUCTURE
 * ONLY: the tests, the smoke check and the CPU-baseline leg of the benchmark
 * call it; the library path never does.  It shares no code with the CUDA
 * path.  Plain, slow, single-threaded C, written so that each function can
 * be checked against the paper by eye.
 *
 * Paper: U. V. Catalyurek, J. Feo, A. H. Gebremedhin, M. Halappanavar and
 * A. Pothen, "Graph coloring algorithms for multi-core and massively
 * multithreaded architectures" (arXiv 1205.3809).
 *
 * Graph input everywhere: n vertices, CSR rowptr[n+1], colidx[rowptr[n]],
 * symmetric, no self loops.  Colors are positive integers; 0 = uncolored.
 *
 * Pins (what the tests check each function against, outside itself):
 *   orc_greedy          - first-fit fixed point vs lower neighbours (the
 *                         plain definition of Algorithm 1 in natural order),
 *                         <= B+1 colors (back degree, Sec. 3.1), brute-force
 *                         chromatic number on tiny graphs, hand-worked cases.
 *   orc_iterative       - closed forms derived by hand from Algorithm 2 in
 *                         synchronous rounds (edgeless, K_n, index-ordered
 *                         path, stars, complete bipartite), hand-worked
 *                         round traces under tests/golden/, the one-thread
 *                         reduction to Algorithm 1 (Sec. 3.2), validity,
 *                         per-vertex bound color <= deg+1, rounds <= n, and
 *                         an exhaustive set-based check on all graphs of up
 *                         to 6 vertices.
 *   orc_chromatic_number - known chromatic numbers (K_n, odd/even cycles,
 *                         bipartite graphs, Petersen graph).
 *   orderings            - hand-worked cases and the permutation property.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID -1
#define ORC_ERR_OOM -3
#define ORC_ERR_MAX_ROUNDS -4

static int64_t max_degree(int32_t n, const int32_t* rowptr) {
    int64_t d = 0;
    for (int32_t v = 0; v < n; ++v)
        if (rowptr[v + 1] - rowptr[v] > d) d = rowptr[v + 1] - rowptr[v];
    return d;
}

/*
 * Algorithm 1 (Greedy), Sec. 3.1.  Vertices are visited in `order` (NULL =
 * natural order 0..n-1).  For each v the colors of its neighbours are marked
 * in forbiddenColors with the label v; the array is initialised once with a
 * value that is not a vertex (-1) and never cleared.  v takes the smallest
 * i > 0 whose entry is not labelled v.  The array needs Delta+2 entries:
 * colors never exceed Delta+1.
 */
int orc_greedy(int32_t n, const int32_t* rowptr, const int32_t* colidx, const int32_t* order,
               int32_t* color, int32_t* ncolors) {
    if (n < 0 || !color || !ncolors || (n > 0 && (!rowptr || !colidx))) return ORC_ERR_INVALID;
    const int64_t delta = max_degree(n, rowptr);
    int64_t* forbiddenColors = (int64_t*)malloc((size_t)(delta + 2) * sizeof(int64_t));
    if (!forbiddenColors) return ORC_ERR_OOM;
    for (int64_t i = 0; i < delta + 2; ++i) forbiddenColors[i] = -1;
    for (int32_t v = 0; v < n; ++v) color[v] = 0;
    for (int32_t k = 0; k < n; ++k) {
        const int32_t v = order ? order[k] : k;
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            const int32_t w = colidx[e];
            forbiddenColors[color[w]] = v;
        }
        int32_t c = 1;
        while (forbiddenColors[c] == v) ++c;
        color[v] = c;
    }
    int32_t mx = 0;
    for (int32_t v = 0; v < n; ++v)
        if (color[v] > mx) mx = color[v];
    *ncolors = mx;
    free(forbiddenColors);
    return ORC_OK;
}

/*
 * Precedence used by the conflict test of Algorithm 2 (Sec. 3.2): of two
 * adjacent vertices with the same color, the one with the higher index is
 * recolored.  With a priority array p the order is the lexicographic
 * (p[w], w) < (p[v], v); p == NULL is index order, exactly the paper's
 * "v > w" test.
 */
static int precedes(int32_t w, int32_t v, const uint32_t* p) {
    if (p && p[w] != p[v]) return p[w] < p[v];
    return w < v;
}

/*
 * Algorithm 2 (Iterative), Sec. 3.2.
 *
 *   U <- V
 *   while U is not empty:
 *     Phase 1 (tentative coloring): for each v in U, mark the colors of all
 *       neighbours w in forbiddenColors with a label and give v the smallest
 *       color i > 0 not carrying that label;
 *     Phase 2 (conflict detection): R <- { v in U : some neighbour w has
 *       color[w] == color[v] and w precedes v };
 *     U <- R
 *
 * mode 0, synchronous rounds: Phase 1 of a round reads only the colors the
 *   previous round left (a snapshot taken when the round starts), so the
 *   result does not depend on any schedule.  Phase 1 forbids the snapshot
 *   color of every neighbour, including the stale tentative colors of other
 *   vertices of U (Algorithm 2 reads color[w] for every w in adj(v)).
 * mode 1, sequential visibility: Phase 1 visits U in precedence order and
 *   reads colors as they are written, which is Algorithm 2 run by a single
 *   thread.  Sec. 3.2 notes that Phase 1 is then Algorithm 1, so round 1
 *   colors the graph greedily and no conflict remains.
 *
 * The label of Algorithm 2 is the vertex v.  Because Algorithm 2 recolors a
 * vertex in several rounds, a label equal to v would let v meet its own
 * marks from an earlier round and skip colors that no neighbour holds; the
 * label here is (round, v), which keeps the array's never-cleared property
 * and gives the smallest permissible color the text of Sec. 3.1 defines.
 *
 * Outputs: color[n] (1-based), *ncolors = max color (0 for n == 0), *rounds
 * = number of while-loop iterations, round_sizes[r-1] = |U| at the start of
 * round r for r = 1..min(rounds, round_sizes_cap), and, if settle_round is
 * not NULL, settle_round[v] = the round after whose Phase 2 v left U for
 * good.  max_rounds <= 0 means n.  Returns ORC_ERR_MAX_ROUNDS if U is not
 * empty after max_rounds rounds.
 */
int orc_iterative(int32_t n, const int32_t* rowptr, const int32_t* colidx, const uint32_t* prio,
                  int32_t mode, int32_t max_rounds, int32_t* color, int32_t* ncolors,
                  int32_t* rounds, int32_t* round_sizes, int32_t round_sizes_cap,
                  int32_t* settle_round) {
    if (n < 0 || !color || !ncolors || !rounds || (n > 0 && (!rowptr || !colidx))) return ORC_ERR_INVALID;
    if (mode != 0 && mode != 1) return ORC_ERR_INVALID;
    if (max_rounds <= 0) max_rounds = n;
    const int64_t delta = max_degree(n, rowptr);

    /* Initialize data structures */
    int64_t* forbiddenColors = (int64_t*)malloc((size_t)(delta + 2) * sizeof(int64_t));
    int32_t* snapshot = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t* U = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int32_t* R = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    if (!forbiddenColors || !snapshot || !U || !R) {
        free(forbiddenColors); free(snapshot); free(U); free(R);
        return ORC_ERR_OOM;
    }
    for (int64_t i = 0; i < delta + 2; ++i) forbiddenColors[i] = -1;
    for (int32_t v = 0; v < n; ++v) color[v] = 0;

    /* U <- V, listed in precedence order (index order when prio is NULL) */
    int32_t nU = n;
    for (int32_t v = 0; v < n; ++v) U[v] = v;
    if (prio) {
        /* bottom-up merge sort of U by precedence */
        int32_t* tmp = R;
        for (int64_t width = 1; width < n; width *= 2) {
            for (int64_t lo = 0; lo < n; lo += 2 * width) {
                int64_t mid = lo + width < n ? lo + width : n;
                int64_t hi = lo + 2 * width < n ? lo + 2 * width : n;
                int64_t i = lo, j = mid, k = lo;
                while (i < mid && j < hi) tmp[k++] = precedes(U[j], U[i], prio) ? U[j++] : U[i++];
                while (i < mid) tmp[k++] = U[i++];
                while (j < hi) tmp[k++] = U[j++];
            }
            memcpy(U, tmp, (size_t)n * sizeof(int32_t));
        }
    }

    int32_t r = 0;
    int rc = ORC_OK;
    while (nU > 0) {
        if (r == max_rounds) { rc = ORC_ERR_MAX_ROUNDS; break; }
        r += 1;
        if (round_sizes && r <= round_sizes_cap) round_sizes[r - 1] = nU;

        /* colors Phase 1 reads: the previous round's (mode 0) or live (mode 1) */
        const int32_t* seen = color;
        if (mode == 0) {
            memcpy(snapshot, color, (size_t)n * sizeof(int32_t));
            seen = snapshot;
        }

        /* Phase 1: tentative coloring.  The mark is unique to this round and
         * vertex: a vertex recolored in a later round must not meet the marks
         * it left in an earlier one (the smallest permissible color of
         * Sec. 3.1 is the smallest color no neighbour holds now). */
        for (int32_t k = 0; k < nU; ++k) {
            const int32_t v = U[k];
            const int64_t label = (int64_t)r * (int64_t)n + v;
            for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                const int32_t w = colidx[e];
                forbiddenColors[seen[w]] = label;
            }
            int32_t c = 1;
            while (forbiddenColors[c] == label) ++c;
            color[v] = c;
        }

        /* Phase 2: conflict detection */
        int32_t nR = 0;
        for (int32_t k = 0; k < nU; ++k) {
            const int32_t v = U[k];
            int conflict = 0;
            for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
                const int32_t w = colidx[e];
                if (color[v] == color[w] && precedes(w, v, prio)) conflict = 1;
            }
            if (conflict) R[nR++] = v;
            else if (settle_round) settle_round[v] = r;
        }

        /* U <- R */
        memcpy(U, R, (size_t)nR * sizeof(int32_t));
        nU = nR;
    }
    int32_t mx = 0;
    for (int32_t v = 0; v < n; ++v)
        if (color[v] > mx) mx = color[v];
    *ncolors = mx;
    *rounds = r;
    free(forbiddenColors); free(snapshot); free(U); free(R);
    return rc;
}

/*
 * Chromatic number by exhaustive backtracking (vertices in index order,
 * colors tried in increasing order, k = 1, 2, ... until a proper k-coloring
 * exists).  For tiny graphs only (n <= 20).
 */
static int try_color(int32_t v, int32_t n, const int32_t* rowptr, const int32_t* colidx,
                     int32_t k, int32_t* col) {
    if (v == n) return 1;
    for (int32_t c = 1; c <= k; ++c) {
        int ok = 1;
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            int32_t w = colidx[e];
            if (w < v && col[w] == c) { ok = 0; break; }
        }
        if (!ok) continue;
        col[v] = c;
        if (try_color(v + 1, n, rowptr, colidx, k, col)) return 1;
        col[v] = 0;
    }
    return 0;
}

int orc_chromatic_number(int32_t n, const int32_t* rowptr, const int32_t* colidx, int32_t* chi) {
    if (n < 0 || n > 20 || !chi || (n > 0 && (!rowptr || !colidx))) return ORC_ERR_INVALID;
    if (n == 0) { *chi = 0; return ORC_OK; }
    int32_t col[20];
    for (int32_t k = 1; k <= n; ++k) {
        for (int32_t v = 0; v < n; ++v) col[v] = 0;
        if (try_color(0, n, rowptr, colidx, k, col)) { *chi = k; return ORC_OK; }
    }
    return ORC_ERR_INVALID; /* unreachable for a simple graph */
}

/* ---------------------------------------------------------- orderings */

/*
 * Largest-degree-first ordering: degree descending, ties by smaller index.
 * One of the ordering heuristics the paper cites for Greedy (Sec. 1, Sec. 3.1).
 */
int orc_largest_first_order(int32_t n, const int32_t* rowptr, int32_t* order) {
    if (n < 0 || !order || (n > 0 && !rowptr)) return ORC_ERR_INVALID;
    /* counting sort by degree, descending; stable in index */
    const int64_t delta = max_degree(n, rowptr);
    int64_t* cnt = (int64_t*)calloc((size_t)(delta + 2), sizeof(int64_t));
    if (!cnt) return ORC_ERR_OOM;
    for (int32_t v = 0; v < n; ++v) cnt[delta - (rowptr[v + 1] - rowptr[v]) + 1]++;
    for (int64_t d = 0; d <= delta; ++d) cnt[d + 1] += cnt[d];
    for (int32_t v = 0; v < n; ++v) order[cnt[delta - (rowptr[v + 1] - rowptr[v])]++] = v;
    free(cnt);
    return ORC_OK;
}

/* binary min-heap of (key, vertex) with lazy deletion */
typedef struct { int64_t key; int32_t v; } heap_item;

static int item_less(heap_item a, heap_item b) {
    return a.key < b.key || (a.key == b.key && a.v < b.v);
}

static void heap_push(heap_item* h, int64_t* size, heap_item x) {
    int64_t i = (*size)++;
    h[i] = x;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!item_less(h[i], h[p])) break;
        heap_item t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}

static heap_item heap_pop(heap_item* h, int64_t* size) {
    heap_item top = h[0];
    h[0] = h[--(*size)];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < *size && item_less(h[l], h[s])) s = l;
        if (r < *size && item_less(h[r], h[s])) s = r;
        if (s == i) break;
        heap_item t = h[i]; h[i] = h[s]; h[s] = t;
        i = s;
    }
    return top;
}

/*
 * Smallest-last ordering (Matula and Beck; cited in Sec. 1 and Sec. 3.1):
 * repeatedly remove a vertex of minimum degree in the remaining graph (ties:
 * smaller index); the ordering is the reverse of the removal sequence.
 * Optionally returns the degeneracy-style back degree of each vertex: its
 * degree in the remaining graph when it was removed.
 */
int orc_smallest_last_order(int32_t n, const int32_t* rowptr, const int32_t* colidx,
                            int32_t* order, int32_t* removal_degree) {
    if (n < 0 || !order || (n > 0 && (!rowptr || !colidx))) return ORC_ERR_INVALID;
    int64_t* deg = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    char* removed = (char*)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t cap = (int64_t)n + (n > 0 ? rowptr[n] : 0) + 1;
    heap_item* h = (heap_item*)malloc((size_t)cap * sizeof(heap_item));
    if (!deg || !removed || !h) { free(deg); free(removed); free(h); return ORC_ERR_OOM; }
    int64_t size = 0;
    for (int32_t v = 0; v < n; ++v) {
        deg[v] = rowptr[v + 1] - rowptr[v];
        heap_item it = { deg[v], v };
        heap_push(h, &size, it);
    }
    int32_t k = n;
    while (size > 0) {
        heap_item it = heap_pop(h, &size);
        if (removed[it.v] || it.key != deg[it.v]) continue; /* stale entry */
        const int32_t v = it.v;
        removed[v] = 1;
        order[--k] = v;
        if (removal_degree) removal_degree[v] = (int32_t)deg[v];
        for (int32_t e = rowptr[v]; e < rowptr[v + 1]; ++e) {
            const int32_t w = colidx[e];
            if (removed[w]) continue;
            deg[w] -= 1;
            heap_item nw = { deg[w], w };
            heap_push(h, &size, nw);
        }
    }
    free(deg); free(removed); free(h);
    return ORC_OK;
}
