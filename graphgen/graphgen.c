/*
 * Seeded synthetic graph generators: R-MAT, G(n,m), 2-D 5-point grids and
 * random geometric graphs, all returned as a simple symmetric int32 CSR
 * (no self loops, no duplicate entries, every row sorted ascending).
 *
 * This file holds no arithmetic of the coloring method.  It produces the
 * inputs that both the CUDA path and the CPU oracle consume.
 *
 * Randomness is counter based: draw i of stream s under seed k is
 * SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) started from a per-(k, s) state.  Every value is
 * a pure function of (k, s, i), so the output does not depend on the number
 * of threads, and integer-only decisions make it identical on x86-64 and
 * aarch64.  The random geometric generator compares doubles; it is compiled
 * with -ffp-contract=off so that no fused multiply-add changes a decision.
 *
 * R-MAT follows Sec. 4.1 of Catalyurek et al. (arXiv 1205.3809): each edge
 * sample descends `scale` levels of the adjacency matrix, choosing quadrant
 * (1,1), (1,2), (2,1), (2,2) with probabilities a, b, c, d; duplicates and
 * self loops are removed afterwards (Sec. 4.1), and vertex ids are shuffled
 * at random (Sec. 5.1) through a keyed Feistel bijection.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GG_OK 0
#define GG_ERR_INVALID -1
#define GG_ERR_OOM -3
#define GG_ERR_TOO_LARGE -7

static const uint64_t SM_GAMMA = 0x9E3779B97F4A7C15ULL;

static inline uint64_t sm_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Initial SplitMix64 state of stream `stream` under `seed`. */
static inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
    return sm_mix(sm_mix(seed + SM_GAMMA) ^ (stream * 0xD1B54A32D192ED03ULL + 1ULL));
}

/* Draw number i (0-based) of the SplitMix64 sequence that starts at `key`. */
static inline uint64_t draw(uint64_t key, uint64_t i) {
    return sm_mix(key + (i + 1ULL) * SM_GAMMA);
}

uint64_t gg_draw(uint64_t seed, uint64_t stream, uint64_t i) {
    return draw(stream_key(seed, stream), i);
}

/* Stream ids, one per purpose, so that no two decisions share draws. */
enum { ST_RMAT = 1, ST_PERM = 2, ST_GNM = 3, ST_RGG = 4 };

/* ---------------------------------------------------------------- perm */

/* Balanced 4-round Feistel network on 2*half bits, keyed by `key`.  A Feistel
 * network is a bijection for any round function; cycle walking restricts it
 * to a bijection of [0, n). */
static inline uint64_t feistel(uint64_t x, int half, uint64_t key) {
    const uint64_t mask = (half >= 64) ? ~0ULL : ((1ULL << half) - 1ULL);
    uint64_t L = x >> half, R = x & mask;
    for (uint64_t round = 0; round < 4; ++round) {
        uint64_t F = sm_mix(key ^ (R * SM_GAMMA) ^ (round << 56)) & mask;
        uint64_t nL = R;
        R = L ^ F;
        L = nL;
    }
    return (L << half) | R;
}

static int perm_half_bits(uint64_t n) {
    int bits = 1;
    while (bits < 62 && (1ULL << bits) < n) ++bits;
    return (bits + 1) / 2;
}

static inline uint64_t perm_apply(uint64_t i, uint64_t n, int half, uint64_t key) {
    uint64_t x = feistel(i, half, key);
    while (x >= n) x = feistel(x, half, key);
    return x;
}

/* Random permutation of [0, n): out[i] = image of i. */
int gg_permutation(int64_t n, uint64_t seed, int32_t* out) {
    if (n < 0 || n > INT32_MAX || (n > 0 && !out)) return GG_ERR_INVALID;
    const uint64_t key = stream_key(seed, ST_PERM);
    const int half = perm_half_bits((uint64_t)n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) out[i] = (int32_t)perm_apply((uint64_t)i, (uint64_t)n, half, key);
    return GG_OK;
}

/* ----------------------------------------------------------------- CSR */

static void sort_i32(int32_t* a, int64_t len);

static int cmp_i32(const void* x, const void* y) {
    int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
    return (a > b) - (a < b);
}

static void sort_i32(int32_t* a, int64_t len) {
    if (len < 24) {
        for (int64_t i = 1; i < len; ++i) {
            int32_t x = a[i];
            int64_t j = i - 1;
            while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
            a[j + 1] = x;
        }
    } else {
        qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

/*
 * Simple symmetric CSR from an undirected edge multiset (eu[k], ev[k]):
 * self loops dropped, both directions inserted, rows sorted, duplicates
 * dropped.  On success *rowptr_out (n+1) and *colidx_out (*nnz_out) are
 * malloc'd and owned by the caller (release with gg_free).
 */
static int csr_build(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev,
                     int32_t** rowptr_out, int32_t** colidx_out, int64_t* nnz_out) {
    int64_t* off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!off) return GG_ERR_OOM;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m; ++k) {
        int32_t u = eu[k], v = ev[k];
        if (u == v) continue;
#pragma omp atomic
        off[u + 1]++;
#pragma omp atomic
        off[v + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) off[v + 1] += off[v];
    const int64_t raw = off[n];
    int32_t* tmp = (int32_t*)malloc((size_t)(raw > 0 ? raw : 1) * sizeof(int32_t));
    int64_t* cur = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!tmp || !cur) { free(off); free(tmp); free(cur); return GG_ERR_OOM; }
    memcpy(cur, off, (size_t)n * sizeof(int64_t));
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m; ++k) {
        int32_t u = eu[k], v = ev[k];
        if (u == v) continue;
        int64_t pu, pv;
#pragma omp atomic capture
        pu = cur[u]++;
#pragma omp atomic capture
        pv = cur[v]++;
        tmp[pu] = v;
        tmp[pv] = u;
    }
    free(cur);
    /* sort and deduplicate each row in place; keep the unique count */
    int64_t* ndeg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    if (!ndeg) { free(off); free(tmp); return GG_ERR_OOM; }
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < n; ++v) {
        int32_t* row = tmp + off[v];
        int64_t len = off[v + 1] - off[v];
        sort_i32(row, len);
        int64_t u = 0;
        for (int64_t i = 0; i < len; ++i)
            if (u == 0 || row[u - 1] != row[i]) row[u++] = row[i];
        ndeg[v + 1] = u;
    }
    for (int64_t v = 0; v < n; ++v) ndeg[v + 1] += ndeg[v];
    const int64_t nnz = ndeg[n];
    if (nnz > INT32_MAX) { free(off); free(tmp); free(ndeg); return GG_ERR_TOO_LARGE; }
    int32_t* rowptr = (int32_t*)malloc((size_t)(n + 1) * sizeof(int32_t));
    int32_t* colidx = (int32_t*)malloc((size_t)(nnz > 0 ? nnz : 1) * sizeof(int32_t));
    if (!rowptr || !colidx) { free(off); free(tmp); free(ndeg); free(rowptr); free(colidx); return GG_ERR_OOM; }
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t v = 0; v < n; ++v) {
        int64_t len = ndeg[v + 1] - ndeg[v];
        memcpy(colidx + ndeg[v], tmp + off[v], (size_t)len * sizeof(int32_t));
    }
    for (int64_t v = 0; v <= n; ++v) rowptr[v] = (int32_t)ndeg[v];
    free(off); free(tmp); free(ndeg);
    *rowptr_out = rowptr;
    *colidx_out = colidx;
    *nnz_out = nnz;
    return GG_OK;
}

int gg_csr_from_edges(int64_t n, int64_t m, const int32_t* eu, const int32_t* ev,
                      int32_t** rowptr_out, int32_t** colidx_out, int64_t* nnz_out) {
    if (n < 0 || n > INT32_MAX || m < 0 || !rowptr_out || !colidx_out || !nnz_out) return GG_ERR_INVALID;
    for (int64_t k = 0; k < m; ++k)
        if (eu[k] < 0 || eu[k] >= n || ev[k] < 0 || ev[k] >= n) return GG_ERR_INVALID;
    return csr_build(n, m, eu, ev, rowptr_out, colidx_out, nnz_out);
}

void gg_free(void* p) { free(p); }

/* --------------------------------------------------------------- R-MAT */

static uint64_t prob_threshold(double p) {
    if (p <= 0.0) return 0;
    if (p >= 1.0) return 1ULL << 32;
    return (uint64_t)llround(p * 4294967296.0);
}

/*
 * R-MAT (Sec. 4.1): 2^scale vertices, edge_factor * 2^scale edge samples.
 * Edge sample k reads draws k*ceil(scale/2) ... of the R-MAT stream; each
 * 64-bit draw gives two 32-bit uniforms, one per level, most significant
 * level first.  A uniform u picks quadrant (1,1) if u < a, (1,2) if u < a+b,
 * (2,1) if u < a+b+c, else (2,2).  Quadrant (i,j) sets row bit i-1 and
 * column bit j-1.  With permute != 0 both endpoints go through the random
 * vertex-id shuffle of Sec. 5.1.
 */
int gg_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c, double d,
            uint64_t seed, int32_t permute,
            int32_t** rowptr_out, int32_t** colidx_out, int64_t* nnz_out) {
    if (scale < 0 || scale > 30 || edge_factor < 0 || a < 0 || b < 0 || c < 0 || d < 0) return GG_ERR_INVALID;
    if (fabs(a + b + c + d - 1.0) > 1e-9) return GG_ERR_INVALID;
    const int64_t n = 1LL << scale;
    const int64_t m = (int64_t)edge_factor * n;
    const uint64_t tA = prob_threshold(a), tAB = prob_threshold(a + b), tABC = prob_threshold(a + b + c);
    const uint64_t key = stream_key(seed, ST_RMAT);
    const uint64_t pkey = stream_key(seed, ST_PERM);
    const int half = perm_half_bits((uint64_t)n);
    const int64_t per_edge = (scale + 1) / 2;
    int32_t* eu = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int32_t* ev = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (!eu || !ev) { free(eu); free(ev); return GG_ERR_OOM; }
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < m; ++k) {
        uint64_t row = 0, col = 0;
        for (int32_t l = 0; l < scale; ++l) {
            uint64_t x = draw(key, (uint64_t)(k * per_edge + l / 2));
            uint64_t u = (l & 1) ? (x >> 32) : (x & 0xFFFFFFFFULL);
            uint64_t rb, cb;
            if (u < tA) { rb = 0; cb = 0; }
            else if (u < tAB) { rb = 0; cb = 1; }
            else if (u < tABC) { rb = 1; cb = 0; }
            else { rb = 1; cb = 1; }
            row = (row << 1) | rb;
            col = (col << 1) | cb;
        }
        if (permute) {
            row = perm_apply(row, (uint64_t)n, half, pkey);
            col = perm_apply(col, (uint64_t)n, half, pkey);
        }
        eu[k] = (int32_t)row;
        ev[k] = (int32_t)col;
    }
    int rc = csr_build(n, m, eu, ev, rowptr_out, colidx_out, nnz_out);
    free(eu); free(ev);
    return rc;
}

/* -------------------------------------------------------------- G(n,m) */

/*
 * Uniform simple graph with exactly m undirected edges: candidate pairs come
 * from the G(n,m) stream in order; a pair is kept if it is not a self loop
 * and not already present.  Sequential, for small graphs.
 */
int gg_gnm(int64_t n, int64_t m, uint64_t seed,
           int32_t** rowptr_out, int32_t** colidx_out, int64_t* nnz_out) {
    if (n < 0 || n > INT32_MAX || m < 0) return GG_ERR_INVALID;
    if (m > 0 && (n < 2 || (double)m > (double)n * (double)(n - 1) / 2.0)) return GG_ERR_INVALID;
    int64_t cap = 16;
    while (cap < 4 * m + 16) cap <<= 1;
    uint64_t* table = (uint64_t*)malloc((size_t)cap * sizeof(uint64_t));
    int32_t* eu = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int32_t* ev = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (!table || !eu || !ev) { free(table); free(eu); free(ev); return GG_ERR_OOM; }
    for (int64_t i = 0; i < cap; ++i) table[i] = ~0ULL;
    const uint64_t key = stream_key(seed, ST_GNM);
    int64_t have = 0;
    for (uint64_t i = 0; have < m; ++i) {
        uint64_t x = draw(key, i);
        uint64_t u = (x & 0xFFFFFFFFULL) % (uint64_t)n, v = (x >> 32) % (uint64_t)n;
        if (u == v) continue;
        uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
        uint64_t k = (lo << 32) | hi;
        uint64_t h = sm_mix(k) & (uint64_t)(cap - 1);
        int dup = 0;
        while (table[h] != ~0ULL) {
            if (table[h] == k) { dup = 1; break; }
            h = (h + 1) & (uint64_t)(cap - 1);
        }
        if (dup) continue;
        table[h] = k;
        eu[have] = (int32_t)lo;
        ev[have] = (int32_t)hi;
        ++have;
    }
    free(table);
    int rc = csr_build(n, m, eu, ev, rowptr_out, colidx_out, nnz_out);
    free(eu); free(ev);
    return rc;
}

/* ------------------------------------------------------------- 2-D grid */

/* rows x cols 5-point mesh; vertex (i,j) = i*cols + j, optionally shuffled. */
int gg_grid2d(int64_t rows, int64_t cols, uint64_t seed, int32_t permute,
              int32_t** rowptr_out, int32_t** colidx_out, int64_t* nnz_out) {
    if (rows < 0 || cols < 0 || rows * cols > INT32_MAX) return GG_ERR_INVALID;
    const int64_t n = rows * cols;
    const int64_t m = (rows > 0 && cols > 0) ? rows * (cols - 1) + (rows - 1) * cols : 0;
    int32_t* eu = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int32_t* ev = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (!eu || !ev) { free(eu); free(ev); return GG_ERR_OOM; }
    const uint64_t pkey = stream_key(seed, ST_PERM);
    const int half = perm_half_bits((uint64_t)(n > 0 ? n : 1));
    int64_t k = 0;
    for (int64_t i = 0; i < rows; ++i)
        for (int64_t j = 0; j < cols; ++j) {
            int64_t v = i * cols + j;
            if (j + 1 < cols) { eu[k] = (int32_t)v; ev[k] = (int32_t)(v + 1); ++k; }
            if (i + 1 < rows) { eu[k] = (int32_t)v; ev[k] = (int32_t)(v + cols); ++k; }
        }
    if (permute)
        for (int64_t e = 0; e < m; ++e) {
            eu[e] = (int32_t)perm_apply((uint64_t)eu[e], (uint64_t)n, half, pkey);
            ev[e] = (int32_t)perm_apply((uint64_t)ev[e], (uint64_t)n, half, pkey);
        }
    int rc = csr_build(n, m, eu, ev, rowptr_out, colidx_out, nnz_out);
    free(eu); free(ev);
    return rc;
}

/* ------------------------------------------------ random geometric graph */

/*
 * n points uniform in the unit square (coordinates = 32-bit uniforms of the
 * RGG stream), an edge between every pair closer than `radius`.  Points are
 * bucketed in cells of side >= radius; ids follow draw order, which is
 * already random.
 */
int gg_rgg(int64_t n, double radius, uint64_t seed,
           int32_t** rowptr_out, int32_t** colidx_out, int64_t* nnz_out) {
    if (n < 0 || n > INT32_MAX || !(radius > 0.0) || radius > 1.0) return GG_ERR_INVALID;
    const uint64_t key = stream_key(seed, ST_RGG);
    double* px = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    double* py = (double*)malloc((size_t)(n > 0 ? n : 1) * sizeof(double));
    int64_t g = (int64_t)floor(1.0 / radius);
    if (g < 1) g = 1;
    if (g > 4096) g = 4096;
    int64_t* cell_off = (int64_t*)calloc((size_t)(g * g + 1), sizeof(int64_t));
    int32_t* cell_pts = (int32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int64_t* cid = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!px || !py || !cell_off || !cell_pts || !cid) {
        free(px); free(py); free(cell_off); free(cell_pts); free(cid); return GG_ERR_OOM;
    }
    for (int64_t i = 0; i < n; ++i) {
        uint64_t x = draw(key, (uint64_t)i);
        px[i] = (double)(x & 0xFFFFFFFFULL) / 4294967296.0;
        py[i] = (double)(x >> 32) / 4294967296.0;
        int64_t cx = (int64_t)(px[i] * (double)g), cy = (int64_t)(py[i] * (double)g);
        if (cx >= g) cx = g - 1;
        if (cy >= g) cy = g - 1;
        cid[i] = cy * g + cx;
        cell_off[cid[i] + 1]++;
    }
    for (int64_t c = 0; c < g * g; ++c) cell_off[c + 1] += cell_off[c];
    {
        int64_t* cur = (int64_t*)malloc((size_t)(g * g) * sizeof(int64_t));
        if (!cur) { free(px); free(py); free(cell_off); free(cell_pts); free(cid); return GG_ERR_OOM; }
        memcpy(cur, cell_off, (size_t)(g * g) * sizeof(int64_t));
        for (int64_t i = 0; i < n; ++i) cell_pts[cur[cid[i]]++] = (int32_t)i;
        free(cur);
    }
    const double r2 = radius * radius;
    int64_t cap = 1024, m = 0;
    int32_t* eu = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
    int32_t* ev = (int32_t*)malloc((size_t)cap * sizeof(int32_t));
    int rc = GG_OK;
    for (int64_t i = 0; i < n && rc == GG_OK; ++i) {
        int64_t cx = cid[i] % g, cy = cid[i] / g;
        for (int64_t dy = -1; dy <= 1 && rc == GG_OK; ++dy)
            for (int64_t dx = -1; dx <= 1 && rc == GG_OK; ++dx) {
                int64_t qx = cx + dx, qy = cy + dy;
                if (qx < 0 || qy < 0 || qx >= g || qy >= g) continue;
                int64_t c = qy * g + qx;
                for (int64_t t = cell_off[c]; t < cell_off[c + 1] && rc == GG_OK; ++t) {
                    int32_t j = cell_pts[t];
                    if (j <= i) continue;
                    double ddx = px[i] - px[j], ddy = py[i] - py[j];
                    if (ddx * ddx + ddy * ddy < r2) {
                        if (m == cap) {
                            cap *= 2;
                            int32_t* nu = (int32_t*)realloc(eu, (size_t)cap * sizeof(int32_t));
                            if (nu) eu = nu;
                            int32_t* nv = (int32_t*)realloc(ev, (size_t)cap * sizeof(int32_t));
                            if (nv) ev = nv;
                            if (!nu || !nv) { rc = GG_ERR_OOM; break; }
                        }
                        eu[m] = (int32_t)i;
                        ev[m] = j;
                        ++m;
                    }
                }
            }
    }
    if (rc == GG_OK) rc = csr_build(n, m, eu, ev, rowptr_out, colidx_out, nnz_out);
    free(px); free(py); free(cell_off); free(cell_pts); free(cid); free(eu); free(ev);
    return rc;
}

int gg_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
