/*
 * Oracle for the learned vertex priority.  TEST INFRASTRUCTURE ONLY: tests,
 * the smoke check and the CPU baseline of the benchmark use it; the library
 * never does.  Plain single-threaded C, built with -ffp-contract=off so that
 * every product and sum is rounded exactly as written.
 *
 * The paper colors in index order (Sec. 3.2) and cites vertex orderings for
 * Greedy (smallest-last, largest-first: Sec. 1, Sec. 3.1).  The learned
 * priority replaces the index with a key computed per vertex:
 *   features (below) -> 6-32-32-1 ReLU network -> monotone float->uint32 key.
 * The network's arithmetic is fixed by its definition rather than by the
 * paper: operands rounded to bf16 (round to nearest, ties to even), every dot
 * product accumulated in fp32 with fused multiply-add in index order, biases
 * added in fp32.  The score decides an integer (the order of the keys), so
 * this oracle takes it in that same precision; a float64 form with the same
 * roundings lives in learned.py for the gradient.
 *
 * Pins (tests/test_oracle_learned.py): bf16 rounding against torch's
 * conversion; features in closed form on stars and paths and against a
 * scipy.sparse computation on random graphs; Mitchell's log exact at powers
 * of two and within its published error bound elsewhere; the forward against
 * a float64 torch network with the same roundings and a hand-worked case.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

enum { IN = 6, H = 32 };
enum { OFF_W1 = 0, OFF_B1 = OFF_W1 + H * IN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
       OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H, N_PARAMS = OFF_B3 + 1 };

int orc_mlp_param_count(void) { return N_PARAMS; }

/* bf16 value of x: keep the top 16 bits of the binary32 pattern, rounding the
 * dropped 16 to nearest with ties to the even kept pattern; NaN stays NaN. */
float orc_bf16(float x) {
    uint32_t u;
    memcpy(&u, &x, 4);
    if ((u & 0x7f800000u) == 0x7f800000u && (u & 0x007fffffu) != 0) {
        u |= 0x00400000u;  /* quiet NaN */
        u &= 0xffff0000u;
    } else {
        uint32_t dropped = u & 0xffffu;
        uint32_t kept = u >> 16;
        if (dropped > 0x8000u || (dropped == 0x8000u && (kept & 1u))) kept += 1u;
        u = kept << 16;
    }
    float r;
    memcpy(&r, &u, 4);
    return r;
}

/* Mitchell's log2(1 + x) (J. N. Mitchell, 1962): write m = 1 + x as 2^e (1 + f)
 * with 0 <= f < 1 and take e + f, with f truncated to 16 binary places. */
static float mitchell(uint64_t x) {
    uint64_t m = x + 1;
    int e = 0;
    while (e < 63 && (m >> (e + 1)) != 0) e++;
    unsigned __int128 rest = (unsigned __int128)(m - ((uint64_t)1 << e));
    uint64_t f16 = (uint64_t)((rest * 65536u) / ((unsigned __int128)1 << e));
    return (float)((double)e + (double)f16 / 65536.0);
}

/* Per-vertex features, six per vertex (deg = degree of v; the neighbour
 * statistics are over the degrees of v's neighbours):
 *   0: L(deg)   1: floor(log2(1 + deg))   2: L(floor(sum / deg))
 *   3: L(max)   4: L(sum)                 5: L(min)
 * with L = mitchell; 2..5 are 0 for an isolated vertex. */
int orc_features(int32_t n, const int32_t* rowptr, const int32_t* colidx, float* out) {
    if (n < 0) return -1;
    for (int32_t v = 0; v < n; ++v) {
        int64_t deg = (int64_t)rowptr[v + 1] - rowptr[v];
        uint64_t sum = 0;
        int64_t mx = 0, mn = 0;
        for (int64_t k = rowptr[v]; k < rowptr[v + 1]; ++k) {
            int32_t w = colidx[k];
            int64_t dw = (int64_t)rowptr[w + 1] - rowptr[w];
            sum += (uint64_t)dw;
            if (k == rowptr[v] || dw > mx) mx = dw;
            if (k == rowptr[v] || dw < mn) mn = dw;
        }
        float* f = out + (int64_t)v * IN;
        int lg = 0;
        while ((((uint64_t)deg + 1) >> (lg + 1)) != 0) lg++;
        f[0] = mitchell((uint64_t)deg);
        f[1] = (float)lg;
        if (deg > 0) {
            f[2] = mitchell(sum / (uint64_t)deg);
            f[3] = mitchell((uint64_t)mx);
            f[4] = mitchell(sum);
            f[5] = mitchell((uint64_t)mn);
        } else {
            f[2] = f[3] = f[4] = f[5] = 0.f;
        }
    }
    return 0;
}

static float relu(float z) { return z > 0.f ? z : 0.f; }

/* Network output for each of the n rows of x (6 floats per row):
 *   a0 = bf16(x); a1 = bf16(relu(bf16(W1) a0 + b1));
 *   a2 = bf16(relu(bf16(W2) a1 + b2)); y = bf16(W3) . a2 + b3.
 * Optional a1_out / a2_out receive the activations (32 per row). */
int orc_mlp_forward(const float* params, const float* x, int64_t n, float* y, float* a1_out,
                    float* a2_out) {
    if (n < 0) return -1;
    float w[N_PARAMS];
    for (int i = 0; i < N_PARAMS; ++i) {
        int is_bias = (i >= OFF_B1 && i < OFF_W2) || (i >= OFF_B2 && i < OFF_W3) || i == OFF_B3;
        w[i] = is_bias ? params[i] : orc_bf16(params[i]);
    }
    for (int64_t r = 0; r < n; ++r) {
        float a0[IN], a1[H], a2[H];
        for (int i = 0; i < IN; ++i) a0[i] = orc_bf16(x[r * IN + i]);
        for (int j = 0; j < H; ++j) {
            float z = 0.f;
            for (int i = 0; i < IN; ++i) z = fmaf(w[OFF_W1 + j * IN + i], a0[i], z);
            z = z + w[OFF_B1 + j];
            a1[j] = orc_bf16(relu(z));
        }
        for (int j = 0; j < H; ++j) {
            float z = 0.f;
            for (int i = 0; i < H; ++i) z = fmaf(w[OFF_W2 + j * H + i], a1[i], z);
            z = z + w[OFF_B2 + j];
            a2[j] = orc_bf16(relu(z));
        }
        float out = 0.f;
        for (int j = 0; j < H; ++j) out = fmaf(w[OFF_W3 + j], a2[j], out);
        y[r] = out + w[OFF_B3];
        if (a1_out) memcpy(a1_out + r * H, a1, sizeof a1);
        if (a2_out) memcpy(a2_out + r * H, a2, sizeof a2);
    }
    return 0;
}

/* orc_bf16 over an array. */
int orc_bf16_array(const float* x, int64_t n, float* out) {
    if (n < 0) return -1;
    for (int64_t i = 0; i < n; ++i) out[i] = orc_bf16(x[i]);
    return 0;
}
