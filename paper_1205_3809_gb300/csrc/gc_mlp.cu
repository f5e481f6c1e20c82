// Learned vertex priority: per-vertex features, a 6-32-32-1 ReLU MLP with
// bf16 operands and fp32 accumulation (forward, loss gradient, Adam), and
// the monotone map from a score to a uint32 key for gc_color's priority.
// The paper colors in index order (Sec. 3.2) and cites ordering heuristics
// for Greedy (smallest-last, largest-first: Sec. 1, Sec. 3.1); the network
// is trained to place a vertex where such an ordering would put it.
//
// Parameter vector (fp32 master copy, kMlpParams floats):
//   W1[32][6] | b1[32] | W2[32][32] | b2[32] | W3[32] | b3
// Forward, per sample x (6 features):
//   a0 = bf16(x); z1 = bf16(W1) a0 + b1; a1 = bf16(relu(z1));
//   z2 = bf16(W2) a1 + b2; a2 = bf16(relu(z2)); y = bf16(W3) . a2 + b3
// with every dot product accumulated in fp32 in index order (bf16 = round
// to nearest even).  The loss of a batch of B samples is mean (y - t)^2; its
// gradient uses the same bf16 weights and activations.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "gc.h"

namespace {

constexpr int kIn = 6, kH = 32;
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kH * kIn, kOffW2 = kOffB1 + kH, kOffB2 = kOffW2 + kH * kH,
              kOffW3 = kOffB2 + kH, kOffB3 = kOffW3 + kH, kMlpParams = kOffB3 + 1;
static_assert(kMlpParams == 1313, "parameter layout");
constexpr int kTile = 64;   // samples per tile of the gradient kernel (static shared memory < 48 KB)

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Parameters with the matrix operands rounded to bf16 (biases stay fp32).
__device__ __forceinline__ void load_params(const float* __restrict__ params, float* s) {
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
        const bool weight = i < kOffB1 || (i >= kOffW2 && i < kOffB2) || (i >= kOffW3 && i < kOffB3);
        const float p = params[i];
        s[i] = weight ? bf16r(p) : p;
    }
}

// Layer 1 of one sample: a1 = bf16(relu(bf16(W1) a0 + b1)).
__device__ __forceinline__ void layer1(const float* s, const float a0[kIn], float a1[kH]) {
#pragma unroll
    for (int j = 0; j < kH; ++j) {
        float acc = 0.f;
#pragma unroll
        for (int i = 0; i < kIn; ++i) acc = fmaf(s[kOffW1 + j * kIn + i], a0[i], acc);
        acc += s[kOffB1 + j];
        a1[j] = bf16r(fmaxf(acc, 0.f));
    }
}

// Unit j of layer 2: bf16(relu(bf16(W2[j]) . a1 + b2[j])).
__device__ __forceinline__ float layer2_unit(const float* s, const float a1[kH], int j) {
    float acc = 0.f;
#pragma unroll
    for (int i = 0; i < kH; ++i) acc = fmaf(s[kOffW2 + j * kH + i], a1[i], acc);
    acc += s[kOffB2 + j];
    return bf16r(fmaxf(acc, 0.f));
}

__global__ void __launch_bounds__(256) mlp_forward_kernel(const float* __restrict__ params,
                                                          const float* __restrict__ x, int64_t n,
                                                          float* __restrict__ y) {
    __shared__ __align__(16) float s[kMlpParams];
    load_params(params, s);
    __syncthreads();
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        float a0[kIn], a1[kH];
#pragma unroll
        for (int i = 0; i < kIn; ++i) a0[i] = bf16r(__ldg(x + r * kIn + i));
        layer1(s, a0, a1);
        // output = bf16(W3) . a2 + b3, accumulated in unit order
        float out = 0.f;
#pragma unroll 4
        for (int j = 0; j < kH; ++j) out = fmaf(s[kOffW3 + j], layer2_unit(s, a1, j), out);
        y[r] = out + s[kOffB3];
    }
}

// Gradient of scale * sum_b (y_b - t_b)^2 over n samples, added into grad;
// the sum of squared errors is added into *sse.  Rounding to bf16 passes
// gradients straight through, and the backward pass uses the same bf16
// weights and activations as the forward.  One block handles kTile samples at
// a time: forward and backward per sample (thread per sample) with
// activations and deltas staged in shared memory, then each thread sums the
// tile's contribution to the parameters it owns.
__global__ void __launch_bounds__(kTile) mlp_grad_kernel(const float* __restrict__ params,
                                                         const float* __restrict__ x,
                                                         const float* __restrict__ t, int64_t n,
                                                         float scale, float* grad, float* sse) {
    __shared__ float s[kMlpParams];
    __shared__ float g[kMlpParams];
    __shared__ float sa0[kTile][kIn + 1];
    __shared__ float sa1[kTile][kH + 1];
    __shared__ float sa2[kTile][kH + 1];
    __shared__ float sd1[kTile][kH + 1];
    __shared__ float sd2[kTile][kH + 1];
    __shared__ float sdy[kTile];
    __shared__ float s_sse;
    load_params(params, s);
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) g[i] = 0.f;
    if (threadIdx.x == 0) s_sse = 0.f;
    __syncthreads();
    float sse_local = 0.f;
    const int q = threadIdx.x;
    for (int64_t base = (int64_t)blockIdx.x * kTile; base < n; base += (int64_t)gridDim.x * kTile) {
        const int64_t r = base + q;
        const bool valid = r < n;
        float a0[kIn], a1[kH];
#pragma unroll
        for (int i = 0; i < kIn; ++i) {
            a0[i] = valid ? bf16r(x[r * kIn + i]) : 0.f;
            sa0[q][i] = a0[i];
        }
        layer1(s, a0, a1);
#pragma unroll
        for (int i = 0; i < kH; ++i) sa1[q][i] = a1[i];
        float out = 0.f;
#pragma unroll 4
        for (int j = 0; j < kH; ++j) {
            const float a2 = layer2_unit(s, a1, j);
            sa2[q][j] = a2;
            out = fmaf(s[kOffW3 + j], a2, out);
        }
        out += s[kOffB3];
        const float err = valid ? out - t[r] : 0.f;
        sse_local += err * err;
        const float dy = 2.f * scale * err;
        sdy[q] = dy;
        // relu masks: a > 0 exactly when z > 0 (rounding to bf16 keeps a positive value positive)
#pragma unroll
        for (int j = 0; j < kH; ++j) sd2[q][j] = sa2[q][j] > 0.f ? dy * s[kOffW3 + j] : 0.f;
#pragma unroll 4
        for (int i = 0; i < kH; ++i) {
            float acc = 0.f;
#pragma unroll
            for (int j = 0; j < kH; ++j) acc = fmaf(s[kOffW2 + j * kH + i], sd2[q][j], acc);
            sd1[q][i] = sa1[q][i] > 0.f ? acc : 0.f;
        }
        __syncthreads();
        // parameter gradients of this tile: sums over its samples
        for (int p = threadIdx.x; p < kMlpParams; p += blockDim.x) {
            float acc = 0.f;
            if (p < kOffB1) {
                const int j = p / kIn, i = p % kIn;
                for (int b = 0; b < kTile; ++b) acc = fmaf(sd1[b][j], sa0[b][i], acc);
            } else if (p < kOffW2) {
                const int j = p - kOffB1;
                for (int b = 0; b < kTile; ++b) acc += sd1[b][j];
            } else if (p < kOffB2) {
                const int j = (p - kOffW2) / kH, i = (p - kOffW2) % kH;
                for (int b = 0; b < kTile; ++b) acc = fmaf(sd2[b][j], sa1[b][i], acc);
            } else if (p < kOffW3) {
                const int j = p - kOffB2;
                for (int b = 0; b < kTile; ++b) acc += sd2[b][j];
            } else if (p < kOffB3) {
                const int i = p - kOffW3;
                for (int b = 0; b < kTile; ++b) acc = fmaf(sdy[b], sa2[b][i], acc);
            } else {
                for (int b = 0; b < kTile; ++b) acc += sdy[b];
            }
            g[p] += acc;
        }
        __syncthreads();
    }
    atomicAdd(&s_sse, sse_local);
    __syncthreads();
    for (int p = threadIdx.x; p < kMlpParams; p += blockDim.x) atomicAdd(&grad[p], g[p]);
    if (threadIdx.x == 0) atomicAdd(sse, s_sse);
}

// Adam (Kingma & Ba): m <- b1 m + (1-b1) g; v <- b2 v + (1-b2) g^2;
// p <- p - lr * (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps).
__global__ void mlp_adam_kernel(float* params, float* m, float* v, const float* grad, float lr,
                                float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const float gi = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    params[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Per-vertex features (deg = degree; nbr = the neighbours' degrees), every
// degree-like count on a log2 scale, since R-MAT degrees span five decades:
//   f0 = L(deg)                   f1 = floor(log2(1 + deg))
//   f2 = L(floor(sum nbr / deg))  f3 = L(max nbr)
//   f4 = L(sum nbr)               f5 = L(min nbr)
// (f2..f5 = 0 for an isolated vertex; sum nbr counts the walks of length 2).
// L(x) is Mitchell's piecewise-linear log2(1 + x) (J. N. Mitchell, 1962):
// with m = 1 + x = 2^e (1 + f), 0 <= f < 1, L = e + f, f truncated to 16
// bits.  It is exact in integer arithmetic, so every feature is an exact
// float, equal on any machine; it matches log2 at powers of two and is off by
// less than 0.087 elsewhere.
__device__ __forceinline__ float mitchell_log2_1p(unsigned long long x) {
    const unsigned long long m = x + 1ull;
    const int e = 63 - __clzll((long long)m);
    const unsigned long long r = m - (1ull << e);
    const unsigned long long frac = e >= 16 ? (r >> (e - 16)) : (r << (16 - e));
    return (float)((unsigned long long)e * 65536ull + frac) * (1.f / 65536.f);
}

__device__ __forceinline__ void write_features(float* f, int32_t d, unsigned long long sum, int32_t mx,
                                               int32_t mn) {
    f[0] = mitchell_log2_1p((unsigned long long)d);
    f[1] = (float)(31 - __clz(d + 1));
    if (d > 0) {
        f[2] = mitchell_log2_1p(sum / (unsigned long long)d);
        f[3] = mitchell_log2_1p((unsigned long long)mx);
        f[4] = mitchell_log2_1p(sum);
        f[5] = mitchell_log2_1p((unsigned long long)mn);
    } else {
        f[2] = f[3] = f[4] = f[5] = 0.f;
    }
}

__global__ void features_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                int32_t n, float* __restrict__ out) {
    const unsigned lane = threadIdx.x & 31u;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t W = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = gw * 32; base < n; base += W * 32) {
        const int64_t v = base + lane;
        const bool valid = v < n;
        const int32_t b = valid ? __ldg(rowptr + v) : 0, e = valid ? __ldg(rowptr + v + 1) : 0;
        const int32_t d = e - b;
        unsigned long long sum = 0;
        int32_t mx = 0, mn = 0x7fffffff;
        if (valid && d <= 32) {
            // eight entries at a time: their ids first, then their degrees, so that a
            // row costs two round trips per eight entries rather than per entry
            for (int32_t i = b; i < e; i += 8) {
                int32_t w[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) w[u] = i + u < e ? __ldg(colidx + i + u) : -1;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (w[u] >= 0) {
                        const int32_t dw = __ldg(rowptr + w[u] + 1) - __ldg(rowptr + w[u]);
                        sum += (unsigned long long)dw;
                        mx = max(mx, dw);
                        mn = min(mn, dw);
                    }
                }
            }
            write_features(out + v * 6, d, sum, mx, mn);
        }
        unsigned big = __ballot_sync(0xffffffffu, valid && d > 32);
        while (big) {
            const int j = __ffs(big) - 1;
            big &= big - 1;
            const int32_t jb = __shfl_sync(0xffffffffu, b, j), je = __shfl_sync(0xffffffffu, e, j);
            unsigned long long s2 = 0;
            int32_t x2 = 0, n2 = 0x7fffffff;
            for (int32_t i = jb + (int32_t)lane; i < je; i += 32) {
                const int32_t w = __ldg(colidx + i);
                const int32_t dw = __ldg(rowptr + w + 1) - __ldg(rowptr + w);
                s2 += (unsigned long long)dw;
                x2 = max(x2, dw);
                n2 = min(n2, dw);
            }
            for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            x2 = __reduce_max_sync(0xffffffffu, x2);
            n2 = __reduce_min_sync(0xffffffffu, n2);
            if ((int)lane == j) write_features(out + v * 6, d, s2, x2, n2);
        }
    }
}

// Score -> key with the same order: smaller score = smaller key (higher
// precedence).  IEEE order of floats is the order of their bit patterns
// with the sign bit flipped (positives) or all bits flipped (negatives).
__global__ void keys_kernel(const float* __restrict__ y, int64_t n, uint32_t* __restrict__ keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float f = y[i];
        if (f != f) f = __int_as_float(0x7f800000);  // NaN sorts last
        if (f == 0.f) f = 0.f;                        // -0 and +0 alike
        const uint32_t u = (uint32_t)__float_as_int(f);
        keys[i] = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    }
}

int grid_for(int64_t items, int per_block, int cap) {
    int64_t g = (items + per_block - 1) / per_block;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return (int)g;
}

int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
    return sms;
}

int check_launch() {
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GC_OK : GC_ERR_CUDA;
}

}  // namespace

extern "C" {

int gc_features(const int32_t* rowptr, const int32_t* colidx, int32_t n, float* features, void* stream) {
    if (n < 0 || (n > 0 && (!rowptr || !features))) return GC_ERR_INVALID;
    if (n == 0) return GC_OK;
    features_kernel<<<grid_for((int64_t)n, 256, sm_count() * 16), 256, 0, (cudaStream_t)stream>>>(
        rowptr, colidx, n, features);
    return check_launch();
}

int gc_mlp_forward(const float* params, const float* x, int64_t n, float* y, void* stream) {
    if (n < 0 || !params || (n > 0 && (!x || !y))) return GC_ERR_INVALID;
    if (n == 0) return GC_OK;
    mlp_forward_kernel<<<grid_for(n, 256, sm_count() * 8), 256, 0, (cudaStream_t)stream>>>(params, x, n, y);
    return check_launch();
}

int gc_mlp_grad(const float* params, const float* x, const float* t, int64_t n, float scale, float* grad,
                float* sse, void* stream) {
    if (n < 0 || !params || !grad || !sse || (n > 0 && (!x || !t))) return GC_ERR_INVALID;
    if (n == 0) return GC_OK;
    mlp_grad_kernel<<<grid_for(n, kTile, sm_count() * 4), kTile, 0, (cudaStream_t)stream>>>(
        params, x, t, n, scale, grad, sse);
    return check_launch();
}

int gc_mlp_adam(float* params, float* m, float* v, const float* grad, int32_t step, float lr, float beta1,
                float beta2, float eps, void* stream) {
    if (!params || !m || !v || !grad || step < 1) return GC_ERR_INVALID;
    const float c1 = 1.f - (float)std::pow((double)beta1, (double)step);
    const float c2 = 1.f - (float)std::pow((double)beta2, (double)step);
    mlp_adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, m, v, grad, lr, beta1,
                                                                                 beta2, eps, c1, c2);
    return check_launch();
}

int gc_priority_keys(const float* scores, int64_t n, uint32_t* keys, void* stream) {
    if (n < 0 || (n > 0 && (!scores || !keys))) return GC_ERR_INVALID;
    if (n == 0) return GC_OK;
    keys_kernel<<<grid_for(n, 256, sm_count() * 8), 256, 0, (cudaStream_t)stream>>>(scores, n, keys);
    return check_launch();
}

int gc_mlp_train_step(float* params, float* m, float* v, float* grad, float* sse, const float* x,
                      const float* t, int64_t n, int32_t step, float lr, float beta1, float beta2, float eps,
                      void* stream) {
    if (n < 1 || !params || !m || !v || !grad || !sse || !x || !t || step < 1) return GC_ERR_INVALID;
    const cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(grad, 0, sizeof(float) * kMlpParams, st) != cudaSuccess) return GC_ERR_CUDA;
    if (cudaMemsetAsync(sse, 0, sizeof(float), st) != cudaSuccess) return GC_ERR_CUDA;
    const int rc = gc_mlp_grad(params, x, t, n, 1.f / (float)n, grad, sse, stream);
    if (rc != GC_OK) return rc;
    return gc_mlp_adam(params, m, v, grad, step, lr, beta1, beta2, eps, stream);
}

int gc_mlp_param_count(void) { return kMlpParams; }

}  // extern "C"
