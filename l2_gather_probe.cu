// Ceiling probe: random 16-bit gathers from a table, driven by a streamed
// int32 index array (the access pattern of a coloring round: stream an
// adjacency list, gather each neighbour's color).  Prints gathers per second
// for table sizes from L2-resident down to L1-sized, and for shared memory.
// Built and run by `python bench.py --measure-l2-ceiling`.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <vector>

__global__ void gather_global(const int* __restrict__ idx, const uint16_t* tab, long long m,
                              unsigned* out, int cached) {
    unsigned acc = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride * 4) {
        int w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long j = i + u * stride;
            w[u] = j < m ? __ldg(idx + j) : -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (w[u] >= 0) acc ^= cached ? __ldg(tab + w[u]) : __ldcg(tab + w[u]);
    }
    // a condition the compiler cannot decide keeps the gathers alive
    if (acc == (unsigned)m) out[0] = acc;
}

__global__ void gather_smem(const int* __restrict__ idx, const uint16_t* tab, int N, long long m,
                            unsigned* out) {
    extern __shared__ uint16_t s[];
    for (int i = threadIdx.x; i < N; i += blockDim.x) s[i] = tab[i];
    __syncthreads();
    unsigned acc = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride * 4) {
        int w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long j = i + u * stride;
            w[u] = j < m ? __ldg(idx + j) : -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (w[u] >= 0) acc ^= s[w[u] % N];
    }
    if (acc == (unsigned)m) out[0] = acc;
}

int main() {
    const long long m = 128ll << 20;        // 134M indices (512 MB, larger than L2)
    const long long tab_max = 16ll << 20;   // 16M entries (32 MB)
    int *idx = nullptr;
    uint16_t* tab = nullptr;
    unsigned* out = nullptr;
    char* flush = nullptr;
    if (cudaMalloc(&idx, m * 4) != cudaSuccess || cudaMalloc(&tab, tab_max * 2) != cudaSuccess ||
        cudaMalloc(&out, 4) != cudaSuccess || cudaMalloc(&flush, 256 << 20) != cudaSuccess) {
        std::printf("allocation failed\n");
        return 1;
    }
    cudaMemset(tab, 1, tab_max * 2);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    std::vector<int> h(m);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    for (long long N : {16777216ll, 1048576ll, 131072ll, 65536ll}) {
        unsigned long long x = 88172645463325252ull;  // xorshift64
        for (long long i = 0; i < m; ++i) {
            x ^= x << 13; x ^= x >> 7; x ^= x << 17;
            h[i] = (int)(x % (unsigned long long)N);
        }
        cudaMemcpy(idx, h.data(), m * 4, cudaMemcpyHostToDevice);
        for (int mode = 0; mode < 2; ++mode) {
            float best = 1e30f;
            for (int r = 0; r < 4; ++r) {
                cudaMemset(flush, r, 256 << 20);
                cudaEventRecord(a);
                gather_global<<<sms * 8, 256>>>(idx, tab, m, out, mode);
                cudaEventRecord(b);
                cudaEventSynchronize(b);
                float ms = 0;
                cudaEventElapsedTime(&ms, a, b);
                if (r) best = ms < best ? ms : best;
            }
            std::printf("table %9lld entries (%6.0f KB) %-10s %8.3f ms %7.1f G gathers/s\n", N, N * 2 / 1024.0,
                        mode ? "L1-cached" : "L2 (.cg)", best, m / best / 1e6);
        }
        if (N * 2 <= 200 * 1024) {
            cudaFuncSetAttribute(gather_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(N * 2));
            float best = 1e30f;
            for (int r = 0; r < 4; ++r) {
                cudaMemset(flush, r, 256 << 20);
                cudaEventRecord(a);
                gather_smem<<<sms, 1024, N * 2>>>(idx, tab, (int)N, m, out);
                cudaEventRecord(b);
                cudaEventSynchronize(b);
                float ms = 0;
                cudaEventElapsedTime(&ms, a, b);
                if (r) best = ms < best ? ms : best;
            }
            std::printf("table %9lld entries (%6.0f KB) %-10s %8.3f ms %7.1f G gathers/s\n", N, N * 2 / 1024.0,
                        "shared", best, m / best / 1e6);
        }
    }
    std::printf("status %s\n", cudaGetErrorString(cudaGetLastError()));
    return 0;
}
