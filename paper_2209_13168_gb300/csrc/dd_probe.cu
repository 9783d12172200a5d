// Micro-benchmarks for the roofline denominators of the evaluation kernel:
// shared-memory atomic increments (with the returned previous value, as the
// IWE scatter uses them) at random cells of a tile-sized array, and
// streaming reads of a buffer that stays in L2 (a window's sorted events are
// read from L2, not HBM).  Each is timed with CUDA events on the given
// stream, best of several launches.
#include "../../include/dd.h"

#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr int PROBE_THREADS = 512;
constexpr int TILE_WORDS = 16 * 641;   // a 16-row band of a 640-pixel frame (odd pitch)
constexpr int ATOM_ITERS = 512;

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_atomics(unsigned long long* sink) {
    __shared__ uint32_t tile[TILE_WORDS];
    for (int i = threadIdx.x; i < TILE_WORDS; i += blockDim.x) tile[i] = 0u;
    __syncthreads();
    uint32_t h = (blockIdx.x * PROBE_THREADS + threadIdx.x) * 2654435761u + 12345u;
    unsigned long long S = 0;
    for (int i = 0; i < ATOM_ITERS; i++) {
        h ^= h << 13;                           // xorshift32 (Marsaglia 2003)
        h ^= h >> 17;
        h ^= h << 5;
        const uint32_t v = atomicAdd(&tile[h % TILE_WORDS], 1u);
        S += 2u * v + 1u;
    }
    if (S == 0xFFFFFFFFFFFFFFFFull) *sink = S;  // keeps the work; never true
}

__global__ void __launch_bounds__(PROBE_THREADS) k_probe_read(const uint4* __restrict__ a, size_t n, int reps,
                                                              unsigned long long* sink) {
    uint32_t x = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; r++)
        for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
            const uint4 v = __ldcg(&a[i]);
            x ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (x == 0xFFFFFFFFu) *sink = x;
}

}  // namespace

extern "C" int dd_probe_peaks(double* shared_atomics_per_s, double* l2_read_bytes_per_s, void* stream) {
    if (!shared_atomics_per_s || !l2_read_bytes_per_s) return DD_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_atomics, PROBE_THREADS, 0) != cudaSuccess)
        return DD_ERR_NO_DEVICE;
    const size_t bytes = (size_t)32 << 20;     // 32 MiB: resident in L2
    const int reps = 8;
    unsigned long long* sink = nullptr;
    uint4* buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = DD_OK;
    if (cudaMalloc((void**)&sink, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void**)&buf, bytes) != cudaSuccess) {
        rc = DD_ERR_OOM;
    } else if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
               cudaMemsetAsync(buf, 1, bytes, s) != cudaSuccess) {
        rc = DD_ERR_CUDA;
    }
    float best_a = 1e30f, best_r = 1e30f;
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    for (int k = 0; rc == DD_OK && k < 6; k++) {
        float ms = 0.0f;
        k_probe_atomics<<<blocks, PROBE_THREADS, 0, s>>>(sink);   // first launch of each pair warms up
        if (cudaEventRecord(e0, s) != cudaSuccess) rc = DD_ERR_CUDA;
        k_probe_atomics<<<blocks, PROBE_THREADS, 0, s>>>(sink);
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            rc = DD_ERR_CUDA;
        if (ms < best_a) best_a = ms;
        k_probe_read<<<sms * 4, PROBE_THREADS, 0, s>>>(buf, bytes / sizeof(uint4), 1, sink);
        if (cudaEventRecord(e0, s) != cudaSuccess) rc = DD_ERR_CUDA;
        k_probe_read<<<sms * 4, PROBE_THREADS, 0, s>>>(buf, bytes / sizeof(uint4), reps, sink);
        if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            rc = DD_ERR_CUDA;
        if (ms < best_r) best_r = ms;
    }
    if (rc == DD_OK && cudaGetLastError() != cudaSuccess) rc = DD_ERR_CUDA;
    if (rc == DD_OK) {
        *shared_atomics_per_s = (double)blocks * PROBE_THREADS * ATOM_ITERS / (best_a * 1e-3);
        *l2_read_bytes_per_s = (double)bytes * reps / (best_r * 1e-3);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (buf) cudaFree(buf);
    if (sink) cudaFree(sink);
    return rc;
}
