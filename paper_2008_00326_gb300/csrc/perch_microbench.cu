// Shared-memory atomicMin throughput of this device, for the rasteriser's
// roofline (its z-buffer is a shared-memory atomicMin per covered sample).
// Not part of the method: a measurement helper.
#include "perch.h"

#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kBytes = 32768;     // each block's target array
constexpr int kThreads = 256;
constexpr int kIters = 2048;

template <typename T>
__global__ void __launch_bounds__(kThreads) k_smem_atomic_min(T* sink)
{
    constexpr int kWords = kBytes / (int)sizeof(T);
    __shared__ T buf[kWords];
    for (int i = threadIdx.x; i < kWords; i += kThreads) buf[i] = ~T(0);
    __syncthreads();
    uint32_t x = (blockIdx.x * kThreads + threadIdx.x) * 2654435761u + 1u;
    for (int i = 0; i < kIters; ++i) {
        x ^= x << 13;
        x ^= x >> 17;
        x ^= x << 5;
        atomicMin(&buf[x & (kWords - 1)], (T)x);
    }
    __syncthreads();
    if (threadIdx.x == 0) sink[blockIdx.x] = buf[blockIdx.x & (kWords - 1)];
}

template <typename T>
perch_status rate(int sms, double* out)
{
    const int grid = sms * 8;
    T* sink = nullptr;
    if (cudaMalloc(&sink, sizeof(T) * grid) != cudaSuccess) {
        cudaGetLastError();
        return PERCH_E_NOMEM;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (!e) e = cudaEventCreate(&e1);
    if (!e) {
        k_smem_atomic_min<T><<<grid, kThreads>>>(sink);            // warm-up
        e = cudaEventRecord(e0);
    }
    const int reps = 5;
    for (int r = 0; r < reps && !e; ++r) k_smem_atomic_min<T><<<grid, kThreads>>>(sink);
    if (!e) e = cudaEventRecord(e1);
    if (!e) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (!e) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    if (e || ms <= 0.0f) {
        cudaGetLastError();
        return PERCH_E_CUDA;
    }
    *out = (double)reps * grid * kThreads * kIters / (ms * 1e-3);
    return PERCH_OK;
}

}  // namespace

extern "C" perch_status perch_measure_smem_atomics(int32_t device, double* u32_per_s, double* u64_per_s)
{
    if (!u32_per_s || !u64_per_s) return PERCH_E_INVALID;
    int prev = -1, sms = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return PERCH_E_INVALID;
    }
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    perch_status st = rate<unsigned int>(sms, u32_per_s);
    if (st == PERCH_OK) st = rate<unsigned long long>(sms, u64_per_s);
    cudaSetDevice(prev);
    return st;
}
