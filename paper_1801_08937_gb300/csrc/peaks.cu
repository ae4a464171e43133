// Measured CUDA-core FMA rates of the device (float32 and float64), the
// denominators of the arithmetic view of the filter kernels' roofline.  Not a
// step of the map-making method: a calibration the benchmark runs beside it.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/mapmaker.h"
#include "common.cuh"

namespace mm {

// CH independent FMA chains per thread, UNROLL chain steps per loop trip: enough
// independent work per warp to keep the FMA pipes busy at full occupancy.
template <typename T, int CH, int UNROLL>
__global__ void __launch_bounds__(256) k_fma_rate(T* out, int trips, T a, T b) {
    T x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = T(threadIdx.x + c) * T(1e-3);
#pragma unroll 1
    for (int t = 0; t < trips; ++t) {
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
#pragma unroll
            for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
    }
    T s = T(0);
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    if (s == T(12345.678)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

template <typename T>
static mm_status fma_rate(int device, double seconds, double* flops_per_s) {
    constexpr int CH = 8, UNROLL = 16, NT = 256;
    int n_sm = 0;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return MM_ERR_CUDA;
    const int grid = n_sm * 8;   // 2048 threads per SM
    T* out = nullptr;
    if (cudaMalloc(&out, (size_t)grid * NT * sizeof(T)) != cudaSuccess) return MM_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // a short run sizes the timed one to about `seconds`
    int trips = 1000;
    float ms = 0.f;
    mm_status st = MM_OK;
    for (int pass = 0; pass < 3 && st == MM_OK; ++pass) {
        cudaEventRecord(e0);
        k_fma_rate<T, CH, UNROLL><<<grid, NT>>>(out, trips, T(0.999999), T(1e-7));
        cudaEventRecord(e1);
        if (cudaEventSynchronize(e1) != cudaSuccess) st = MM_ERR_CUDA;
        cudaEventElapsedTime(&ms, e0, e1);
        if (pass < 2 && ms > 0.f) {
            const double scale = std::max(1.0, seconds * 1e3 / ms);
            trips = (int)std::min(2.0e9, trips * scale);
        }
    }
    if (st == MM_OK && cudaGetLastError() != cudaSuccess) st = MM_ERR_CUDA;
    const double flops = 2.0 * CH * UNROLL * (double)trips * grid * NT;
    *flops_per_s = ms > 0.f ? flops / (ms * 1e-3) : 0.0;
    count_launches(3);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    return st;
}

}  // namespace mm

extern "C" mm_status mm_fma_peak(int device, int fp64, double seconds, double* flops_per_s) {
    if (!flops_per_s || !(seconds > 0.0) || seconds > 60.0) return MM_ERR_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    const mm_status st = fp64 ? mm::fma_rate<double>(device, seconds, flops_per_s)
                              : mm::fma_rate<float>(device, seconds, flops_per_s);
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}
