// Allocation-free application of the two-level preconditioner.
//
// mm_apply_precond(MM_PRECOND_2L) allocates temporaries on every call (the
// padded copies of x and y and the reduction scratch of Z^T x).  This file
// gives callers that must not allocate device memory during the call a
// variant that reads and writes the caller's [nrhs][n_pix][3] arrays
// directly and keeps its reduction scratch in one fixed, file-scope device
// array.  Such callers include latency-critical serving loops (cudaMalloc and
// cudaFree can synchronise the whole device and can fail under memory
// pressure) and host applications or plug-ins whose device memory is owned
// by another allocator and that are not allowed to allocate themselves.
//
// The scratch array is g_noalloc_scratch below: NOALLOC_SCRATCH_DOUBLES
// float64 values (1 MiB), held by every GPU that loads the library until the
// process exits.  Every call on a device shares it and it keeps the last
// call's contents; the ticket counters are cleared at the start of each
// call, the rest is fully overwritten before it is read.  Calls that overlap
// on the GPU (two streams, or two host threads) race on it.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/mapmaker.h"
#include "common.cuh"

namespace mm {

bool ctx_coarse_view(mm_ctx* ctx, CoarseView* v);
void ctx_set_error(mm_ctx* ctx, const std::string& msg);

constexpr int NOALLOC_SCRATCH_DOUBLES = 1 << 17;   // 1 MiB
constexpr int NOALLOC_COUNTER_SLOTS = 128;         // first 64 doubles hold 128 unsigned tickets
constexpr int NOALLOC_COUNTER_DOUBLES = 64;
constexpr int NOALLOC_VT = 256;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    return v;
}

// t = Z^T x per right-hand side (x in the 3-wide layout), partial sums per
// CTA, then u = E^-1 t in the CTA that takes the last ticket.
__global__ void k_m2l_ztr3(const double* __restrict__ x, const V4<double>* __restrict__ Z,
                           const double* __restrict__ Einv, int k, int n_pix, int nrhs, double* partial,
                           double* u, unsigned* counter) {
    const int rhs = blockIdx.y;
    const double* xr = x + (int64_t)rhs * n_pix * 3;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = NOALLOC_VT / 32;
    const int chunk = (n_pix + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * chunk, i1 = min(n_pix, i0 + chunk);
    for (int c = warp; c < k; c += nw) {
        const V4<double>* zc = Z + (int64_t)c * n_pix;
        double s = 0.0;
        for (int i = i0 + lane; i < i1; i += 32) {
            const V4<double> zv = zc[i];
            s += zv.x * xr[3 * i] + zv.y * xr[3 * i + 1] + zv.z * xr[3 * i + 2];
        }
        s = na_warp_sum(s);
        if (lane == 0) partial[((int64_t)blockIdx.x * nrhs + rhs) * k + c] = s;
    }
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(counter + rhs, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    __shared__ double t[128];
    for (int c = threadIdx.x; c < k; c += NOALLOC_VT) {
        double s = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) s += __ldcg(partial + ((int64_t)b * nrhs + rhs) * k + c);
        t[c] = s;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += NOALLOC_VT) {
        double s = 0.0;
        for (int j = 0; j < k; ++j) s += Einv[c * k + j] * t[j];
        u[(int64_t)rhs * k + c] = s;
    }
    if (threadIdx.x == 0) counter[rhs] = 0;
}

// y = M_BD (x - AZ u) + Z u, both in the 3-wide layout.
__global__ void k_m2l_apply3(const double* __restrict__ x, double* __restrict__ y, const double* __restrict__ bd,
                             const V4<double>* __restrict__ Z, const V4<double>* __restrict__ AZ,
                             const double* __restrict__ u, int k, int n_pix) {
    const int rhs = blockIdx.y;
    __shared__ double us[128];
    for (int c = threadIdx.x; c < k; c += NOALLOC_VT) us[c] = u[(int64_t)rhs * k + c];
    __syncthreads();
    const double* xr = x + (int64_t)rhs * n_pix * 3;
    double* yr = y + (int64_t)rhs * n_pix * 3;
    for (int i = blockIdx.x * NOALLOC_VT + threadIdx.x; i < n_pix; i += gridDim.x * NOALLOC_VT) {
        double r0 = xr[3 * i], r1 = xr[3 * i + 1], r2 = xr[3 * i + 2];
        double z0 = 0.0, z1 = 0.0, z2 = 0.0;
        for (int c = 0; c < k; ++c) {
            const V4<double> a = AZ[(int64_t)c * n_pix + i];
            const V4<double> zc = Z[(int64_t)c * n_pix + i];
            const double uc = us[c];
            r0 -= a.x * uc;
            r1 -= a.y * uc;
            r2 -= a.z * uc;
            z0 += zc.x * uc;
            z1 += zc.y * uc;
            z2 += zc.z * uc;
        }
        const double* m = bd + (int64_t)i * 6;
        yr[3 * i] = m[0] * r0 + m[1] * r1 + m[2] * r2 + z0;
        yr[3 * i + 1] = m[1] * r0 + m[3] * r1 + m[4] * r2 + z1;
        yr[3 * i + 2] = m[2] * r0 + m[4] * r1 + m[5] * r2 + z2;
    }
}

// Device address of g_noalloc_scratch, looked up once per device with that
// device current and kept for the life of the process (like the library's
// contexts, it does not survive a cudaDeviceReset of that device).
constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

static cudaError_t noalloc_scratch(int device, double** out) {
    if (device < 0 || device >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[device] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[device];
    return cudaSuccess;
}

}  // namespace mm

using namespace mm;

extern "C" mm_status mm_apply_precond_2l_noalloc(mm_ctx* ctx, const double* x, double* y, int32_t nrhs) {
    CoarseView v{};
    if (!ctx || !ctx_coarse_view(ctx, &v)) return MM_ERR_ARG;
    if (!v.have_bd || v.k <= 0) {
        ctx_set_error(ctx, "mm_apply_precond_2l_noalloc: build M_BD and a coarse space first");
        return MM_ERR_STATE;
    }
    if (!x || !y || nrhs <= 0) {
        ctx_set_error(ctx, "mm_apply_precond_2l_noalloc: null array or nrhs <= 0");
        return MM_ERR_ARG;
    }
    const int64_t need_min = (int64_t)nrhs * v.k * 2;   // one CTA of partial sums plus u
    if (nrhs > NOALLOC_COUNTER_SLOTS || v.k > 128 ||
        NOALLOC_COUNTER_DOUBLES + need_min > NOALLOC_SCRATCH_DOUBLES) {
        ctx_set_error(ctx, "mm_apply_precond_2l_noalloc: nrhs * k exceeds the fixed scratch (nrhs <= 128, k <= 128, "
                           "2 * nrhs * k + 64 <= 131072 doubles)");
        return MM_ERR_ARG;
    }
    // the kernels take x and y as distinct arrays (__restrict__): overlapping ranges are refused
    const uintptr_t xb = reinterpret_cast<uintptr_t>(x), yb = reinterpret_cast<uintptr_t>(y);
    const uintptr_t bytes = (uintptr_t)nrhs * (uintptr_t)v.n_pix * 3u * sizeof(double);
    if (xb < yb + bytes && yb < xb + bytes) {
        ctx_set_error(ctx, "mm_apply_precond_2l_noalloc: x and y overlap (the call does not work in place)");
        return MM_ERR_ARG;
    }
    DeviceScope dev_scope(v.device);
    cudaError_t e = dev_scope.err;
    double* base = nullptr;
    if (e == cudaSuccess) e = noalloc_scratch(v.device, &base);
    if (e != cudaSuccess) {
        ctx_set_error(ctx, std::string("mm_apply_precond_2l_noalloc: ") + cudaGetErrorString(e));
        return MM_ERR_CUDA;
    }
    unsigned* counter = reinterpret_cast<unsigned*>(base);
    double* u = base + NOALLOC_COUNTER_DOUBLES;
    double* partial = u + (int64_t)nrhs * v.k;
    const int64_t room = NOALLOC_SCRATCH_DOUBLES - NOALLOC_COUNTER_DOUBLES - (int64_t)nrhs * v.k;
    int grid = v.grid_x;
    if ((int64_t)grid * nrhs * v.k > room) grid = (int)(room / ((int64_t)nrhs * v.k));
    if (grid < 1) grid = 1;
    e = cudaMemsetAsync(counter, 0, sizeof(unsigned) * nrhs, v.stream);
    if (e == cudaSuccess) {
        k_m2l_ztr3<<<dim3(grid, nrhs), NOALLOC_VT, 0, v.stream>>>(x, v.Z, v.Einv, v.k, v.n_pix, nrhs, partial, u,
                                                                   counter);
        k_m2l_apply3<<<dim3(v.grid_x, nrhs), NOALLOC_VT, 0, v.stream>>>(x, y, v.bd, v.Z, v.AZ, u, v.k, v.n_pix);
        count_launches(2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(v.stream);
    if (e != cudaSuccess) {
        ctx_set_error(ctx, std::string("mm_apply_precond_2l_noalloc: ") + cudaGetErrorString(e));
        return MM_ERR_CUDA;
    }
    return MM_OK;
}
