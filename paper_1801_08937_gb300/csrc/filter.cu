// Set-up kernels of the filter (spectra, pointing weights) and the launch counter.
#include "filter_impl.cuh"

namespace mm {

static long long g_launches = 0;
long long launches_total() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }
void count_launches(int n) { __atomic_fetch_add(&g_launches, (long long)n, __ATOMIC_RELAXED); }
std::mutex& smem_config_mutex() {
    static std::mutex m;
    return m;
}

// ---------------- setup kernels ----------------
__global__ void k_fft_spectrum(const double* h, double* H, C2<double>* work, const C2<double>* tw,
                               const FftPasses fp) {
    const int L = fp.L;
    C2<double>* s = work + (int64_t)blockIdx.x * (L + (L >> 4));
    const double* hb = h + (int64_t)blockIdx.x * L;
    for (int i = threadIdx.x; i < L; i += blockDim.x) s[sidx(i)] = C2<double>{hb[i], 0.0};
    __syncthreads();
    fft_dif<double>(s, tw, fp);
    const double inv = 1.0 / (double)L;
    for (int i = threadIdx.x; i < L; i += blockDim.x) H[(int64_t)blockIdx.x * L + i] = s[sidx(i)].x * inv;
}

__global__ void k_weights64(const float* psi, double2* cs, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        double sn, c;
        sincos(2.0 * (double)psi[t], &sn, &c);
        cs[t] = make_double2(c, sn);
    }
}

// Double-float weights (cos 2psi, sin 2psi) from the float64 table.
__global__ void k_weights_df(const double2* cs, float4* out, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const double2 v = cs[t];
        const df c(v.x), s(v.y);
        out[t] = make_float4(c.hi, c.lo, s.hi, s.lo);
    }
}
__global__ void k_map_to_df(const V4<double>* src, V4<df>* dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const V4<double> v = src[i];
        dst[i] = V4<df>{df(v.x), df(v.y), df(v.z), df(0.0)};
    }
}

// ---------------- launchers ----------------
size_t fft_smem_bytes(int L, bool f64) { return (size_t)(L + (L >> 4)) * (f64 ? 16 : 8); }
size_t direct_smem_bytes(int V, int lam, bool f64) {
    return (size_t)(((lam + 2) & ~1) + V + 2 * lam) * (f64 ? 8 : 4);
}


void launch_fft_spectrum(const double* h, double* H_out, double2* work, const double2* tw, int n_bands,
                         const FftPasses& fp, cudaStream_t s) {
    if (n_bands <= 0) return;
    k_fft_spectrum<<<n_bands, 256, 0, s>>>(h, H_out, reinterpret_cast<C2<double>*>(work),
                                           reinterpret_cast<const C2<double>*>(tw), fp);
    count_launches(1);
}

void launch_weights_df(const double2* cs, float4* out, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t blocks = (n + 255) / 256;
    k_weights_df<<<(int)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(cs, out, n);
    count_launches(1);
}
void launch_map_to_df(const V4<double>* src, void* dst, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t blocks = (n + 255) / 256;
    k_map_to_df<<<(int)(blocks < 152 * 8 ? blocks : 152 * 8), 256, 0, s>>>(src, reinterpret_cast<V4<df>*>(dst), n);
    count_launches(1);
}
void launch_weights64(const float* psi, double2* cs, int64_t n, cudaStream_t s) {
    if (n <= 0) return;
    const int64_t blocks = (n + 255) / 256;
    k_weights64<<<(int)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, s>>>(psi, cs, n);
    count_launches(1);
}

}  // namespace mm
