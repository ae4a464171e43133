// Template-filtered product A x = P^T F P x (and P^T F d, P^T F (d - P x)) for
// ground-based scans: F = F_B W^-1 F_G W^-1 F_B (Sect. 5.1) with the weighted
// template filter F_X = W - W X (X^T W X)^-1 X^T W of Sect. 2.1 (Eq.
// filtnoise), X = B the Legendre polynomials P_0..P_K of each azimuth sweep
// (subscan) and X = G the azimuth-bin indicators of each constant-elevation
// scan (Sect. 4), and W = w_b I on stationary block b (white noise, Sect.
// 4.1).  With W constant on a block both filters are w_b times orthogonal
// projections, so F = w_b (1 - Pi_B)(1 - Pi_G)(1 - Pi_B) on the block.
//
// One CTA per (block, right-hand side); the block's timeline lives in shared
// memory through
//   1. gather y = P x (rows (1, cos 2psi, sin 2psi); (0, cos, sin) for the
//      differenced timeline d^- and (1, 0, 0) for the summed timeline d^+ of
//      Sect. 5.1), or the timeline d, or d - P x;
//   2. y -= B (B^T B)^-1 B^T y per subscan: one warp per subscan sums the
//      moments sum_i y_i P_j(u_i), u_i = 2 (i + 1/2)/m - 1, multiplies by the
//      subscan's inverse Gram matrix (float64, precomputed on the host) and
//      subtracts the fit (the order K is a compile-time parameter);
//   3. y -= bin means of y over the block's azimuth bins, all warps over the
//      whole block (runs of equal bins in a warp are summed before one
//      shared-memory atomic per run; folding this into the per-subscan
//      passes, which keep only one warp per subscan busy, was slower);
//   4. step 2 again;
//   5. z = w_b y scattered into the map (P^T), runs of equal pixels summed in
//      the warp first.
// The arithmetic type is float32, float64, or double-float (float32 pairs,
// float64 atomics for the bin sums and the map); the double-float kernel gives
// float64-accurate products from the float32 units, which GB300 issues at 64
// times its float64 rate.
#include "filter_impl.cuh"

namespace mm {

constexpr int TMPL_NT = 512;

__device__ __forceinline__ int shfl_down_t(int v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ float shfl_xor_t(float v, int d) { return __shfl_xor_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double shfl_xor_t(double v, int d) { return __shfl_xor_sync(0xffffffffu, v, d); }
__device__ __forceinline__ df shfl_xor_t(df v, int d) {
    return df(__shfl_xor_sync(0xffffffffu, v.hi, d), __shfl_xor_sync(0xffffffffu, v.lo, d));
}

// 2 / m in the arithmetic type (double-float: from the float64 quotient).
template <typename T> __device__ __forceinline__ T two_over(int m) { return T(2) / T(m); }
template <> __device__ __forceinline__ df two_over<df>(int m) { return df(2.0 / (double)m); }

// A value in the accumulator type of the bin sums and the map.
__device__ __forceinline__ float to_acc(float v) { return v; }
__device__ __forceinline__ double to_acc(double v) { return v; }
__device__ __forceinline__ double to_acc(df v) { return (double)v; }

// Sum of v over the run of lanes with equal key that starts at this lane
// (valid on the run's first lane, `head`); runs are consecutive lanes.
template <typename T>
__device__ __forceinline__ T warp_run_sum(int key, T v, bool& head) {
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const int kprev = __shfl_up_sync(FULL, key, 1);
    head = (lane == 0) || (key != kprev);
    const unsigned heads = __ballot_sync(FULL, head);
    const unsigned above = heads & ~((2u << lane) - 1u);
    const int end = above ? (__ffs(above) - 1) : 32;
    const int need = (int)__reduce_max_sync(FULL, head ? (unsigned)(end - (int)lane) : 0u);
#pragma unroll 1
    for (int d = 1; d < need; d <<= 1) {
        const T o = shfl_down_t(v, d);
        if ((int)lane + d < end) v += o;
    }
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_sum_all(T v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += shfl_xor_t(v, d);
    return v;
}

// Legendre polynomials P_0..P_3 at u.
template <typename T>
__device__ __forceinline__ void legendre4(T u, T (&p)[4]) {
    p[0] = T(1);
    p[1] = u;
    p[2] = T(1.5) * u * u - T(0.5);
    p[3] = (T(2.5) * u * u - T(1.5)) * u;
}

// Coefficients c = G^-1 m of the subscan's Legendre fit from the moments m
// (every lane holds them after the warp sum).
template <typename T, int K>
__device__ __forceinline__ void fit_coef(const double* __restrict__ gi, const T (&mom)[4], T (&c)[4]) {
#pragma unroll
    for (int j = 0; j <= K; ++j) {
        T acc = T(0);
#pragma unroll
        for (int l = 0; l <= K; ++l) acc += T(gi[j * 4 + l]) * mom[l];
        c[j] = acc;
    }
}

// y -= B (B^T B)^-1 B^T y on every subscan of the block, one warp per
// subscan (warp-uniform sample loops, lanes on consecutive samples).
template <typename T, int K>
__device__ void project_poly(T* y, const TmplArgs& t, int blk, int64_t b0) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = TMPL_NT / 32;
    for (int s = t.blk_sub[blk] + warp; s < t.blk_sub[blk + 1]; s += nw) {
        const int64_t s0 = t.sub_off[s];
        const int m = (int)(t.sub_off[s + 1] - s0);
        const int o = (int)(s0 - b0);
        const T inv_m = two_over<T>(m);
        const T u0 = inv_m * T(0.5) - T(1);
        T mom[4] = {T(0), T(0), T(0), T(0)};
        for (int i = lane; i < m; i += 32) {
            T p[4];
            legendre4<T>(T(i) * inv_m + u0, p);
            const T v = y[o + i];
#pragma unroll
            for (int j = 0; j <= K; ++j) mom[j] += v * p[j];
        }
#pragma unroll
        for (int j = 0; j <= K; ++j) mom[j] = warp_sum_all(mom[j]);
        T c[4];
        fit_coef<T, K>(t.ginv + (int64_t)s * 16, mom, c);
        for (int i = lane; i < m; i += 32) {
            T p[4];
            legendre4<T>(T(i) * inv_m + u0, p);
            T fit = T(0);
#pragma unroll
            for (int j = 0; j <= K; ++j) fit += c[j] * p[j];
            y[o + i] -= fit;
        }
    }
}

// Map components a pointing row touches: stokes 0 (I, Q, U), 1 (Q, U: the
// differenced timeline), 2 (I: the summed timeline).
template <int ST> struct StokesCols { static constexpr int n = 3, c0 = 0; };
template <> struct StokesCols<1> { static constexpr int n = 2, c0 = 1; };
template <> struct StokesCols<2> { static constexpr int n = 1, c0 = 0; };

template <typename A> __device__ __forceinline__ A& vcomp(V4<A>* q, int c) {
    return c == 0 ? q->x : (c == 1 ? q->y : q->z);
}

// P^T of a warp's 128 consecutive samples (four per lane) for NC map
// components starting at C0: in-lane suffix sums over runs of equal pixels,
// the lane's last run continued through later lanes by doubling (as in the
// float32 half-length scatter), one atomic per run and component.
template <typename T, int NC, int C0>
__device__ __forceinline__ void tmpl_run_scatter(const int (&p)[4], T (&v)[NC][4], V4<typename AccT<T>::type>* q) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool e01 = p[0] == p[1], e12 = p[1] == p[2], e23 = p[2] == p[3];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        if (e23) v[c][2] += v[c][3];
        if (e12) v[c][1] += v[c][2];
        if (e01) v[c][0] += v[c][1];
    }
    const bool whole = e01 && e12 && e23;
    const int pnext = __shfl_down_sync(FULL, p[0], 1);
    const bool cont = lane < 31 && pnext == p[3];
    T x[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        x[c] = shfl_down_t(v[c][0], 1);
        if (!cont) x[c] = T(0);
    }
    // every lane takes part in each shuffle (no short-circuit around it)
    const bool wnext = __shfl_down_sync(FULL, (int)whole, 1) != 0;
    bool chain = cont && wnext;
#pragma unroll 1
    for (int d = 1; __any_sync(FULL, chain); d <<= 1) {
        T y[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) y[c] = shfl_down_t(x[c], d);
        const bool cn = __shfl_down_sync(FULL, (int)chain, d) != 0;
        if (chain) {
#pragma unroll
            for (int c = 0; c < NC; ++c) x[c] += y[c];
        }
        chain = chain && cn;
    }
    const int plast = __shfl_up_sync(FULL, p[3], 1);
    const bool head[4] = {lane == 0 || p[0] != plast, !e01, !e12, !e23};
    const bool reach[4] = {whole, e12 && e23, e23, true};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if (head[j] && p[j] >= 0) {
            V4<typename AccT<T>::type>* dst = q + p[j];
            if constexpr (NC == 3 && std::is_same<T, float>::value) {
                atomic_add3(dst, reach[j] ? v[0][j] + x[0] : v[0][j], reach[j] ? v[1][j] + x[1] : v[1][j],
                            reach[j] ? v[2][j] + x[2] : v[2][j]);
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c)
                    atomicAdd(&vcomp(dst, C0 + c), to_acc(reach[j] ? v[c][j] + x[c] : v[c][j]));
            }
        }
    }
}

template <typename T, bool FROM_TOD, int K, int ST>
__global__ void __launch_bounds__(TMPL_NT) k_filter_tmpl(const FilterArgs a, const TmplArgs t) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int blk = blockIdx.x, rhs = blockIdx.y;
    if (a.state && !a.state[rhs].active) return;
    const int64_t b0 = t.block_off[blk];
    const int nb = (int)(t.block_off[blk + 1] - b0);
    using Acc = typename AccT<T>::type;
    static_assert(sizeof(Acc) == sizeof(T), "bin means overwrite the bin sums in place");
    T* y = reinterpret_cast<T*>(smraw);
    Acc* gsum = reinterpret_cast<Acc*>(y + ((nb + 1) & ~1));
    int* gcnt = reinterpret_cast<int*>(gsum + t.n_bins);
    const T iw = ST == 1 ? T(0) : T(1);   // I column of P
    const T pw = ST == 2 ? T(0) : T(1);   // Q, U columns
    const V4<T>* xm = nullptr;
    if (!FROM_TOD) xm = reinterpret_cast<const V4<T>*>(a.src) + (int64_t)rhs * a.n_pix;
    else if (a.xmap) xm = reinterpret_cast<const V4<T>*>(a.xmap) + (int64_t)rhs * a.n_pix;
    // 1. gather (float32 and double-float: four consecutive samples per thread, vector pointing loads)
    if constexpr (!std::is_same<T, double>::value) {
        for (int u = threadIdx.x; 4 * u < nb; u += TMPL_NT) {
            const int i0 = 4 * u;
            const int64_t t0 = b0 + i0;
            int p[4];
            float ps[4];
            if constexpr (ST == 2) load4_pix(a, t0, true, nb - i0, p);   // intensity rows need no angle
            else load4(a, t0, true, nb - i0, p, ps);
            T v[4] = {T(0), T(0), T(0), T(0)};
            if (FROM_TOD) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (i0 + j < nb)
                        v[j] = a.tod_is_float ? T(__ldg(reinterpret_cast<const float*>(a.src) + rhs * a.n_samples + t0 + j))
                                              : T(__ldg(reinterpret_cast<const double*>(a.src) + rhs * a.n_samples + t0 + j));
            }
            if (xm) {
                V4<T> m[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (p[j] >= 0) m[j] = ldmap<T>(xm + p[j]);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (p[j] >= 0) {
                        T px;
                        if constexpr (ST == 2) {
                            px = m[j].x;
                        } else {
                            T c, s;
                            weights_from(a, t0 + j, ps[j], c, s);
                            px = ST == 1 ? c * m[j].y + s * m[j].z : m[j].x + (c * m[j].y + s * m[j].z);
                        }
                        v[j] = FROM_TOD ? v[j] - px : px;
                    }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (i0 + j < nb) y[i0 + j] = v[j];
        }
    } else
    for (int i = threadIdx.x; i < nb; i += TMPL_NT) {
        const int64_t ts = b0 + i;
        T v = T(0);
        if (FROM_TOD)
            v = a.tod_is_float ? T(__ldg(reinterpret_cast<const float*>(a.src) + rhs * a.n_samples + ts))
                               : T(__ldg(reinterpret_cast<const double*>(a.src) + rhs * a.n_samples + ts));
        if (xm) {
            const int p = __ldg(a.pix + ts);
            if (p >= 0) {
                T c, s;
                weights(a, ts, c, s);
                const V4<T> m = ldmap<T>(xm + p);
                const T px = iw * m.x + pw * (c * m.y + s * m.z);
                v = FROM_TOD ? v - px : px;
            }
        }
        y[i] = v;
    }
    for (int i = threadIdx.x; i < t.n_bins; i += TMPL_NT) {
        gsum[i] = Acc(0);
        gcnt[i] = 0;
    }
    __syncthreads();
    const bool ground = t.az && t.n_bins > 0;
    // 2. (1 - Pi_B) y (one warp per subscan)
    if constexpr (K >= 0) {
        project_poly<T, K>(y, t, blk, b0);
        __syncthreads();
    }
    if (ground) {
        // 3. y - azimuth-bin means over the block (all warps: runs of equal bins summed in the warp)
        for (int base = 0; base < nb; base += TMPL_NT) {
            const int i = base + threadIdx.x;
            int g = -1;
            T v = T(0);
            if (i < nb) {
                g = __ldg(t.az + b0 + i);
                if (g >= t.n_bins) g = -1;   // out-of-range bins belong to no column
                v = y[i];
            }
            bool head;
            const T sv = warp_run_sum<T>(g, v, head);
            const int cn = warp_run_sum<int>(g, (g >= 0) ? 1 : 0, head);
            if (head && g >= 0) {
                atomicAdd(gsum + g, to_acc(sv));
                atomicAdd(gcnt + g, cn);
            }
        }
        __syncthreads();
        // bin means, in place of the sums (one division per bin, not per sample)
        T* gmean = reinterpret_cast<T*>(gsum);
        for (int i = threadIdx.x; i < t.n_bins; i += TMPL_NT) {
            const Acc sm = gsum[i];
            const int n = gcnt[i];
            gmean[i] = n > 0 ? T(sm / Acc(n)) : T(0);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < nb; i += TMPL_NT) {
            const int g = __ldg(t.az + b0 + i);
            if (g >= 0 && g < t.n_bins) y[i] -= gmean[g];
        }
        __syncthreads();
        // 4. (1 - Pi_B) again
        if constexpr (K >= 0) {
            project_poly<T, K>(y, t, blk, b0);
            __syncthreads();
        }
    }
    // without a ground template F_B W^-1 F_B = w_b (1 - Pi_B)^2 = w_b (1 - Pi_B): one projection
    // 5. weight and scatter
    V4<Acc>* q = reinterpret_cast<V4<Acc>*>(a.dst) + (int64_t)rhs * a.n_pix;
    const T wb = T(t.w_block[blk]);
    if constexpr (!std::is_same<T, double>::value) {
        // four consecutive samples per lane, in-lane run sums, then the warp-segmented sums
        constexpr int NW = TMPL_NT / 32;
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int base = warp * 128; base < nb; base += NW * 128) {
            const int i0 = base + 4 * lane;
            const int64_t t0 = b0 + i0;
            int p[4];
            float ps[4];
            if constexpr (ST == 2) load4_pix(a, t0, i0 < nb, nb - i0, p);
            else load4(a, t0, i0 < nb, nb - i0, p, ps);
            constexpr int NC = StokesCols<ST>::n;
            T v[NC][4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const T z = (p[j] >= 0 && i0 + j < nb) ? wb * y[min(i0 + j, nb - 1)] : T(0);
                if constexpr (ST == 2) {
                    v[0][j] = z;
                } else {
                    T c = T(0), sn = T(0);
                    if (p[j] >= 0) weights_from(a, t0 + j, ps[j], c, sn);
                    if constexpr (ST == 0) v[0][j] = z;
                    v[NC - 2][j] = z * c;
                    v[NC - 1][j] = z * sn;
                }
            }
            tmpl_run_scatter<T, NC, StokesCols<ST>::c0>(p, v, q);
        }
        return;
    }
    for (int base = 0; base < nb; base += TMPL_NT) {
        const int i = base + threadIdx.x;
        int p = -1;
        T z = T(0), c = T(0), s = T(0);
        if (i < nb) {
            const int64_t ts = b0 + i;
            p = __ldg(a.pix + ts);
            if (p >= 0) {
                weights(a, ts, c, s);
                z = wb * y[i];
            }
        }
        scatter_vals<T>(p, iw * z, pw * z * c, pw * z * s, q);
    }
}

size_t tmpl_smem_bytes(int64_t max_block, int n_bins, bool f64) {
    const size_t e = f64 ? 8 : 4;
    return (size_t)((max_block + 1) & ~1LL) * e + (size_t)n_bins * (e + 4);
}

template <typename T, bool FROM_TOD, int K, int ST>
static void launch_tmpl_ks(const FilterArgs& a, const TmplArgs& t, int nrhs, cudaStream_t s) {
    const size_t sm = tmpl_smem_bytes(t.max_block, t.n_bins, sizeof(T) == 8);
    static std::atomic<size_t> configured{0};
    raise_smem_once(configured, sm, [](size_t v) {
        cudaFuncSetAttribute(k_filter_tmpl<T, FROM_TOD, K, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v);
    });
    k_filter_tmpl<T, FROM_TOD, K, ST><<<dim3(t.n_blocks, nrhs), TMPL_NT, sm, s>>>(a, t);
    count_launches(1);
}
template <typename T, bool FROM_TOD, int K>
static void launch_tmpl_k(const FilterArgs& a, const TmplArgs& t, int nrhs, cudaStream_t s) {
    switch (t.stokes) {
        case 1: return launch_tmpl_ks<T, FROM_TOD, K, 1>(a, t, nrhs, s);
        case 2: return launch_tmpl_ks<T, FROM_TOD, K, 2>(a, t, nrhs, s);
        default: return launch_tmpl_ks<T, FROM_TOD, K, 0>(a, t, nrhs, s);
    }
}

template <typename T, bool FROM_TOD>
static void launch_tmpl_t(const FilterArgs& a, const TmplArgs& t, int nrhs, cudaStream_t s) {
    switch (t.order) {
        case 0: return launch_tmpl_k<T, FROM_TOD, 0>(a, t, nrhs, s);
        case 1: return launch_tmpl_k<T, FROM_TOD, 1>(a, t, nrhs, s);
        case 2: return launch_tmpl_k<T, FROM_TOD, 2>(a, t, nrhs, s);
        case 3: return launch_tmpl_k<T, FROM_TOD, 3>(a, t, nrhs, s);
        default: return launch_tmpl_k<T, FROM_TOD, -1>(a, t, nrhs, s);
    }
}

void launch_filter_tmpl(const FilterArgs& a, const TmplArgs& t, int nrhs, int prec, bool from_tod, cudaStream_t s) {
    if (t.n_blocks <= 0 || nrhs <= 0) return;
    if (prec == 2) {
        if (from_tod) launch_tmpl_t<df, true>(a, t, nrhs, s);
        else launch_tmpl_t<df, false>(a, t, nrhs, s);
    } else if (prec == 1) {
        if (from_tod) launch_tmpl_t<double, true>(a, t, nrhs, s);
        else launch_tmpl_t<double, false>(a, t, nrhs, s);
    } else {
        if (from_tod) launch_tmpl_t<float, true>(a, t, nrhs, s);
        else launch_tmpl_t<float, false>(a, t, nrhs, s);
    }
}

}  // namespace mm
