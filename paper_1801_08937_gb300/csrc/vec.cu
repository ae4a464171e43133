// Map-space kernels: M_BD build and apply (Sect. 3.1, Eq. mbd), the fused
// PCG vector steps with float64 inner products (Sect. 3, Eq. pcg), the
// two-level preconditioner M_2l (Sect. 3.2, Eq. m2l) and the tall-skinny
// float64 products of the Arnoldi process (Appendix A).
//
// Every reduction is two-phase and deterministic: each CTA writes its
// partial sums, and the last CTA to finish (an atomic ticket, no waiting)
// adds them in CTA order and applies the scalar update.
#include <cuda_runtime.h>

#include "common.cuh"
#include "fconv.cuh"
#include "df64.cuh"

namespace mm {

constexpr int VT = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
    return v;
}

// Sum D per-thread values over the CTA; thread d < D writes partial[d].
template <int D>
__device__ __forceinline__ void block_partials(const double (&v)[D], double* out) {
    __shared__ double red[VT / 32][D > 0 ? D : 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int d = 0; d < D; ++d) {
        const double s = warp_sum(v[d]);
        if (lane == 0) red[warp][d] = s;
    }
    __syncthreads();
    if (threadIdx.x < D) {
        double s = 0.0;
        for (int w = 0; w < VT / 32; ++w) s += red[w][threadIdx.x];
        out[threadIdx.x] = s;
    }
}

// Last-CTA election for the reduction of slice `rhs` (grid.y); returns true
// in every thread of the CTA that finishes last.
__device__ __forceinline__ bool last_block(unsigned* counter, int rhs) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned prev = atomicAdd(counter + rhs, 1u);
        is_last = (prev == gridDim.x - 1);
    }
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// Sum of the CTA partials of value d for slice rhs, by the whole (last) CTA:
// strided per-thread sums, then warp and CTA trees -- a fixed order, so the
// result is deterministic.  Every thread of the CTA must call it; the sum is
// returned to all threads.
template <int D>
__device__ __forceinline__ double gather_partial(const double* partial, int nblk, int nrhs, int rhs, int d) {
    __shared__ double red[VT / 32];
    __shared__ double total;
    double s = 0.0;
    for (int b = threadIdx.x; b < nblk; b += VT) s += __ldcg(partial + ((int64_t)b * nrhs + rhs) * D + d);
    s = warp_sum(s);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < VT / 32; ++w) t += red[w];
        total = t;
    }
    __syncthreads();
    return total;
}

// Warp w sums partials of the values c = w, w + 8, ... (k values per slice).
__device__ __forceinline__ double warp_gather(const double* partial, int nblk, int64_t stride, int64_t off) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += __ldcg(partial + (int64_t)b * stride + off);
    s = warp_sum(s);
    return __shfl_sync(0xffffffffu, s, 0);
}

__device__ __forceinline__ V4<double> ld4(const V4<double>* p) { return *p; }
__device__ __forceinline__ V4<double> ld4(const V4<float>* p) {
    const V4<float> v = *p;
    return {v.x, v.y, v.z, 0.0};
}
__device__ __forceinline__ double dot3(const V4<double>& a, const V4<double>& b) {
    return a.x * b.x + a.y * b.y + a.z * b.z;
}
__device__ __forceinline__ V4<double> bd_mul(const double* m, const V4<double>& v) {
    return {m[0] * v.x + m[1] * v.y + m[2] * v.z, m[1] * v.x + m[3] * v.y + m[4] * v.z,
            m[2] * v.x + m[4] * v.y + m[5] * v.z, 0.0};
}

#define PIX_LOOP(i) for (int i = blockIdx.x * VT + threadIdx.x; i < a.n_pix; i += gridDim.x * VT)

// ---------------- conversions ----------------
__global__ void k_map_in(const double* src, V4<double>* dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)VT + threadIdx.x; i < n; i += (int64_t)gridDim.x * VT)
        dst[i] = V4<double>{src[3 * i], src[3 * i + 1], src[3 * i + 2], 0.0};
}
__global__ void k_map_out(const V4<double>* src, double* dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)VT + threadIdx.x; i < n; i += (int64_t)gridDim.x * VT) {
        const V4<double> v = src[i];
        dst[3 * i] = v.x;
        dst[3 * i + 1] = v.y;
        dst[3 * i + 2] = v.z;
    }
}
__global__ void k_to_f32(const V4<double>* src, V4<float>* dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)VT + threadIdx.x; i < n; i += (int64_t)gridDim.x * VT) {
        const V4<double> v = src[i];
        dst[i] = V4<float>{(float)v.x, (float)v.y, (float)v.z, 0.0f};
    }
}
__global__ void k_from_f32(const V4<float>* src, V4<double>* dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)VT + threadIdx.x; i < n; i += (int64_t)gridDim.x * VT)
        dst[i] = ld4(src + i);
}
static int grid_for(int64_t n) {
    const int64_t b = (n + VT - 1) / VT;
    return (int)(b < 152 * 8 ? (b > 0 ? b : 1) : 152 * 8);
}
void launch_map_in(const double* src3, V4<double>* dst4, int64_t n, cudaStream_t s) {
    if (n > 0) {
        k_map_in<<<grid_for(n), VT, 0, s>>>(src3, dst4, n);
        count_launches(1);
    }
}
void launch_map_out(const V4<double>* src4, double* dst3, int64_t n, cudaStream_t s) {
    if (n > 0) {
        k_map_out<<<grid_for(n), VT, 0, s>>>(src4, dst3, n);
        count_launches(1);
    }
}
void launch_to_f32(const V4<double>* src, V4<float>* dst, int64_t n, cudaStream_t s) {
    if (n > 0) {
        k_to_f32<<<grid_for(n), VT, 0, s>>>(src, dst, n);
        count_launches(1);
    }
}
void launch_from_f32(const V4<float>* src, V4<double>* dst, int64_t n, cudaStream_t s) {
    if (n > 0) {
        k_from_f32<<<grid_for(n), VT, 0, s>>>(src, dst, n);
        count_launches(1);
    }
}
void launch_zero(void* p, size_t bytes, cudaStream_t s) {
    if (bytes) cudaMemsetAsync(p, 0, bytes, s);
}

// ---------------- M_BD ----------------
// Per sample: bucket j = number of right-hand-side lengths <= the sample's
// position in its detector timeline (lengths sorted ascending); the sample
// belongs to every right-hand side of sorted rank >= j.  Sums of
// c_0 w w^T (6 entries) and the hit count go to bucket j.
__global__ void k_bd_accumulate(const int32_t* pix, const float* psi, const int64_t* block_off,
                                const int32_t* block_band, const double* band, int lam1, int64_t n_t,
                                const int64_t* sorted_len, int nrhs, double* sums, int n_pix) {
    const int b = blockIdx.x;
    const int64_t o0 = block_off[b], o1 = block_off[b + 1];
    const double c0 = band[(int64_t)block_band[b] * lam1];
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    for (int64_t base = o0 + (threadIdx.x & ~31); base < o1; base += blockDim.x) {
        const int64_t t = base + lane;
        int key = -1;
        double v[7] = {0, 0, 0, 0, 0, 0, 0};
        if (t < o1) {
            const int p = pix[t];
            if (p >= 0) {
                const int64_t pos = t % n_t;
                int j = 0;
                while (j < nrhs && sorted_len[j] <= pos) ++j;
                if (j < nrhs) {
                    key = j * n_pix + p;
                    double sn, cs;
                    sincos(2.0 * (double)psi[t], &sn, &cs);
                    v[0] = c0;
                    v[1] = c0 * cs;
                    v[2] = c0 * sn;
                    v[3] = c0 * cs * cs;
                    v[4] = c0 * cs * sn;
                    v[5] = c0 * sn * sn;
                    v[6] = 1.0;
                }
            }
        }
        const int kprev = __shfl_up_sync(FULL, key, 1);
        const bool head = (lane == 0) || (key != kprev);
        const unsigned heads = __ballot_sync(FULL, head);
        const unsigned above = heads & ~((2u << lane) - 1u);
        const int end = above ? (__ffs(above) - 1) : 32;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
            for (int e = 0; e < 7; ++e) {
                const double o = __shfl_down_sync(FULL, v[e], d);
                if ((int)lane + d < end) v[e] += o;
            }
        }
        if (head && key >= 0) {
#pragma unroll
            for (int e = 0; e < 7; ++e) atomicAdd(sums + (int64_t)key * 7 + e, v[e]);
        }
    }
}

// Prefix over buckets: sorted rank r holds the sum of buckets 0..r.
__global__ void k_bd_prefix(double* sums, int n_pix, int nrhs) {
    for (int64_t i = blockIdx.x * (int64_t)VT + threadIdx.x; i < (int64_t)n_pix * 7; i += (int64_t)gridDim.x * VT) {
        double acc = 0.0;
        for (int j = 0; j < nrhs; ++j) {
            acc += sums[(int64_t)j * n_pix * 7 + i];
            sums[(int64_t)j * n_pix * 7 + i] = acc;
        }
    }
}

void launch_bd_accumulate(const int32_t* pix, const float* psi, const int64_t* block_off, const int32_t* block_band,
                          const double* band, int lam1, int n_blocks, int64_t /*unused*/, int64_t n_t,
                          const int64_t* sorted_len, int nrhs, double* sums, int n_pix, cudaStream_t s) {
    if (n_blocks <= 0) return;
    k_bd_accumulate<<<n_blocks, VT, 0, s>>>(pix, psi, block_off, block_band, band, lam1, n_t, sorted_len, nrhs, sums,
                                            n_pix);
    count_launches(1);
    if (nrhs > 1) {
        k_bd_prefix<<<grid_for((int64_t)n_pix * 7), VT, 0, s>>>(sums, n_pix, nrhs);
        count_launches(1);
    }
}

// Eigenvalues of a symmetric 3x3 matrix by cyclic Jacobi rotations.
__device__ void sym3_eig(double a[3][3], double& lmin, double& lmax) {
    for (int sweep = 0; sweep < 12; ++sweep) {
        const double off = fabs(a[0][1]) + fabs(a[0][2]) + fabs(a[1][2]);
        const double diag = fabs(a[0][0]) + fabs(a[1][1]) + fabs(a[2][2]);
        if (off <= 1e-300 || off <= 1e-17 * diag) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (a[p][q] == 0.0) continue;
                const double theta = (a[q][q] - a[p][p]) / (2.0 * a[p][q]);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), sn = t * c;
                for (int k = 0; k < 3; ++k) {
                    const double akp = a[k][p], akq = a[k][q];
                    a[k][p] = c * akp - sn * akq;
                    a[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    const double apk = a[p][k], aqk = a[q][k];
                    a[p][k] = c * apk - sn * aqk;
                    a[q][k] = sn * apk + c * aqk;
                }
            }
    }
    lmin = fmin(a[0][0], fmin(a[1][1], a[2][2]));
    lmax = fmax(a[0][0], fmax(a[1][1], a[2][2]));
}

// sums [nrhs][n_pix][7] -> bd [nrhs][n_pix][6] = inverse blocks (upper
// triangle by rows).  With set_good, the keep/drop decision is made here
// (hits >= 3 and rcond >= rcond_min); otherwise `good` is read and a kept
// pixel whose block is numerically singular for this right-hand side gets a
// zero block.
// stokes 1: only the (Q, U) block counts (pointing rows (0, cos, sin) of the
// differenced timeline): at least 2 hits and a conditioned 2x2 block; the I
// entries of the inverse are zero.  stokes 2: only I (rows (1, 0, 0) of the
// summed timeline): at least 1 hit, the 1x1 inverse, Q and U entries zero.
__global__ void k_bd_invert(const double* sums, double* bd, uint8_t* good, int* n_dropped, int n_pix, int nrhs,
                            double rcond_min, int set_good, int stokes) {
    const int64_t total = (int64_t)n_pix * nrhs;
    for (int64_t idx = blockIdx.x * (int64_t)VT + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * VT) {
        const int p = (int)(idx % n_pix);
        const double* S = sums + idx * 7;
        const double s00 = S[0], s01 = S[1], s02 = S[2], s11 = S[3], s12 = S[4], s22 = S[5], hits = S[6];
        if (stokes == 2) {
            bool keep1;
            if (set_good) {
                keep1 = hits >= 1.0 && s00 > 0.0;
                good[p] = keep1 ? 1 : 0;
                if (!keep1) atomicAdd(n_dropped, 1);
            } else {
                keep1 = good[p] != 0 && s00 > 0.0;
            }
            double* o = bd + idx * 6;
            for (int e = 0; e < 6; ++e) o[e] = 0.0;
            if (keep1) o[0] = 1.0 / s00;
            continue;
        }
        if (stokes == 1) {
            const double tr = s11 + s22, det2 = s11 * s22 - s12 * s12;
            const double disc = sqrt(fmax(0.25 * (s11 - s22) * (s11 - s22) + s12 * s12, 0.0));
            const double lmax2 = 0.5 * tr + disc, lmin2 = 0.5 * tr - disc;
            const double rc2 = lmax2 > 0.0 ? lmin2 / lmax2 : 0.0;
            bool keep2;
            if (set_good) {
                keep2 = hits >= 2.0 && rc2 >= rcond_min;
                good[p] = keep2 ? 1 : 0;
                if (!keep2) atomicAdd(n_dropped, 1);
            } else {
                keep2 = good[p] != 0 && rc2 > 1e-12;
            }
            double* o = bd + idx * 6;
            for (int e = 0; e < 6; ++e) o[e] = 0.0;
            if (keep2) {
                o[3] = s22 / det2;
                o[4] = -s12 / det2;
                o[5] = s11 / det2;
            }
            continue;
        }
        double m[3][3] = {{s00, s01, s02}, {s01, s11, s12}, {s02, s12, s22}};
        double lmin, lmax;
        sym3_eig(m, lmin, lmax);
        const double rc = lmax > 0.0 ? lmin / lmax : 0.0;
        bool keep;
        if (set_good) {
            keep = hits >= 3.0 && rc >= rcond_min;
            good[p] = keep ? 1 : 0;
            if (!keep) atomicAdd(n_dropped, 1);
        } else {
            keep = good[p] != 0 && rc > 1e-12;
        }
        double* o = bd + idx * 6;
        if (!keep) {
            for (int e = 0; e < 6; ++e) o[e] = 0.0;
            continue;
        }
        // inverse of the symmetric block by cofactors
        const double c00 = s11 * s22 - s12 * s12;
        const double c01 = s02 * s12 - s01 * s22;
        const double c02 = s01 * s12 - s02 * s11;
        const double c11 = s00 * s22 - s02 * s02;
        const double c12 = s01 * s02 - s00 * s12;
        const double c22 = s00 * s11 - s01 * s01;
        const double det = s00 * c00 + s01 * c01 + s02 * c02;
        const double id = 1.0 / det;
        o[0] = c00 * id;
        o[1] = c01 * id;
        o[2] = c02 * id;
        o[3] = c11 * id;
        o[4] = c12 * id;
        o[5] = c22 * id;
    }
}
void launch_bd_invert(const double* sums, double* bd, uint8_t* good, int* n_dropped, int n_pix, int nrhs,
                      double rcond_min, int set_good, cudaStream_t s, int stokes) {
    k_bd_invert<<<grid_for((int64_t)n_pix * nrhs), VT, 0, s>>>(sums, bd, good, n_dropped, n_pix, nrhs, rcond_min,
                                                              set_good, stokes);
    count_launches(1);
}

__global__ void k_flag_samples(int32_t* pix, const uint8_t* good, int64_t n) {
    for (int64_t t = blockIdx.x * (int64_t)VT + threadIdx.x; t < n; t += (int64_t)gridDim.x * VT) {
        const int p = pix[t];
        if (p >= 0 && !good[p]) pix[t] = -1;
    }
}
void launch_flag_samples(int32_t* pix, const uint8_t* good, int64_t n, cudaStream_t s) {
    if (n > 0) {
        k_flag_samples<<<grid_for(n), VT, 0, s>>>(pix, good, n);
        count_launches(1);
    }
}

__global__ void k_bd_apply(const double* bd, int per_rhs, const V4<double>* x, V4<double>* y, int n_pix) {
    const int rhs = blockIdx.y;
    for (int i = blockIdx.x * VT + threadIdx.x; i < n_pix; i += gridDim.x * VT) {
        const double* m = bd + ((int64_t)(per_rhs ? rhs : 0) * n_pix + i) * 6;
        y[(int64_t)rhs * n_pix + i] = bd_mul(m, x[(int64_t)rhs * n_pix + i]);
    }
}
void launch_bd_apply(const double* bd, int bd_per_rhs, const V4<double>* x, V4<double>* y, int n_pix, int nrhs,
                     cudaStream_t s) {
    dim3 g(grid_for(n_pix), nrhs);
    k_bd_apply<<<g, VT, 0, s>>>(bd, bd_per_rhs, x, y, n_pix);
    count_launches(1);
}

// ---------------- PCG ----------------
__device__ __forceinline__ const double* bd_of(const PcgArgs& a, int rhs, int i) {
    return a.bd + ((int64_t)(a.bd_per_rhs ? rhs : 0) * a.n_pix + i) * 6;
}

// x = 0, r = b, p = 0; ||b||.
__global__ void k_pcg_init(const PcgArgs a, const V4<double>* b) {
    const int rhs = blockIdx.y;
    const int64_t off = (int64_t)rhs * a.n_pix;
    double acc[1] = {0.0};
    const V4<double> zero{0, 0, 0, 0};
    PIX_LOOP(i) {
        const V4<double> bv = b[off + i];
        a.x[off + i] = zero;
        a.r[off + i] = bv;
        a.p[off + i] = zero;
        acc[0] += dot3(bv, bv);
    }
    double* part = a.partial + ((int64_t)blockIdx.x * a.nrhs + rhs) * 1;
    block_partials<1>(acc, part);
    if (last_block(a.counter, rhs)) {
        const double bb = gather_partial<1>(a.partial, gridDim.x, a.nrhs, rhs, 0);
        if (threadIdx.x == 0) {
            RhsState& st = a.st[rhs];
            st.bnorm = sqrt(bb);
            st.relres = 1.0;
            st.iters = 0;
            st.status = 0;
            st.alpha = st.beta = 0.0;
            st.active = (bb > 0.0 && st.max_iter > 0) ? 1 : 0;
            if (!(bb > 0.0)) st.relres = 0.0;
            a.hist[(int64_t)rhs * a.hist_stride] = st.relres;
            a.counter[rhs] = 0;
        }
    }
}

// z = M_BD r and r^T z; finalize_beta: beta = rz_new / rz (else rz = rz_new only).
__global__ void k_bd_dot(const PcgArgs a, int finalize_beta) {
    const int rhs = blockIdx.y;
    if (!a.st[rhs].active) return;
    const int64_t off = (int64_t)rhs * a.n_pix;
    double acc[1] = {0.0};
    PIX_LOOP(i) {
        const V4<double> rv = a.r[off + i];
        const V4<double> zv = bd_mul(bd_of(a, rhs, i), rv);
        a.z[off + i] = zv;
        acc[0] += dot3(rv, zv);
    }
    block_partials<1>(acc, a.partial + ((int64_t)blockIdx.x * a.nrhs + rhs));
    if (last_block(a.counter, rhs)) {
        const double rz = gather_partial<1>(a.partial, gridDim.x, a.nrhs, rhs, 0);
        if (threadIdx.x == 0) {
            RhsState& st = a.st[rhs];
            st.beta = finalize_beta ? rz / st.rz : 0.0;
            st.rz = rz;
            a.counter[rhs] = 0;
        }
    }
}

// p = z + beta p (first: p = z); src = p in the operator precision; qacc = 0.
__global__ void k_pcg_src(const PcgArgs a, int first) {
    const int rhs = blockIdx.y;
    if (!a.st[rhs].active) return;
    const double beta = first ? 0.0 : a.st[rhs].beta;
    const int64_t off = (int64_t)rhs * a.n_pix;
    PIX_LOOP(i) {
        const V4<double> zv = a.z[off + i];
        V4<double> pv = a.p[off + i];
        pv = first ? zv : V4<double>{zv.x + beta * pv.x, zv.y + beta * pv.y, zv.z + beta * pv.z, 0.0};
        a.p[off + i] = pv;
        if (a.src_f32 == 1) {
            reinterpret_cast<V4<float>*>(a.src)[off + i] = V4<float>{(float)pv.x, (float)pv.y, (float)pv.z, 0.0f};
            reinterpret_cast<V4<float>*>(a.qacc)[off + i] = V4<float>{0.f, 0.f, 0.f, 0.f};
        } else if (a.src_f32 == 2) {
            // double-float operator input, float64 accumulators
            reinterpret_cast<V4<df>*>(a.src)[off + i] = V4<df>{df(pv.x), df(pv.y), df(pv.z), df(0.0)};
            reinterpret_cast<V4<double>*>(a.qacc)[off + i] = V4<double>{0, 0, 0, 0};
        } else {
            reinterpret_cast<V4<double>*>(a.src)[off + i] = pv;
            reinterpret_cast<V4<double>*>(a.qacc)[off + i] = V4<double>{0, 0, 0, 0};
        }
    }
}

__device__ __forceinline__ V4<double> load_q(const PcgArgs& a, int64_t j) {
    return a.q32 ? ld4(a.q32 + j) : a.q64[j];
}

// p^T q; alpha = rz / pq; a non-positive or non-finite pq is a breakdown.
__global__ void k_pcg_pq(const PcgArgs a) {
    const int rhs = blockIdx.y;
    if (!a.st[rhs].active) return;
    const int64_t off = (int64_t)rhs * a.n_pix;
    double acc[1] = {0.0};
    PIX_LOOP(i) acc[0] += dot3(a.p[off + i], load_q(a, off + i));
    block_partials<1>(acc, a.partial + ((int64_t)blockIdx.x * a.nrhs + rhs));
    if (last_block(a.counter, rhs)) {
        const double pq = gather_partial<1>(a.partial, gridDim.x, a.nrhs, rhs, 0);
        if (threadIdx.x == 0) {
            RhsState& st = a.st[rhs];
            st.pq = pq;
            if (!(pq > 0.0) || !isfinite(pq) || !isfinite(st.rz)) {
                st.status = 6;
                st.active = 0;
                st.alpha = 0.0;
            } else {
                st.alpha = st.rz / pq;
            }
            if (a.ahist) a.ahist[(int64_t)rhs * a.hist_stride + st.iters] = st.alpha;
            a.counter[rhs] = 0;
        }
    }
}

// x += alpha p, r -= alpha q, ||r||; with M_BD fused (two_level == 0) also
// z = M_BD r and r^T z, with M_2l (two_level == 1) t = Z^T r (k values)
// and u = E^-1 t.
template <int TWO_LEVEL>
__global__ void k_pcg_update(const PcgArgs a) {
    const int rhs = blockIdx.y;
    if (!a.st[rhs].active) return;
    const double alpha = a.st[rhs].alpha;
    const int64_t off = (int64_t)rhs * a.n_pix;
    double acc[2] = {0.0, 0.0};
    PIX_LOOP(i) {
        const V4<double> pv = a.p[off + i];
        const V4<double> qv = load_q(a, off + i);
        V4<double> xv = a.x[off + i], rv = a.r[off + i];
        xv.x += alpha * pv.x;
        xv.y += alpha * pv.y;
        xv.z += alpha * pv.z;
        rv.x -= alpha * qv.x;
        rv.y -= alpha * qv.y;
        rv.z -= alpha * qv.z;
        a.x[off + i] = xv;
        a.r[off + i] = rv;
        acc[0] += dot3(rv, rv);
        if (!TWO_LEVEL) {
            const V4<double> zv = bd_mul(bd_of(a, rhs, i), rv);
            a.z[off + i] = zv;
            acc[1] += dot3(rv, zv);
        }
    }
    block_partials<2>(acc, a.partial + ((int64_t)blockIdx.x * a.nrhs + rhs) * 2);
    if (last_block(a.counter, rhs)) {
        const double rr = gather_partial<2>(a.partial, gridDim.x, a.nrhs, rhs, 0);
        const double rz_new = TWO_LEVEL ? 0.0 : gather_partial<2>(a.partial, gridDim.x, a.nrhs, rhs, 1);
        if (threadIdx.x == 0) {
            RhsState& st = a.st[rhs];
            st.iters += 1;
            st.relres = sqrt(rr) / st.bnorm;
            a.hist[(int64_t)rhs * a.hist_stride + st.iters] = st.relres;
            if (!isfinite(st.relres)) {
                st.status = 6;
                st.active = 0;
            } else if (st.relres <= st.tol) {
                st.active = 0;
            } else if (st.iters >= st.max_iter) {
                st.status = 5;
                st.active = 0;
            }
            if (!TWO_LEVEL) {
                const double rz = rz_new;
                st.beta = rz / st.rz;
                st.rz = rz;
                if (a.bhist) a.bhist[(int64_t)rhs * a.hist_stride + st.iters - 1] = st.beta;
            }
            a.counter[rhs] = 0;
        }
    }
}

// t = Z^T v for the k coarse vectors (one warp per coarse vector per pass),
// then u = E^-1 t in the last CTA.
__global__ void k_m2l_ztr(const PcgArgs a, const V4<double>* v) {
    const int rhs = blockIdx.y;
    if (a.st && !a.st[rhs].active) return;
    const int64_t off = (int64_t)rhs * a.n_pix;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = VT / 32;
    const int k = a.k;
    // this CTA's pixel range
    const int chunk = (a.n_pix + gridDim.x - 1) / gridDim.x;
    const int i0 = blockIdx.x * chunk, i1 = min(a.n_pix, i0 + chunk);
    for (int c = warp; c < k; c += nw) {
        double s = 0.0;
        if (a.Z32) {
            // float32 products summed per lane in float32 (a few dozen terms), the lanes in float64
            const V4<float>* zc = a.Z32 + (int64_t)c * a.n_pix;
            float sf = 0.0f;
#pragma unroll 4
            for (int i = i0 + lane; i < i1; i += 32) {
                const V4<float> z = zc[i];
                const V4<double> x = v[off + i];
                sf = fmaf(z.x, d2f_trunc(x.x), fmaf(z.y, d2f_trunc(x.y), fmaf(z.z, d2f_trunc(x.z), sf)));
            }
            s = f2d_exact(sf);
        } else {
            const V4<double>* zc = a.Z + (int64_t)c * a.n_pix;
            for (int i = i0 + lane; i < i1; i += 32) s += dot3(zc[i], v[off + i]);
        }
        s = warp_sum(s);
        if (lane == 0) a.partial[((int64_t)blockIdx.x * a.nrhs + rhs) * k + c] = s;
    }
    if (last_block(a.counter, rhs)) {
        __shared__ double t[MM_K_MAX];
        for (int c = warp; c < k; c += nw) {
            const double s = warp_gather(a.partial, gridDim.x, (int64_t)a.nrhs * k, (int64_t)rhs * k + c);
            if (lane == 0) t[c] = s;
        }
        __syncthreads();
        const double* Einv = a.Einv + (int64_t)rhs * a.einv_stride;
        for (int c = threadIdx.x; c < k; c += VT) {
            double s = 0.0;
            for (int j = 0; j < k; ++j) s += Einv[c * k + j] * t[j];
            a.u[(int64_t)rhs * k + c] = s;
        }
        if (threadIdx.x == 0) a.counter[rhs] = 0;
    }
}

// out = M_BD (v - AZ u) + Z u  (Sect. 3.2, Eq. m2l); with finalize_beta >= 0
// it also forms v^T out and updates rz/beta like k_bd_dot.
__global__ void k_m2l_apply(const PcgArgs a, const V4<double>* v, V4<double>* out, int finalize_beta) {
    const int rhs = blockIdx.y;
    if (a.st && !a.st[rhs].active) return;
    const int64_t off = (int64_t)rhs * a.n_pix;
    __shared__ double u[MM_K_MAX];
    __shared__ float uf[MM_K_MAX];
    for (int c = threadIdx.x; c < a.k; c += VT) {
        u[c] = a.u[(int64_t)rhs * a.k + c];
        uf[c] = d2f_trunc(u[c]);
    }
    __syncthreads();
    double acc[1] = {0.0};
    const V4<double>* AZ = a.AZ + (int64_t)rhs * a.az_stride;
    PIX_LOOP(i) {
        V4<double> y = v[off + i];
        V4<double> zu{0, 0, 0, 0};
        if (a.Z32) {
            // the coarse sums AZ u and Z u in float32 (mixed precision), the rest in float64
            float ax = 0.0f, ay = 0.0f, az = 0.0f, zx = 0.0f, zy = 0.0f, zz = 0.0f;
#pragma unroll 8
            for (int c = 0; c < a.k; ++c) {
                const V4<float> azc = a.AZ32[(int64_t)c * a.n_pix + i];
                const V4<float> zc = a.Z32[(int64_t)c * a.n_pix + i];
                const float uc = uf[c];
                ax = fmaf(azc.x, uc, ax);
                ay = fmaf(azc.y, uc, ay);
                az = fmaf(azc.z, uc, az);
                zx = fmaf(zc.x, uc, zx);
                zy = fmaf(zc.y, uc, zy);
                zz = fmaf(zc.z, uc, zz);
            }
            y.x -= f2d_exact(ax);
            y.y -= f2d_exact(ay);
            y.z -= f2d_exact(az);
            zu = V4<double>{f2d_exact(zx), f2d_exact(zy), f2d_exact(zz), 0.0};
        } else
        for (int c = 0; c < a.k; ++c) {
            const V4<double> azc = AZ[(int64_t)c * a.n_pix + i];
            const V4<double> zc = a.Z[(int64_t)c * a.n_pix + i];
            const double uc = u[c];
            y.x -= azc.x * uc;
            y.y -= azc.y * uc;
            y.z -= azc.z * uc;
            zu.x += zc.x * uc;
            zu.y += zc.y * uc;
            zu.z += zc.z * uc;
        }
        V4<double> o = bd_mul(bd_of(a, rhs, i), y);
        o.x += zu.x;
        o.y += zu.y;
        o.z += zu.z;
        out[off + i] = o;
        acc[0] += dot3(v[off + i], o);
    }
    if (finalize_beta < 0) return;
    block_partials<1>(acc, a.partial + ((int64_t)blockIdx.x * a.nrhs + rhs));
    if (last_block(a.counter, rhs)) {
        const double rz = gather_partial<1>(a.partial, gridDim.x, a.nrhs, rhs, 0);
        if (threadIdx.x == 0) {
            RhsState& st = a.st[rhs];
            st.beta = finalize_beta ? rz / st.rz : 0.0;
            st.rz = rz;
            a.counter[rhs] = 0;
        }
    }
}

// Lanczos vectors of M_BD A from PCG with M_BD: v_j = z_j / sqrt(r_j^T z_j)
// (right-hand side 0), stored while j < harvest_m.
__global__ void k_harvest(const PcgArgs a) {
    const RhsState st = a.st[0];
    if (!st.active || st.iters >= a.harvest_m) return;
    const double sc = 1.0 / sqrt(st.rz);
    V4<double>* w = a.harvest + (int64_t)st.iters * a.n_pix;
    for (int i = blockIdx.x * VT + threadIdx.x; i < a.n_pix; i += gridDim.x * VT) {
        const V4<double> z = a.z[i];
        w[i] = V4<double>{z.x * sc, z.y * sc, z.z * sc, 0.0};
    }
}
void launch_harvest(const PcgArgs& a, cudaStream_t s) {
    k_harvest<<<a.grid_x, VT, 0, s>>>(a);
    count_launches(1);
}

void launch_pcg_init(const PcgArgs& a, const V4<double>* b, cudaStream_t s) {
    k_pcg_init<<<dim3(a.grid_x, a.nrhs), VT, 0, s>>>(a, b);
    count_launches(1);
}
void launch_pcg_src(const PcgArgs& a, int first, cudaStream_t s) {
    k_pcg_src<<<dim3(a.grid_x, a.nrhs), VT, 0, s>>>(a, first);
    count_launches(1);
}
void launch_pcg_pq(const PcgArgs& a, cudaStream_t s) {
    k_pcg_pq<<<dim3(a.grid_x, a.nrhs), VT, 0, s>>>(a);
    count_launches(1);
}
void launch_pcg_update(const PcgArgs& a, int two_level, cudaStream_t s) {
    if (two_level) {
        k_pcg_update<1><<<dim3(a.grid_x, a.nrhs), VT, 0, s>>>(a);
        count_launches(1);
    }
    else {
        k_pcg_update<0><<<dim3(a.grid_x, a.nrhs), VT, 0, s>>>(a);
        count_launches(1);
    }
}
void launch_precond_bd_dot(const PcgArgs& a, int finalize_beta, cudaStream_t s) {
    k_bd_dot<<<dim3(a.grid_x, a.nrhs), VT, 0, s>>>(a, finalize_beta);
    count_launches(1);
}
void launch_m2l_ztr(const PcgArgs& a, const V4<double>* v, cudaStream_t s) {
    k_m2l_ztr<<<dim3(a.grid_x, a.nrhs), VT, 0, s>>>(a, v);
    count_launches(1);
}
void launch_m2l_apply(const PcgArgs& a, const V4<double>* v, V4<double>* out, int finalize_beta, cudaStream_t s) {
    k_m2l_apply<<<dim3(a.grid_x, a.nrhs), VT, 0, s>>>(a, v, out, finalize_beta);
    count_launches(1);
}

// ---------------- tall-skinny float64 products ----------------
__global__ void k_multidot(const double* X, int64_t ldx, int m, const double* v, int64_t n, double* h,
                           double* partial, unsigned* counter) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = VT / 32;
    const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    for (int r = warp; r < m; r += nw) {
        const double* xr = X + (int64_t)r * ldx;
        double s = 0.0;
        for (int64_t i = i0 + lane; i < i1; i += 32) s += xr[i] * v[i];
        s = warp_sum(s);
        if (lane == 0) partial[(int64_t)blockIdx.x * m + r] = s;
    }
    if (last_block(counter, 0)) {
        for (int r = warp; r < m; r += nw) {
            const double s = warp_gather(partial, gridDim.x, m, r);
            if (lane == 0) h[r] = s;
        }
        if (threadIdx.x == 0) counter[0] = 0;
    }
}
void launch_multidot(const double* X, int64_t ldx, int m, const double* v, int64_t n, double* h, double* partial,
                     unsigned* counter, int grid_x, cudaStream_t s) {
    if (m <= 0) return;
    k_multidot<<<grid_x, VT, 0, s>>>(X, ldx, m, v, n, h, partial, counter);
    count_launches(1);
}

__global__ void k_sub_combo(const double* X, int64_t ldx, int m, const double* h, double* v, int64_t n) {
    extern __shared__ double hs[];
    for (int r = threadIdx.x; r < m; r += VT) hs[r] = h[r];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)VT + threadIdx.x; i < n; i += (int64_t)gridDim.x * VT) {
        double acc = v[i];
        for (int r = 0; r < m; ++r) acc -= X[(int64_t)r * ldx + i] * hs[r];
        v[i] = acc;
    }
}
void launch_sub_combo(const double* X, int64_t ldx, int m, const double* h, double* v, int64_t n, cudaStream_t s) {
    if (m <= 0) return;
    k_sub_combo<<<grid_for(n), VT, m * sizeof(double), s>>>(X, ldx, m, h, v, n);
    count_launches(1);
}

// Y[c][i] = sum_r X[r][i] C[r*kc + c], eight outputs per pass.
__global__ void k_combo(const double* X, int64_t ldx, int m, const double* C, int kc, double* Y, int64_t ldy,
                        int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)VT + threadIdx.x; i < n; i += (int64_t)gridDim.x * VT) {
        for (int c0 = 0; c0 < kc; c0 += 8) {
            double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int r = 0; r < m; ++r) {
                const double xv = X[(int64_t)r * ldx + i];
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    if (c0 + c < kc) acc[c] += xv * C[(int64_t)r * kc + c0 + c];
            }
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (c0 + c < kc) Y[(int64_t)(c0 + c) * ldy + i] = acc[c];
        }
    }
}
void launch_combo(const double* X, int64_t ldx, int m, const double* C, int kc, double* Y, int64_t ldy, int64_t n,
                  cudaStream_t s) {
    if (kc <= 0) return;
    k_combo<<<grid_for(n), VT, 0, s>>>(X, ldx, m, C, kc, Y, ldy, n);
    count_launches(1);
}

void launch_gram(const double* X, int mx, const double* Y, int my, int64_t ld, int64_t n, double* G, double* partial,
                 unsigned* counter, int grid_x, cudaStream_t s) {
    // column j of G^T: G[i][j] = X_i . Y_j, as multidots against each Y_j
    for (int j = 0; j < my; ++j) {
        k_multidot<<<grid_x, VT, 0, s>>>(X, ld, mx, Y + (int64_t)j * ld, n, G + (int64_t)j * mx, partial, counter);
        count_launches(1);
    }
}

__global__ void k_scale(double* v, int64_t n, double f) {
    for (int64_t i = blockIdx.x * (int64_t)VT + threadIdx.x; i < n; i += (int64_t)gridDim.x * VT) v[i] *= f;
}
void launch_scale_host(double* v, int64_t n, double f, cudaStream_t s) {
    if (n > 0) {
        k_scale<<<grid_for(n), VT, 0, s>>>(v, n, f);
        count_launches(1);
    }
}

}  // namespace mm

namespace mm {

// r_out = b - q (float64), and ||r_out||^2 per right-hand side into norms[rhs].
__global__ void k_residual(const V4<double>* b, const V4<double>* q, V4<double>* r_out, double* norms, int n_pix,
                           int nrhs, double* partial, unsigned* counter) {
    const int rhs = blockIdx.y;
    const int64_t off = (int64_t)rhs * n_pix;
    double acc[1] = {0.0};
    for (int i = blockIdx.x * VT + threadIdx.x; i < n_pix; i += gridDim.x * VT) {
        const V4<double> bv = b[off + i], qv = q[off + i];
        const V4<double> rv{bv.x - qv.x, bv.y - qv.y, bv.z - qv.z, 0.0};
        if (r_out) r_out[off + i] = rv;
        acc[0] += dot3(rv, rv);
    }
    block_partials<1>(acc, partial + ((int64_t)blockIdx.x * nrhs + rhs));
    if (last_block(counter, rhs)) {
        const double v = gather_partial<1>(partial, gridDim.x, nrhs, rhs, 0);
        if (threadIdx.x == 0) {
            norms[rhs] = v;
            counter[rhs] = 0;
        }
    }
}
void launch_residual(const V4<double>* b, const V4<double>* q, V4<double>* r_out, double* norms, int n_pix, int nrhs,
                     double* partial, unsigned* counter, int grid_x, cudaStream_t s) {
    k_residual<<<dim3(grid_x, nrhs), VT, 0, s>>>(b, q, r_out, norms, n_pix, nrhs, partial, counter);
    count_launches(1);
}

// y += x over n doubles, only for right-hand sides whose mask entry is set.
__global__ void k_axpy_masked(double* y, const double* x, int64_t n_per, const int32_t* mask) {
    const int rhs = blockIdx.y;
    if (mask && !mask[rhs]) return;
    const int64_t off = (int64_t)rhs * n_per;
    for (int64_t i = blockIdx.x * (int64_t)VT + threadIdx.x; i < n_per; i += (int64_t)gridDim.x * VT)
        y[off + i] += x[off + i];
}
void launch_axpy_masked(double* y, const double* x, int64_t n_per, int nrhs, const int32_t* mask, cudaStream_t s) {
    if (n_per <= 0 || nrhs <= 0) return;
    k_axpy_masked<<<dim3(grid_for(n_per), nrhs), VT, 0, s>>>(y, x, n_per, mask);
    count_launches(1);
}

}  // namespace mm
