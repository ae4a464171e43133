// Fused A x = P^T W P x and b = P^T W d kernels.
//
// One CTA handles one pair of output segments (see Seg).  Per pair it
//   1. gathers y_t = I_p + Q_p cos 2psi_t + U_p sin 2psi_t over the segment
//      plus a lambda halo on each side, clipped to the block (Sect. 2,
//      Eq. datamodel), or reads d_t for the right-hand side;
//   2. applies the block's banded Toeplitz weight W (Sect. 2, Eq. estimator)
//      -- FFT variant: both segments ride in one complex FFT of length L
//      (real part / imaginary part), are multiplied by the real spectrum of
//      the symmetric band and transformed back (overlap-save: the central
//      L - 2 lambda outputs are exact linear-convolution values);
//      -- direct variant: the band sum in shared memory;
//   3. scatters z_t (1, cos 2psi_t, sin 2psi_t) into the map (P^T), first
//      summing runs of equal consecutive pixels inside each warp so one
//      atomic carries a whole run.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "df64.cuh"

namespace mm {


constexpr int DIRECT_NT = 256;

// Padded shared-memory index: one spare element every 16 keeps the strided
// butterfly accesses of the late passes spread over the banks.
__device__ __forceinline__ int sidx(int i) { return i + (i >> 4); }

template <typename T> __device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) { return {a.x - b.x, a.y - b.y}; }

// float32 complex sums as one packed two-lane instruction (add/sub/fma .f32x2,
// sm_100 and later): the same round-to-nearest result per lane as two scalar
// operations, half the issue slots in the butterflies.
__device__ __forceinline__ unsigned long long pk2(float x, float y) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ C2<float> upk2(unsigned long long r) {
    C2<float> c;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(c.x), "=f"(c.y) : "l"(r));
    return c;
}
template <> __device__ __forceinline__ C2<float> cadd(C2<float> a, C2<float> b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a.x, a.y)), "l"(pk2(b.x, b.y)));
    return upk2(r);
}
template <> __device__ __forceinline__ C2<float> csub(C2<float> a, C2<float> b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pk2(a.x, a.y)), "l"(pk2(b.x, b.y)));
    return upk2(r);
}
// d -/+ i e = (d.x + s e.y, d.y - s e.x): one fma.f32x2 of the swapped pair
// (e.y, e.x) with multipliers (s, -s), s = +-1 (exact multiplies, one rounding)
__device__ __forceinline__ C2<float> c_minus_i(C2<float> d, C2<float> e, float sgn) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pk2(e.y, e.x)), "l"(pk2(sgn, -sgn)), "l"(pk2(d.x, d.y)));
    return upk2(r);
}
template <typename T> __device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

__device__ __forceinline__ C2<float> ldtw(const C2<float>* tw, int e) {
    float2 v = __ldg(reinterpret_cast<const float2*>(tw) + e);
    return {v.x, v.y};
}
__device__ __forceinline__ C2<double> ldtw(const C2<double>* tw, int e) {
    double2 v = __ldg(reinterpret_cast<const double2*>(tw) + e);
    return {v.x, v.y};
}
__device__ __forceinline__ C2<df> ldtw(const C2<df>* tw, int e) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(tw) + e);
    return {df(v.x, v.y), df(v.z, v.w)};
}

// Accumulator element type of the scatter: float64 atomics for double-float.
template <typename T> struct AccT { using type = T; };
template <> struct AccT<df> { using type = double; };

__device__ __forceinline__ float ldval(const float* p) { return __ldg(p); }
__device__ __forceinline__ double ldval(const double* p) { return __ldg(p); }
__device__ __forceinline__ df ldval(const df* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return df(v.x, v.y);
}
__device__ __forceinline__ float shfl_down_t(float v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double shfl_down_t(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ df shfl_down_t(df v, int d) { return shfl_down(v, d); }

// ---- small forward DFTs in registers, natural order in and out, W_R = e^{-2 pi i / R} ----
template <typename T> __device__ __forceinline__ void dft4(C2<T>& a0, C2<T>& a1, C2<T>& a2, C2<T>& a3) {
    const C2<T> s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = {d02.x + d13.y, d02.y - d13.x};   // d02 - i d13
    a3 = {d02.x - d13.y, d02.y + d13.x};   // d02 + i d13
}
template <> __device__ __forceinline__ void dft4(C2<float>& a0, C2<float>& a1, C2<float>& a2, C2<float>& a3) {
    const C2<float> s02 = cadd(a0, a2), d02 = csub(a0, a2), s13 = cadd(a1, a3), d13 = csub(a1, a3);
    a0 = cadd(s02, s13);
    a2 = csub(s02, s13);
    a1 = c_minus_i(d02, d13, 1.0f);    // d02 - i d13
    a3 = c_minus_i(d02, d13, -1.0f);   // d02 + i d13
}

template <typename T, int R> struct Dft;
template <typename T> struct Dft<T, 2> {
    static __device__ __forceinline__ void run(C2<T>* a) {
        const C2<T> t = a[0];
        a[0] = cadd(t, a[1]);
        a[1] = csub(t, a[1]);
    }
};
template <typename T> struct Dft<T, 4> {
    static __device__ __forceinline__ void run(C2<T>* a) { dft4(a[0], a[1], a[2], a[3]); }
};
template <typename T> struct Dft<T, 8> {
    static __device__ __forceinline__ void run(C2<T>* a) {
        constexpr T r2 = T(0.70710678118654752440);
        // n = 2 n1 + n2, k = k1 + 4 k2
        dft4(a[0], a[2], a[4], a[6]);
        dft4(a[1], a[3], a[5], a[7]);
        a[3] = cmul(a[3], C2<T>{r2, -r2});
        a[5] = C2<T>{a[5].y, -a[5].x};
        a[7] = cmul(a[7], C2<T>{-r2, -r2});
        C2<T> o[8];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) {
            o[k1] = cadd(a[2 * k1], a[2 * k1 + 1]);
            o[k1 + 4] = csub(a[2 * k1], a[2 * k1 + 1]);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = o[i];
    }
};
template <typename T> __device__ __forceinline__ void dft3(C2<T>& a0, C2<T>& a1, C2<T>& a2) {
    constexpr T h = T(0.86602540378443864676);   // sin(2 pi / 3)
    constexpr T half = T(0.5);
    const C2<T> t1 = cadd(a1, a2);
    const C2<T> u{a0.x - half * t1.x, a0.y - half * t1.y};
    const C2<T> v{h * (a1.x - a2.x), h * (a1.y - a2.y)};
    a0 = cadd(a0, t1);
    a1 = C2<T>{u.x + v.y, u.y - v.x};   // u - i v
    a2 = C2<T>{u.x - v.y, u.y + v.x};   // u + i v
}
template <typename T> struct Dft<T, 3> {
    static __device__ __forceinline__ void run(C2<T>* a) { dft3(a[0], a[1], a[2]); }
};
template <typename T> struct Dft<T, 9> {
    static __device__ __forceinline__ void run(C2<T>* a) {
        // n = 3 n1 + n2, k = k1 + 3 k2; W9^m = (cos 2 pi m / 9, -sin 2 pi m / 9)
        constexpr T c1 = T(0.76604444311897803520), s1 = T(0.64278760968653932632);
        constexpr T c2 = T(0.17364817766693034885), s2 = T(0.98480775301220805936);
        constexpr T c4 = T(-0.93969262078590838405), s4 = T(0.34202014332566873304);
#pragma unroll
        for (int n2 = 0; n2 < 3; ++n2) dft3(a[n2], a[n2 + 3], a[n2 + 6]);
        a[4] = cmul(a[4], C2<T>{c1, -s1});
        a[7] = cmul(a[7], C2<T>{c2, -s2});
        a[5] = cmul(a[5], C2<T>{c2, -s2});
        a[8] = cmul(a[8], C2<T>{c4, -s4});
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1) dft3(a[3 * k1], a[3 * k1 + 1], a[3 * k1 + 2]);
        C2<T> o[9];
#pragma unroll
        for (int k1 = 0; k1 < 3; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < 3; ++k2) o[k1 + 3 * k2] = a[3 * k1 + k2];
#pragma unroll
        for (int i = 0; i < 9; ++i) a[i] = o[i];
    }
};
template <typename T> struct Dft<T, 16> {
    static __device__ __forceinline__ void run(C2<T>* a) {
        constexpr T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173);
        constexpr T r2 = T(0.70710678118654752440);
        // n = 4 n1 + n2, k = k1 + 4 k2
#pragma unroll
        for (int n2 = 0; n2 < 4; ++n2) dft4(a[n2], a[n2 + 4], a[n2 + 8], a[n2 + 12]);
        // a[n2 + 4 k1] *= W16^(n2 k1)
        a[5] = cmul(a[5], C2<T>{c1, -s1});
        a[9] = cmul(a[9], C2<T>{r2, -r2});
        a[13] = cmul(a[13], C2<T>{s1, -c1});
        a[6] = cmul(a[6], C2<T>{r2, -r2});
        a[10] = C2<T>{a[10].y, -a[10].x};
        a[14] = cmul(a[14], C2<T>{-r2, -r2});
        a[7] = cmul(a[7], C2<T>{s1, -c1});
        a[11] = cmul(a[11], C2<T>{-r2, -r2});
        a[15] = cmul(a[15], C2<T>{-c1, s1});
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1) dft4(a[4 * k1], a[4 * k1 + 1], a[4 * k1 + 2], a[4 * k1 + 3]);
        C2<T> o[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) o[k1 + 4 * k2] = a[4 * k1 + k2];
#pragma unroll
        for (int i = 0; i < 16; ++i) a[i] = o[i];
    }
};

// Powers w^q, q < R, of one twiddle, each a product of two earlier powers
// (depth <= 4), from a single table load per butterfly.
template <typename T, int R>
__device__ __forceinline__ void twiddle_powers(C2<T> w1, C2<T>* w) {
    w[1] = w1;
#pragma unroll
    for (int q = 2; q < R; ++q) {
        int hi = 1;
        while (hi * 2 <= q) hi *= 2;
        w[q] = (hi == q) ? cmul(w[q / 2], w[q / 2]) : cmul(w[hi], w[q - hi]);
    }
}

// Decimation-in-frequency pass of radix R over spans of S points (in place):
// for each butterfly j < S/R of each span, DFT_R over elements j + r S/R,
// then output q times W_S^(j q) = W_L^(j q L/S).  After all passes the
// transform sits in mixed-radix digit-reversed order.
template <typename T, int R>
__device__ __forceinline__ void dif_pass(C2<T>* s, const C2<T>* __restrict__ tw, int L, int S) {
    const int Sr = S / R;
    const int nbf = L / R;
    const int tstep = L / S;
    for (int bf = threadIdx.x; bf < nbf; bf += blockDim.x) {
        const int g = bf / Sr;
        const int j = bf - g * Sr;
        const int base = g * S + j;
        C2<T> w1{T(1), T(0)};
        if (Sr > 1) w1 = ldtw(tw, j * tstep);
        C2<T> a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = s[sidx(base + r * Sr)];
        Dft<T, R>::run(a);
        if (Sr > 1) {
            C2<T> w[R];
            twiddle_powers<T, R>(w1, w);
#pragma unroll
            for (int q = 1; q < R; ++q) a[q] = cmul(a[q], w[q]);
        }
#pragma unroll
        for (int q = 0; q < R; ++q) s[sidx(base + q * Sr)] = a[q];
    }
}

// The matching decimation-in-time pass in the conjugate domain: element q
// times W_S^(j q), then DFT_R.  Run on conj(X) in the reverse pass order it
// yields L * conj(x): the exact inverse of the DIF passes.
template <typename T, int R>
__device__ __forceinline__ void dit_pass(C2<T>* s, const C2<T>* __restrict__ tw, int L, int S) {
    const int Sr = S / R;
    const int nbf = L / R;
    const int tstep = L / S;
    for (int bf = threadIdx.x; bf < nbf; bf += blockDim.x) {
        const int g = bf / Sr;
        const int j = bf - g * Sr;
        const int base = g * S + j;
        C2<T> w1{T(1), T(0)};
        if (Sr > 1) w1 = ldtw(tw, j * tstep);
        C2<T> a[R];
#pragma unroll
        for (int q = 0; q < R; ++q) a[q] = s[sidx(base + q * Sr)];
        if (Sr > 1) {
            C2<T> w[R];
            twiddle_powers<T, R>(w1, w);
#pragma unroll
            for (int q = 1; q < R; ++q) a[q] = cmul(a[q], w[q]);
        }
        Dft<T, R>::run(a);
#pragma unroll
        for (int r = 0; r < R; ++r) s[sidx(base + r * Sr)] = a[r];
    }
}

template <typename T, bool DIT>
__device__ __forceinline__ void run_pass(C2<T>* s, const C2<T>* tw, int L, int R, int S) {
    switch (R) {
        case 16: DIT ? dit_pass<T, 16>(s, tw, L, S) : dif_pass<T, 16>(s, tw, L, S); break;
        case 9: DIT ? dit_pass<T, 9>(s, tw, L, S) : dif_pass<T, 9>(s, tw, L, S); break;
        case 8: DIT ? dit_pass<T, 8>(s, tw, L, S) : dif_pass<T, 8>(s, tw, L, S); break;
        case 4: DIT ? dit_pass<T, 4>(s, tw, L, S) : dif_pass<T, 4>(s, tw, L, S); break;
        case 3: DIT ? dit_pass<T, 3>(s, tw, L, S) : dif_pass<T, 3>(s, tw, L, S); break;
        default: DIT ? dit_pass<T, 2>(s, tw, L, S) : dif_pass<T, 2>(s, tw, L, S); break;
    }
}

// Forward transform: the plan's passes in order (spans shrink from L).
template <typename T>
__device__ void fft_dif(C2<T>* s, const C2<T>* tw, const FftPasses& fp) {
    for (int p = 0; p < fp.npass; ++p) {
        run_pass<T, false>(s, tw, fp.L, fp.radix[p], fp.span[p]);
        __syncthreads();
    }
}
template <typename T>
__device__ void fft_dit_conj(C2<T>* s, const C2<T>* tw, const FftPasses& fp) {
    for (int p = fp.npass - 1; p >= 0; --p) {
        run_pass<T, true>(s, tw, fp.L, fp.radix[p], fp.span[p]);
        __syncthreads();
    }
}

// ---- compile-time plans for the lengths the planner uses most ----
// Same pass order as the host planner: a radix-9 or radix-3 pass, radix-16
// passes, then one radix 2, 4 or 8 pass; all spans and index divisors are
// constants, so the butterfly addressing folds to shifts and multiplies.
struct CtPlan {
    int np;
    int r[8];
    int s[8];
    int toff[8];   // offset of pass p in the per-pass twiddle table (see ct_pass)
};
// MAXR: largest power-of-two radix (16, or 8 where registers are scarce).
__host__ __device__ constexpr CtPlan make_ct_plan(int L, int MAXR = 16) {
    CtPlan p{0, {0, 0, 0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0, 0, 0}};
    int rest = L, span = L;
    if (rest % 9 == 0) {
        p.r[p.np] = 9; p.s[p.np] = span; span /= 9; rest /= 9; ++p.np;
    } else if (rest % 3 == 0) {
        p.r[p.np] = 3; p.s[p.np] = span; span /= 3; rest /= 3; ++p.np;
    }
    while (rest % MAXR == 0 && p.np < 8) {
        p.r[p.np] = MAXR; p.s[p.np] = span; span /= MAXR; rest /= MAXR; ++p.np;
    }
    if (MAXR == 8 && rest == 2 && p.np > 0 && p.r[p.np - 1] == 8 && p.np < 8) {
        // end in 4, 4 rather than 8, 2 (the host planner's rule)
        --p.np;
        span *= 8;
        p.r[p.np] = 4; p.s[p.np] = span; span /= 4; ++p.np;
        p.r[p.np] = 4; p.s[p.np] = span; ++p.np;
    } else if (rest > 1 && rest < MAXR && (rest == 8 || rest == 4 || rest == 2)) {
        p.r[p.np] = rest; p.s[p.np] = span; ++p.np;
    }
    int off = 0;
    for (int i = 0; i < p.np; ++i) {
        p.toff[i] = off;
        off += (p.r[i] - 1) * (p.s[i] / p.r[i]);
    }
    return p;
}

// Passes whose twiddle powers come from the per-pass table instead of being
// formed from one twiddle: every pass for float64 and double-float, where a
// complex product costs tens of float32 instructions; none for float32, where
// the table loads of a radix-16 butterfly do not fit the register budget of
// two 512-thread CTAs per SM.
template <typename T> __host__ __device__ constexpr bool table_twiddles(int) {
    return sizeof(T) != 4;
}

// Padded index of point base + r Sr of a butterfly, as sidx(base) plus a
// compile-time offset.  Exact when the butterfly's points keep their place
// within 16-point groups: Sr a multiple of 16 (whole groups apart), S a
// multiple of 16 with Sr dividing 16 (the points of one group stay in it),
// or S dividing 16 (the whole butterfly inside one group).
template <int S, int Sr>
__host__ __device__ constexpr bool pad_const() {
    return Sr % 16 == 0 || (S % 16 == 0 && 16 % Sr == 0) || 16 % S == 0;
}
template <int S, int Sr>
__host__ __device__ constexpr int pad_offset(int r) {
    return Sr % 16 == 0 ? r * (Sr + Sr / 16) : (S % 16 == 0 ? r * Sr + ((r * Sr) >> 4) : r * Sr);
}
template <int S, int Sr>
__device__ __forceinline__ int pad_index(int b0, int base, int r) {
    if constexpr (pad_const<S, Sr>()) return b0 + pad_offset<S, Sr>(r);
    else return sidx(base + r * Sr);
}

// One pass of radix R over spans of S points.  Twiddle powers W_S^(j q):
// formed from W_L^(j L/S) (one table load), or, with TAB, read from the
// pass's table ptab[(q - 1) Sr + j] (neighbouring butterflies read
// neighbouring entries).
template <typename T, int R, int S, int L, int NT, bool DIT, bool TAB = false>
__device__ __forceinline__ void ct_pass(C2<T>* s, const C2<T>* __restrict__ tw,
                                        const C2<T>* __restrict__ ptab = nullptr) {
    constexpr int Sr = S / R;
    constexpr int nbf = L / R;
    constexpr int tstep = L / S;
#pragma unroll 1
    for (int bf = threadIdx.x; bf < nbf; bf += NT) {
        const int g = bf / Sr;
        const int j = bf - g * Sr;
        const int base = g * S + j;
        const int b0 = sidx(base);
        C2<T> w1{T(1), T(0)};
        if (Sr > 1 && !TAB) w1 = ldtw(tw, j * tstep);
        C2<T> a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = s[pad_index<S, Sr>(b0, base, r)];
        if (!DIT) Dft<T, R>::run(a);
        if (Sr > 1) {
            if constexpr (TAB) {
#pragma unroll
                for (int q = 1; q < R; ++q) a[q] = cmul(a[q], ldtw(ptab, (q - 1) * Sr + j));
            } else {
                C2<T> w[R];
                twiddle_powers<T, R>(w1, w);
#pragma unroll
                for (int q = 1; q < R; ++q) a[q] = cmul(a[q], w[q]);
            }
        }
        if (DIT) Dft<T, R>::run(a);
#pragma unroll
        for (int q = 0; q < R; ++q) s[pad_index<S, Sr>(b0, base, q)] = a[q];
    }
}

// Passes P .. PEND - 1 of the forward transform (PEND < 0: to the last pass).
// tt: the per-pass twiddle table (null: powers formed from tw in every pass).
template <typename T, int L, int NT, int MAXR, int P, int PEND = -1>
__device__ __forceinline__ void ct_dif(C2<T>* s, const C2<T>* tw, const C2<T>* tt = nullptr) {
    constexpr CtPlan pl = make_ct_plan(L, MAXR);
    constexpr int end = PEND < 0 ? pl.np : PEND;
    if constexpr (P < end) {
        if (tt && table_twiddles<T>(P)) ct_pass<T, pl.r[P], pl.s[P], L, NT, false, true>(s, tw, tt + pl.toff[P]);
        else ct_pass<T, pl.r[P], pl.s[P], L, NT, false>(s, tw);
        __syncthreads();
        ct_dif<T, L, NT, MAXR, P + 1, PEND>(s, tw, tt);
    }
}
template <typename T, int L, int NT, int MAXR, int P>
__device__ __forceinline__ void ct_dit(C2<T>* s, const C2<T>* tw, const C2<T>* tt = nullptr) {
    constexpr CtPlan pl = make_ct_plan(L, MAXR);
    if constexpr (P >= 0) {
        if (tt && table_twiddles<T>(P)) ct_pass<T, pl.r[P], pl.s[P], L, NT, true, true>(s, tw, tt + pl.toff[P]);
        else ct_pass<T, pl.r[P], pl.s[P], L, NT, true>(s, tw);
        __syncthreads();
        ct_dit<T, L, NT, MAXR, P - 1>(s, tw, tt);
    }
}

// ---- pointing weights ----
// float32: __sincosf on 2 psi - pi in [-pi, pi), where its error stays near
// 4e-7; cos 2psi = -cos(2psi - pi), sin 2psi = -sin(2psi - pi).
__device__ __forceinline__ void weights(const FilterArgs& a, int64_t t, float& c, float& s) {
    const float x = fmaf(2.0f, __ldg(a.psi + t), -3.14159265358979323846f);
    float sn, cs;
    __sincosf(x, &sn, &cs);
    c = -cs;
    s = -sn;
}
__device__ __forceinline__ void weights(const FilterArgs& a, int64_t t, double& c, double& s) {
    const double2 v = __ldg(a.cs64 + t);
    c = v.x;
    s = v.y;
}
__device__ __forceinline__ void weights(const FilterArgs& a, int64_t t, df& c, df& s) {
    const float4 v = __ldg(a.csdf + t);
    c = df(v.x, v.y);
    s = df(v.z, v.w);
}

__device__ __forceinline__ void weights_from(const FilterArgs& a, int64_t t, float psi, float& c, float& s) {
    const float x = fmaf(2.0f, psi, -3.14159265358979323846f);
    float sn, cs;
    __sincosf(x, &sn, &cs);
    c = -cs;
    s = -sn;
}
__device__ __forceinline__ void weights_from(const FilterArgs& a, int64_t t, float, double& c, double& s) {
    const double2 v = __ldg(a.cs64 + t);
    c = v.x;
    s = v.y;
}

__device__ __forceinline__ void weights_from(const FilterArgs& a, int64_t t, float, df& c, df& s) {
    const float4 v = __ldg(a.csdf + t);
    c = df(v.x, v.y);
    s = df(v.z, v.w);
}

template <typename T>
__device__ __forceinline__ V4<T> ldmap(const V4<T>* m);
template <>
__device__ __forceinline__ V4<float> ldmap(const V4<float>* m) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(m));
    return {v.x, v.y, v.z, v.w};
}
template <>
__device__ __forceinline__ V4<double> ldmap(const V4<double>* m) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(m));
    const double2 b = __ldg(reinterpret_cast<const double2*>(m) + 1);
    return {a.x, a.y, b.x, b.y};
}

template <>
__device__ __forceinline__ V4<df> ldmap(const V4<df>* m) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(m));
    const float4 b = __ldg(reinterpret_cast<const float4*>(m) + 1);
    return {df(a.x, a.y), df(a.z, a.w), df(b.x, b.y), df(b.z, b.w)};
}

// (P x)_t for the map a.xmap: the timeline residual d_t - (P x)_t, whose
// filtered transpose is b - A x = P^T W (d - P x) (Sect. 3, Eq. linearsystem).
template <typename T>
__device__ __forceinline__ T xmap_value(const FilterArgs& a, int64_t t, int rhs) {
    const int p = __ldg(a.pix + t);
    if (p < 0) return T(0);
    T c, s;
    weights(a, t, c, s);
    const V4<T> m = ldmap<T>(reinterpret_cast<const V4<T>*>(a.xmap) + (int64_t)rhs * a.n_pix + p);
    return m.x + c * m.y + s * m.z;
}

// y_t of right-hand side `rhs`: (P x)_t, or d_t when FROM_TOD (d_t - (P x)_t
// when a residual map is given).
template <typename T, bool FROM_TOD>
__device__ __forceinline__ T sample_value(const FilterArgs& a, int64_t t, int rhs) {
    if (FROM_TOD) {
        T v = a.tod_is_float ? T(__ldg(reinterpret_cast<const float*>(a.src) + rhs * a.n_samples + t))
                             : T(__ldg(reinterpret_cast<const double*>(a.src) + rhs * a.n_samples + t));
        if (sizeof(T) > 4 && a.xmap) v = v - xmap_value<T>(a, t, rhs);
        return v;
    } else {
        const int p = __ldg(a.pix + t);
        if (p < 0) return T(0);
        T c, s;
        weights(a, t, c, s);
        const V4<T> m = ldmap<T>(reinterpret_cast<const V4<T>*>(a.src) + (int64_t)rhs * a.n_pix + p);
        return m.x + c * m.y + s * m.z;
    }
}

// Gather of a segment pair into s[i] = (y_A[out0_A - lambda + i], y_B[...]),
// zero outside each block.  Loads are issued GB iterations at a time (index
// and angle first, then the map entries) to keep many requests in flight.
template <typename T, bool FROM_TOD>
__device__ __forceinline__ void gather_pair(const FilterArgs& a, const Seg& A, const Seg& B, bool actA, bool actB,
                                            C2<T>* s, int L, int lam) {
    constexpr int GB = 4;
    const int nt = blockDim.x;
    for (int i0 = threadIdx.x; i0 < L; i0 += nt * GB) {
        int pa[GB], pb[GB];
        float fa[GB], fb[GB];
        T ya[GB], yb[GB];
#pragma unroll
        for (int g = 0; g < GB; ++g) {
            const int i = i0 + g * nt;
            const int64_t ta = A.out0 - lam + i, tb = B.out0 - lam + i;
            const bool va = actA && i < L && ta >= A.lo && ta < A.hi;
            const bool vb = actB && i < L && tb >= B.lo && tb < B.hi;
            pa[g] = -1;
            pb[g] = -1;
            ya[g] = T(0);
            yb[g] = T(0);
            if (FROM_TOD) {
                if (va) ya[g] = sample_value<T, true>(a, ta, A.rhs);
                if (vb) yb[g] = sample_value<T, true>(a, tb, B.rhs);
            } else {
                if (va) {
                    pa[g] = __ldg(a.pix + ta);
                    if (sizeof(T) == 4) fa[g] = __ldg(a.psi + ta);
                }
                if (vb) {
                    pb[g] = __ldg(a.pix + tb);
                    if (sizeof(T) == 4) fb[g] = __ldg(a.psi + tb);
                }
            }
        }
        if (!FROM_TOD) {
            const V4<T>* mapA = reinterpret_cast<const V4<T>*>(a.src) + (int64_t)A.rhs * a.n_pix;
            const V4<T>* mapB = reinterpret_cast<const V4<T>*>(a.src) + (int64_t)B.rhs * a.n_pix;
            V4<T> ma[GB], mb[GB];
#pragma unroll
            for (int g = 0; g < GB; ++g) {
                if (pa[g] >= 0) ma[g] = ldmap<T>(mapA + pa[g]);
                if (pb[g] >= 0) mb[g] = ldmap<T>(mapB + pb[g]);
            }
#pragma unroll
            for (int g = 0; g < GB; ++g) {
                const int i = i0 + g * nt;
                if (pa[g] >= 0) {
                    T c, sn;
                    weights_from(a, A.out0 - lam + i, fa[g], c, sn);
                    ya[g] = ma[g].x + c * ma[g].y + sn * ma[g].z;
                }
                if (pb[g] >= 0) {
                    T c, sn;
                    weights_from(a, B.out0 - lam + i, fb[g], c, sn);
                    yb[g] = mb[g].x + c * mb[g].y + sn * mb[g].z;
                }
            }
        }
#pragma unroll
        for (int g = 0; g < GB; ++g) {
            const int i = i0 + g * nt;
            if (i < L) s[sidx(i)] = C2<T>{ya[g], yb[g]};
        }
    }
}

__device__ __forceinline__ void atomic_add3(V4<float>* q, float a, float b, float c) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
    atomicAdd(reinterpret_cast<float4*>(q), make_float4(a, b, c, 0.0f));
#else
    atomicAdd(&q->x, a);
    atomicAdd(&q->y, b);
    atomicAdd(&q->z, c);
#endif
}
__device__ __forceinline__ void atomic_add3(V4<double>* q, double a, double b, double c) {
    atomicAdd(&q->x, a);
    atomicAdd(&q->y, b);
    atomicAdd(&q->z, c);
}
__device__ __forceinline__ void atomic_add3(V4<double>* q, df a, df b, df c) {
    atomicAdd(&q->x, (double)a);
    atomicAdd(&q->y, (double)b);
    atomicAdd(&q->z, (double)c);
}

// Warp-cooperative P^T: every lane holds one sample (p < 0: nothing).
// Consecutive lanes with equal p form a run; a suffix sum inside each run
// leaves the run total on its first lane, which issues one atomic.  The sum
// takes only as many doubling steps as the longest run in the warp needs.
template <typename T>
__device__ __forceinline__ void scatter_vals(int p, T v0, T v1, T v2, V4<typename AccT<T>::type>* q) {
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    const int pprev = __shfl_up_sync(FULL, p, 1);
    const bool head = (lane == 0) || (p != pprev);
    const unsigned heads = __ballot_sync(FULL, head);
    const unsigned above = heads & ~((2u << lane) - 1u);
    const int end = above ? (__ffs(above) - 1) : 32;
    const int need = (int)__reduce_max_sync(FULL, head ? (unsigned)(end - (int)lane) : 0u);
#pragma unroll 1
    for (int d = 1; d < need; d <<= 1) {
        const T o0 = shfl_down_t(v0, d);
        const T o1 = shfl_down_t(v1, d);
        const T o2 = shfl_down_t(v2, d);
        if ((int)lane + d < end) {
            v0 += o0;
            v1 += o1;
            v2 += o2;
        }
    }
    if (head && p >= 0) atomic_add3(q + p, v0, v1, v2);
}

template <typename T>
__device__ __forceinline__ void scatter_warp(int p, T c, T s, T z, V4<typename AccT<T>::type>* q) {
    scatter_vals<T>(p, z, z * c, z * s, q);
}

// Scatter of four consecutive outputs per lane: runs of equal pixels are
// summed in registers first, a lane's leading run joins the previous lane's
// trailing run when they share a pixel, runs strictly inside a lane's four
// samples go out directly, and the trailing runs go through the
// warp-segmented reduction.  Every output is counted once.
template <typename T>
__device__ __forceinline__ void scatter4_vals(const int (&p)[4], const T (&v0)[4], const T (&v1)[4],
                                              const T (&v2)[4], V4<typename AccT<T>::type>* q) {
    const unsigned FULL = 0xffffffffu;
    const unsigned lane = threadIdx.x & 31u;
    int kf = p[0], cur = p[0];
    T f0 = v0[0], f1 = v1[0], f2 = v2[0];
    T c0 = v0[0], c1 = v1[0], c2 = v2[0];
    bool first_done = false;
#pragma unroll
    for (int j = 1; j < 4; ++j) {
        if (p[j] == cur) {
            c0 += v0[j];
            c1 += v1[j];
            c2 += v2[j];
        } else {
            if (!first_done) {
                kf = cur;
                f0 = c0;
                f1 = c1;
                f2 = c2;
                first_done = true;
            } else if (cur >= 0) {
                atomic_add3(q + cur, c0, c1, c2);   // a run strictly inside the lane
            }
            cur = p[j];
            c0 = v0[j];
            c1 = v1[j];
            c2 = v2[j];
        }
    }
    const bool multi = first_done;
    const int prev_last = __shfl_up_sync(FULL, cur, 1);
    const bool give = multi && lane > 0 && kf == prev_last;
    const T r0 = shfl_down_t(f0, 1);
    const T r1 = shfl_down_t(f1, 1);
    const T r2 = shfl_down_t(f2, 1);
    const int rgive = __shfl_down_sync(FULL, (int)give, 1);
    if (lane < 31 && rgive) {
        c0 += r0;
        c1 += r1;
        c2 += r2;
    }
    if (multi && !give && kf >= 0) atomic_add3(q + kf, f0, f1, f2);
    scatter_vals<T>(cur, c0, c1, c2, q);
}

// Pixel indices of four consecutive samples t0..t0+3 (a vector load past L1
// when aligned); samples at or beyond the segment end come back flagged.
__device__ __forceinline__ void load4_pix(const FilterArgs& a, int64_t t0, bool act, int count, int (&p)[4]) {
    if (act && count >= 4 && (t0 & 3) == 0) {
        int4 pv;
        asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(pv.x), "=r"(pv.y), "=r"(pv.z), "=r"(pv.w)
                     : "l"(a.pix + t0));
        p[0] = pv.x; p[1] = pv.y; p[2] = pv.z; p[3] = pv.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) p[j] = (act && j < count) ? __ldg(a.pix + t0 + j) : -1;
    }
}

// Pixel and angle of four consecutive samples t0..t0+3 (vector loads when
// aligned); samples at or beyond `limit` (segment end) come back flagged.
__device__ __forceinline__ void load4(const FilterArgs& a, int64_t t0, bool act, int count, int (&p)[4],
                                      float (&ps)[4]) {
    if (act && count >= 4 && (t0 & 3) == 0) {
        // streamed past L1 (no allocation), so the map entries and tables stay cached there
        int4 pv;
        float4 fv;
        asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(pv.x), "=r"(pv.y), "=r"(pv.z), "=r"(pv.w)
                     : "l"(a.pix + t0));
        asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(fv.x), "=f"(fv.y), "=f"(fv.z), "=f"(fv.w)
                     : "l"(a.psi + t0));
        p[0] = pv.x; p[1] = pv.y; p[2] = pv.z; p[3] = pv.w;
        ps[0] = fv.x; ps[1] = fv.y; ps[2] = fv.z; ps[3] = fv.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool ok = act && j < count;
            p[j] = ok ? __ldg(a.pix + t0 + j) : -1;
            ps[j] = ok ? __ldg(a.psi + t0 + j) : 0.0f;
        }
    }
}

__device__ __forceinline__ void scatter4_f32(const FilterArgs& a, const Seg& S, bool act, int i0, const C2<float>* sm,
                                             int lam, int L, bool imag, V4<float>* q) {
    int p[4];
    float ps[4];
    const int64_t t0 = S.out0 + i0;
    load4(a, t0, act, S.n_out - i0, p, ps);
    float v0[4], v1[4], v2[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float z = 0.0f, c = 0.0f, sn = 0.0f;
        if (p[j] >= 0) {
            const C2<float> v = sm[sidx(min(lam + i0 + j, L - 1))];
            z = imag ? -v.y : v.x;
            weights_from(a, t0 + j, ps[j], c, sn);
        }
        v0[j] = z;
        v1[j] = z * c;
        v2[j] = z * sn;
    }
    scatter4_vals(p, v0, v1, v2, q);
}

template <typename T>
__device__ __forceinline__ void scatter_one(const FilterArgs& a, const Seg& S, bool act, int i, T zval) {
    int p = -1;
    T c = T(0), s = T(0), z = T(0);
    if (act && i < S.n_out) {
        const int64_t t = S.out0 + i;
        p = __ldg(a.pix + t);
        if (p >= 0) {
            weights(a, t, c, s);
            z = zval;
        }
    }
    scatter_warp<T>(p, c, s, z, reinterpret_cast<V4<typename AccT<T>::type>*>(a.dst) + (int64_t)(act ? S.rhs : 0) * a.n_pix);
}

template <typename T>
__device__ __forceinline__ bool seg_active(const FilterArgs& a, const Seg& S) {
    return S.n_out > 0 && (a.state == nullptr || a.state[S.rhs].active);
}

// ---------------- FFT overlap-save variant ----------------
// Largest power-of-two radix of the compile-time transforms: 8 for
// double-float (register pressure at 512 threads), 16 otherwise.  The host
// planner uses the same rule, so the spectra share the digit order.
template <typename T> struct MaxRadix { static constexpr int value = 16; };
template <> struct MaxRadix<df> { static constexpr int value = 8; };

template <typename T, bool FROM_TOD, int NT, int LCT>
__global__ void __launch_bounds__(NT, (sizeof(T) == 4 && NT == 256) ? 3 : 1) k_filter_fft(const FilterArgs a) {
    static_assert(sizeof(C2<T>) == 2 * sizeof(T), "complex layout");
    extern __shared__ __align__(16) unsigned char smraw[];
    C2<T>* s = reinterpret_cast<C2<T>*>(smraw);
    const Seg A = a.segs[2 * blockIdx.x];
    const Seg B = a.segs[2 * blockIdx.x + 1];
    const bool actA = seg_active<T>(a, A);
    const bool actB = seg_active<T>(a, B);
    if (!actA && !actB) return;
    const int L = LCT > 0 ? LCT : a.L;
    const int lam = actA ? A.shift : B.shift;   // left halo of this pair (lambda, or 0 for whole blocks)
    const C2<T>* tw = reinterpret_cast<const C2<T>*>(a.tw);

    gather_pair<T, FROM_TOD>(a, A, B, actA, actB, s, L, lam);
    __syncthreads();
    if constexpr (LCT > 0) ct_dif<T, LCT, NT, MaxRadix<T>::value, 0>(s, tw);
    else fft_dif<T>(s, tw, a.fp);
    const T* H = reinterpret_cast<const T*>(a.H) + (int64_t)(actA ? A.band : B.band) * L;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        const C2<T> v = s[sidx(i)];
        const T h = ldval(H + i);
        s[sidx(i)] = C2<T>{v.x * h, -v.y * h};
    }
    __syncthreads();
    if constexpr (LCT > 0)
        ct_dit<T, LCT, NT, MaxRadix<T>::value, make_ct_plan(LCT > 0 ? LCT : 64, MaxRadix<T>::value).np - 1>(s, tw);
    else fft_dit_conj<T>(s, tw, a.fp);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int vmax = max(actA ? A.n_out : 0, actB ? B.n_out : 0);
    constexpr int SB = 2;
    using Acc = typename AccT<T>::type;
    V4<Acc>* qA = reinterpret_cast<V4<Acc>*>(a.dst) + (int64_t)(actA ? A.rhs : 0) * a.n_pix;
    V4<Acc>* qB = reinterpret_cast<V4<Acc>*>(a.dst) + (int64_t)(actB ? B.rhs : 0) * a.n_pix;
    if constexpr (std::is_same<T, float>::value) {
        for (int base = warp * 128; base < vmax; base += nwarp * 128) {
            const int i0 = base + 4 * lane;
            scatter4_f32(a, A, actA, i0, s, lam, L, false, qA);
            scatter4_f32(a, B, actB, i0, s, lam, L, true, qB);
        }
        return;
    }
    for (int base = warp * 32; base < vmax; base += nwarp * 32 * SB) {
        int pa[SB], pb[SB];
        float fa[SB], fb[SB];
#pragma unroll
        for (int g = 0; g < SB; ++g) {
            const int i = base + g * nwarp * 32 + lane;
            pa[g] = -1;
            pb[g] = -1;
            if (actA && i < A.n_out) {
                pa[g] = __ldg(a.pix + A.out0 + i);
                if (sizeof(T) == 4) fa[g] = __ldg(a.psi + A.out0 + i);
            }
            if (actB && i < B.n_out) {
                pb[g] = __ldg(a.pix + B.out0 + i);
                if (sizeof(T) == 4) fb[g] = __ldg(a.psi + B.out0 + i);
            }
        }
#pragma unroll
        for (int g = 0; g < SB; ++g) {
            const int i = base + g * nwarp * 32 + lane;
            const C2<T> v = s[sidx(min(lam + i, L - 1))];
            T c = T(0), sn = T(0), za = T(0), zb = T(0);
            if (pa[g] >= 0) {
                weights_from(a, A.out0 + i, fa[g], c, sn);
                za = v.x;
            }
            scatter_warp<T>(pa[g], c, sn, za, qA);
            c = T(0);
            sn = T(0);
            if (pb[g] >= 0) {
                weights_from(a, B.out0 + i, fb[g], c, sn);
                zb = -v.y;
            }
            scatter_warp<T>(pb[g], c, sn, zb, qB);
        }
    }
}

// ---------------- whole block as a half-length complex transform ----------------
// One CTA per block.  The block's real samples y_0..y_{N-1} (zero beyond the
// block, N >= n_b + lambda, so the circular product equals the band product)
// ride as M = N/2 complex points z_m = y_{2m} + i y_{2m+1}.  With Z = DFT_M(z)
// and H the length-N spectrum of the band (real and even), the filtered
// sequence y' = W y has, for every k and its partner M - k (mod M),
//   Z'_k = alpha_k Z_k + i beta_k conj(Z_{M-k}),
//   alpha_k = ((H_k + H_{M-k}) + (H_{M-k} - H_k) sin theta_k) / 2,
//   beta_k  = -(H_{M-k} - H_k) cos theta_k / 2,   theta_k = 2 pi k / N,
// which follows from Y_k = (Z_k + conj Z_{M-k}) / 2 - i e^{-i theta_k}
// (Z_k - conj Z_{M-k}) / 2 and its inverse.  The coefficient table holds,
// per pair (k, M - k), k = 0..M/2, (alpha_k, alpha_{M-k}, beta_k) with 1/M
// folded in; the pair table holds the digit-reversed positions of k and
// M - k; both list the pairs in the order of the position of k.  Half
// the shared memory of a two-segment transform, so two CTAs share an SM and
// one's gather and scatter overlap the other's butterflies.

__device__ __forceinline__ void ld_coef(const void* C, int64_t e, float& aa, float& ab, float& be) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(C) + e);
    aa = v.x;
    ab = v.y;
    be = v.z;
}
__device__ __forceinline__ void ld_coef(const void* C, int64_t e, double& aa, double& ab, double& be) {
    const double2 u = __ldg(reinterpret_cast<const double2*>(C) + 2 * e);
    const double2 v = __ldg(reinterpret_cast<const double2*>(C) + 2 * e + 1);
    aa = u.x;
    ab = u.y;
    be = v.x;
}
__device__ __forceinline__ void ld_coef(const void* C, int64_t e, df& aa, df& ab, df& be) {
    const float4 u = __ldg(reinterpret_cast<const float4*>(C) + 2 * e);
    const float4 v = __ldg(reinterpret_cast<const float4*>(C) + 2 * e + 1);
    aa = df(u.x, u.y);
    ab = df(u.z, u.w);
    be = df(v.x, v.y);
}

// Four consecutive timeline values d_{t0..t0+3} of a segment (zero past n_out).
__device__ __forceinline__ void load4_tod(const FilterArgs& a, const Seg& S, int i0, bool act, float (&y)[4]) {
    const int64_t t0 = (int64_t)S.rhs * a.n_samples + S.out0 + i0;
    const int count = S.n_out - i0;
    if (act && a.tod_is_float && count >= 4 && (t0 & 3) == 0) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(a.src) + (t0 >> 2));
        y[0] = v.x;
        y[1] = v.y;
        y[2] = v.z;
        y[3] = v.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float v = 0.0f;
            if (act && j < count)
                v = a.tod_is_float ? __ldg(reinterpret_cast<const float*>(a.src) + t0 + j)
                                   : (float)__ldg(reinterpret_cast<const double*>(a.src) + t0 + j);
            y[j] = v;
        }
    }
}

// ---- float32 gather and scatter of the half-length kernel ----
// Both walk a block in groups of four consecutive samples.  Groups that lie
// wholly inside a block whose first sample is 16-byte aligned (every block of
// the configured scans) take unchecked 16-byte pointing loads; flagged samples
// (pixel -1) are handled without branches: the map entry of pixel 0 is read
// and the sample's value is zeroed.  The remaining groups (a ragged end, an
// unaligned start, the zero padding of the transform) take checked loads.

// pix and psi of four consecutive samples, streamed past L1 so the map
// entries and tables stay cached there
__device__ __forceinline__ void ld4_pointing(const int32_t* pp, const float* pf, int4& pv, float4& fv) {
    asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(pv.x), "=r"(pv.y), "=r"(pv.z), "=r"(pv.w)
                 : "l"(pp));
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(fv.x), "=f"(fv.y), "=f"(fv.z), "=f"(fv.w)
                 : "l"(pf));
}

// cos 2psi, sin 2psi as -cos(2psi - pi), -sin(2psi - pi): __sincosf on [-pi, pi)
__device__ __forceinline__ void neg_cs(float psi, float& nc, float& ns) {
    __sincosf(fmaf(2.0f, psi, -3.14159265358979323846f), &ns, &nc);
}

// y_t = I_p + Q_p cos 2psi + U_p sin 2psi (Sect. 2, Eq. datamodel), 0 for a flagged sample
__device__ __forceinline__ float pointed_value(int p, float psi, const float4& m) {
    float nc, ns;
    neg_cs(psi, nc, ns);
    const float y = fmaf(-ns, m.z, fmaf(-nc, m.y, m.x));
    return p >= 0 ? y : 0.0f;
}

template <int NT>
__device__ __forceinline__ void half_gather_f32_map(const FilterArgs& a, const Seg& S, C2<float>* s, int M) {
    const int ng = M >> 1;   // groups of four samples = pairs of complex points
    const float4* map = reinterpret_cast<const float4*>(a.src) + (int64_t)S.rhs * a.n_pix;
    const int32_t* pix = a.pix + S.out0;
    const float* psi = a.psi + S.out0;
    const int nfull = (S.out0 & 3) == 0 ? (S.n_out >> 2) : 0;
    int u = threadIdx.x;
    if (u < nfull) {
        int4 pv;
        float4 fv;
        ld4_pointing(pix + 4 * u, psi + 4 * u, pv, fv);
        for (; u < nfull; u += NT) {
            // the next group's pointing is requested before this group's map entries
            const int un = min(u + NT, nfull - 1);
            int4 pn;
            float4 fn;
            ld4_pointing(pix + 4 * un, psi + 4 * un, pn, fn);
            const float4 m0 = __ldg(map + max(pv.x, 0));
            const float4 m1 = __ldg(map + max(pv.y, 0));
            const float4 m2 = __ldg(map + max(pv.z, 0));
            const float4 m3 = __ldg(map + max(pv.w, 0));
            const int b = sidx(2 * u);   // points 2u, 2u + 1 share one 16-point padding group
            s[b] = C2<float>{pointed_value(pv.x, fv.x, m0), pointed_value(pv.y, fv.y, m1)};
            s[b + 1] = C2<float>{pointed_value(pv.z, fv.z, m2), pointed_value(pv.w, fv.w, m3)};
            pv = pn;
            fv = fn;
        }
    }
    for (; u < ng; u += NT) {
        float y[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int i = 4 * u + j;
            const bool ok = i < S.n_out;
            const int p = ok ? __ldg(pix + i) : -1;
            const float f = ok ? __ldg(psi + i) : 0.0f;
            y[j] = pointed_value(p, f, __ldg(map + max(p, 0)));
        }
        const int b = sidx(2 * u);
        s[b] = C2<float>{y[0], y[1]};
        s[b + 1] = C2<float>{y[2], y[3]};
    }
}

// P^T of a warp's 128 consecutive samples, four per lane in order: one atomic
// per run of equal pixels.  Within a lane, suffix sums over each run; the
// lane's last run continues into the following lanes while their first
// pixel is the same, and its continuation X(l) = a(l) + b(l) X(l + 1)
// (a = the next lane's leading run when the run continues, b = that run fills
// the next lane) is solved by doubling, taking only the steps the longest
// chain needs.  Every sample is counted once: at the first sample of its run
// inside this warp's 128.
__device__ __forceinline__ void warp_run_scatter(const int (&p)[4], float (&v0)[4], float (&v1)[4], float (&v2)[4],
                                                 V4<float>* q) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool e01 = p[0] == p[1], e12 = p[1] == p[2], e23 = p[2] == p[3];
    if (e23) { v0[2] += v0[3]; v1[2] += v1[3]; v2[2] += v2[3]; }
    if (e12) { v0[1] += v0[2]; v1[1] += v1[2]; v2[1] += v2[2]; }
    if (e01) { v0[0] += v0[1]; v1[0] += v1[1]; v2[0] += v2[1]; }
    const bool whole = e01 && e12 && e23;
    const int pnext = __shfl_down_sync(FULL, p[0], 1);
    const bool cont = lane < 31 && pnext == p[3];
    float x0 = __shfl_down_sync(FULL, v0[0], 1);
    float x1 = __shfl_down_sync(FULL, v1[0], 1);
    float x2 = __shfl_down_sync(FULL, v2[0], 1);
    const bool wnext = __shfl_down_sync(FULL, (int)whole, 1) != 0;
    if (!cont) { x0 = 0.0f; x1 = 0.0f; x2 = 0.0f; }
    bool chain = cont && wnext;
#pragma unroll 1
    for (int d = 1; __any_sync(FULL, chain); d <<= 1) {
        const float y0 = __shfl_down_sync(FULL, x0, d);
        const float y1 = __shfl_down_sync(FULL, x1, d);
        const float y2 = __shfl_down_sync(FULL, x2, d);
        const bool cn = __shfl_down_sync(FULL, (int)chain, d) != 0;
        if (chain) { x0 += y0; x1 += y1; x2 += y2; }
        chain = chain && cn;
    }
    const int plast = __shfl_up_sync(FULL, p[3], 1);
    // heads: the first sample of each run; a run reaching the lane end adds X
    const bool h0 = lane == 0 || p[0] != plast;
    if (h0 && p[0] >= 0) {
        const float w = whole ? 1.0f : 0.0f;
        atomic_add3(q + p[0], fmaf(w, x0, v0[0]), fmaf(w, x1, v1[0]), fmaf(w, x2, v2[0]));
    }
    if (!e01 && p[1] >= 0) {
        const float w = (e12 && e23) ? 1.0f : 0.0f;
        atomic_add3(q + p[1], fmaf(w, x0, v0[1]), fmaf(w, x1, v1[1]), fmaf(w, x2, v2[1]));
    }
    if (!e12 && p[2] >= 0) {
        const float w = e23 ? 1.0f : 0.0f;
        atomic_add3(q + p[2], fmaf(w, x0, v0[2]), fmaf(w, x1, v1[2]), fmaf(w, x2, v2[2]));
    }
    if (!e23 && p[3] >= 0) atomic_add3(q + p[3], v0[3] + x0, v1[3] + x1, v2[3] + x2);
}

// Loads in flight per thread in the float32 gather (groups of four samples)
// and in the scatter (warp iterations of 128 samples).
constexpr int HALF_GB = 1;
constexpr int HALF_SU = 1;

// float32 gather: each thread fills two complex points (four samples) per
// group, GB groups per iteration.  The pointing of the next iteration is
// requested before the map entries of the current one, so its DRAM latency
// overlaps the L2 latency and arithmetic of this iteration.
template <bool FROM_TOD, int NT>
__device__ __forceinline__ void half_gather_f32(const FilterArgs& a, const Seg& S, C2<float>* s, int M) {
    constexpr int GB = HALF_GB;
    const int ng = M >> 1;
    auto store = [&](int u0, const float (&y)[GB][4]) {
#pragma unroll
        for (int g = 0; g < GB; ++g) {
            const int u = u0 + g * NT;
            if (u < ng) {
                s[sidx(2 * u)] = C2<float>{y[g][0], y[g][1]};
                s[sidx(2 * u + 1)] = C2<float>{y[g][2], y[g][3]};
            }
        }
    };
    if constexpr (FROM_TOD) {
        for (int u0 = threadIdx.x; u0 < ng; u0 += NT * GB) {
            float y[GB][4];
#pragma unroll
            for (int g = 0; g < GB; ++g) {
                const int u = u0 + g * NT;
                load4_tod(a, S, 4 * u, u < ng && 4 * u < S.n_out, y[g]);
            }
            store(u0, y);
        }
    } else {
        const V4<float>* map = reinterpret_cast<const V4<float>*>(a.src) + (int64_t)S.rhs * a.n_pix;
        auto pointing = [&](int u0, int (&p)[GB][4], float (&ps)[GB][4]) {
#pragma unroll
            for (int g = 0; g < GB; ++g) {
                const int u = u0 + g * NT;
                const int i0 = 4 * u;
                load4(a, S.out0 + i0, u < ng && i0 < S.n_out, S.n_out - i0, p[g], ps[g]);
            }
        };
        int p[GB][4];
        float ps[GB][4];
        pointing(threadIdx.x, p, ps);
        for (int u0 = threadIdx.x; u0 < ng; u0 += NT * GB) {
            int pn[GB][4];
            float psn[GB][4];
            pointing(u0 + NT * GB, pn, psn);
            V4<float> m[GB][4];
#pragma unroll
            for (int g = 0; g < GB; ++g)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (p[g][j] >= 0) m[g][j] = ldmap<float>(map + p[g][j]);
            float y[GB][4];
#pragma unroll
            for (int g = 0; g < GB; ++g)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float v = 0.0f;
                    if (p[g][j] >= 0) {
                        float c, sn;
                        weights_from(a, 0, ps[g][j], c, sn);
                        v = m[g][j].x + c * m[g][j].y + sn * m[g][j].z;
                    }
                    y[g][j] = v;
                }
            store(u0, y);
#pragma unroll
            for (int g = 0; g < GB; ++g)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    p[g][j] = pn[g][j];
                    ps[g][j] = psn[g][j];
                }
        }
    }
}

// float64 / double-float gather: four consecutive samples (two complex
// points) per thread, pixel indices as one vector load, the weight and map
// loads of all four issued before the arithmetic.  From a timeline, d_t (or
// d_t - (P x)_t when a residual map is given).
template <typename T, bool FROM_TOD, int NT>
__device__ __forceinline__ void half_gather_t(const FilterArgs& a, const Seg& S, C2<T>* s, int M) {
    const int ng = M >> 1;
    const bool with_map = !FROM_TOD || a.xmap != nullptr;
    const V4<T>* map =
        with_map ? reinterpret_cast<const V4<T>*>(FROM_TOD ? a.xmap : a.src) + (int64_t)S.rhs * a.n_pix : nullptr;
    for (int u = threadIdx.x; u < ng; u += NT) {
        const int i0 = 4 * u;
        const int64_t t0 = S.out0 + i0;
        const bool act = i0 < S.n_out;
        T y[4] = {T(0), T(0), T(0), T(0)};
        if (FROM_TOD) {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (act && j < S.n_out - i0)
                    y[j] = a.tod_is_float
                               ? T(__ldg(reinterpret_cast<const float*>(a.src) + S.rhs * a.n_samples + t0 + j))
                               : T(__ldg(reinterpret_cast<const double*>(a.src) + S.rhs * a.n_samples + t0 + j));
        }
        if (with_map) {
            int p[4];
            load4_pix(a, t0, act, S.n_out - i0, p);
            T c[4], sn[4];
            V4<T> m[4];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (p[j] >= 0) {
                    weights(a, t0 + j, c[j], sn[j]);
                    m[j] = ldmap<T>(map + p[j]);
                }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (p[j] >= 0) {
                    const T px = m[j].x + c[j] * m[j].y + sn[j] * m[j].z;
                    y[j] = FROM_TOD ? y[j] - px : px;
                }
        }
        s[sidx(2 * u)] = C2<T>{y[0], y[1]};
        s[sidx(2 * u + 1)] = C2<T>{y[2], y[3]};
    }
}

// After the conjugate-domain inverse, point m holds conj(z'_m):
// y'_{2m} = Re, y'_{2m+1} = -Im.  Each warp takes 128 consecutive samples per
// step (four per lane); z_t (1, cos 2psi, sin 2psi) is summed over runs of
// equal pixels (warp_run_scatter).  The next step's pointing is requested
// before this step's run sums.
template <int NT>
__device__ __forceinline__ void half_scatter_f32(const FilterArgs& a, const Seg& S, const C2<float>* s, int M) {
    constexpr int NW = NT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    V4<float>* q = reinterpret_cast<V4<float>*>(a.dst) + (int64_t)S.rhs * a.n_pix;
    const int32_t* pix = a.pix + S.out0;
    const float* psi = a.psi + S.out0;
    // steps whose 128 samples all lie inside an aligned block take unchecked vector loads
    const int nfull = (S.out0 & 3) == 0 ? (S.n_out >> 7) : 0;
    int st = warp;
    if (st < nfull) {
        int4 pv;
        float4 fv;
        ld4_pointing(pix + 128 * st + 4 * lane, psi + 128 * st + 4 * lane, pv, fv);
        for (; st < nfull; st += NW) {
            const int sn = min(st + NW, nfull - 1);
            int4 pn;
            float4 fn;
            ld4_pointing(pix + 128 * sn + 4 * lane, psi + 128 * sn + 4 * lane, pn, fn);
            const int m0 = 64 * st + 2 * lane;   // even: points m0, m0 + 1 share a padding group
            const C2<float> e0 = s[sidx(m0)], e1 = s[sidx(m0) + 1];
            const int p[4] = {pv.x, pv.y, pv.z, pv.w};
            const float f[4] = {fv.x, fv.y, fv.z, fv.w};
            const float z[4] = {e0.x, -e0.y, e1.x, -e1.y};
            float v0[4], v1[4], v2[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float nc, ns;
                neg_cs(f[j], nc, ns);
                const float zz = p[j] >= 0 ? z[j] : 0.0f;
                v0[j] = zz;
                v1[j] = -zz * nc;
                v2[j] = -zz * ns;
            }
            warp_run_scatter(p, v0, v1, v2, q);
            pv = pn;
            fv = fn;
        }
    }
    for (; 128 * st < S.n_out; st += NW) {
        const int i0 = 128 * st + 4 * lane;
        const int m0 = min(i0 >> 1, M - 2);
        const C2<float> e0 = s[sidx(m0)], e1 = s[sidx(m0) + 1];
        const float z[4] = {e0.x, -e0.y, e1.x, -e1.y};
        int p[4];
        float v0[4], v1[4], v2[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool ok = i0 + j < S.n_out;
            p[j] = ok ? __ldg(pix + i0 + j) : -1;
            float nc, ns;
            neg_cs(ok ? __ldg(psi + i0 + j) : 0.0f, nc, ns);
            const float zz = p[j] >= 0 ? z[j] : 0.0f;
            v0[j] = zz;
            v1[j] = -zz * nc;
            v2[j] = -zz * ns;
        }
        warp_run_scatter(p, v0, v1, v2, q);
    }
}

// float64 / double-float scatter, four consecutive samples per lane as in
// the float32 one (in-lane run sums, then the warp-segmented reduction).
template <typename T, int NT>
__device__ __forceinline__ void half_scatter_t(const FilterArgs& a, const Seg& S, const C2<T>* s, int M) {
    constexpr int NW = NT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    using Acc = typename AccT<T>::type;
    V4<Acc>* q = reinterpret_cast<V4<Acc>*>(a.dst) + (int64_t)S.rhs * a.n_pix;
    for (int base = warp * 128; base < S.n_out; base += NW * 128) {
        const int i0 = base + 4 * lane;
        const int64_t t0 = S.out0 + i0;
        int p[4];
        load4_pix(a, t0, i0 < S.n_out, S.n_out - i0, p);
        const int m0 = min(i0 >> 1, M - 2);
        const C2<T> e0 = s[sidx(m0)], e1 = s[sidx(m0 + 1)];
        const T z[4] = {e0.x, -e0.y, e1.x, -e1.y};
        T v0[4], v1[4], v2[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            T zz = T(0), c = T(0), sn = T(0);
            if (p[j] >= 0) {
                zz = z[j];
                weights(a, t0 + j, c, sn);
            }
            v0[j] = zz;
            v1[j] = zz * c;
            v2[j] = zz * sn;
        }
        scatter4_vals<T>(p, v0, v1, v2, q);
    }
}

// Last forward pass, paired real-spectrum step and first inverse pass in
// registers.  The last pass (radix R, R consecutive positions per butterfly,
// no twiddles) leaves butterfly c with the frequencies kc + (M/R) q; the
// mirror images M - k of those sit in the partner butterfly c' at outputs
// R - 1 - q (for kc = 0 at outputs (R - q) mod R, in c itself; kc = M/(2R)
// is its own partner too).  The item table lists the pairs {c, c'} by the
// position of c (bit 31: the kc = 0 item).  A thread takes one pair: DFT_R of both,
// the spectrum step of every pair (k, M - k), written conjugated, and the
// first conjugate-domain pass (DFT_R, no twiddles), so the spectrum step
// costs no shared-memory round trip and no barrier of its own.
template <typename T, int M, int NT, int R>
__device__ __forceinline__ void ct_fused_spectrum(C2<T>* s, const uint32_t* __restrict__ items, const void* Hi,
                                                  int64_t cb) {
    constexpr int NB = M / R;
    constexpr int NI = NB / 2 + 1;
    static_assert(NB % 2 == 0 && 16 % R == 0, "fused spectrum pass: butterfly pairs inside padding groups");
#pragma unroll 1
    for (int i = threadIdx.x; i < NI; i += NT) {
        const uint32_t pr = __ldg(items + i);
        const int c = (int)(pr & 0xffffu), c2 = (int)((pr >> 16) & 0x7fffu);
        T aa[R], ab[R], be[R];
#pragma unroll
        for (int q = 0; q < R; ++q) ld_coef(Hi, cb + (int64_t)i * R + q, aa[q], ab[q], be[q]);
        // positions c R .. c R + R - 1 stay inside one 16-point padding group
        const int b0 = sidx(c * R), b1 = sidx(c2 * R);
        C2<T> x[R];
#pragma unroll
        for (int q = 0; q < R; ++q) x[q] = s[b0 + q];
        Dft<T, R>::run(x);
        if (c != c2) {
            C2<T> y[R];
#pragma unroll
            for (int q = 0; q < R; ++q) y[q] = s[b1 + q];
            Dft<T, R>::run(y);
            C2<T> xo[R], yo[R];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const C2<T> A = x[q], B = y[R - 1 - q];
                xo[q] = C2<T>{aa[q] * A.x + be[q] * B.y, -(aa[q] * A.y + be[q] * B.x)};
                yo[R - 1 - q] = C2<T>{ab[q] * B.x + be[q] * A.y, -(ab[q] * B.y + be[q] * A.x)};
            }
            Dft<T, R>::run(xo);
            Dft<T, R>::run(yo);
#pragma unroll
            for (int q = 0; q < R; ++q) {
                s[b0 + q] = xo[q];
                s[b1 + q] = yo[q];
            }
        } else {
            const bool zero = (pr >> 31) != 0u;
            C2<T> xo[R];
#pragma unroll
            for (int q = 0; q < R; ++q) {
                const C2<T> A = x[q], B = zero ? x[(R - q) % R] : x[R - 1 - q];
                xo[q] = C2<T>{aa[q] * A.x + be[q] * B.y, -(aa[q] * A.y + be[q] * B.x)};
            }
            Dft<T, R>::run(xo);
#pragma unroll
            for (int q = 0; q < R; ++q) s[b0 + q] = xo[q];
        }
    }
}

template <typename T> struct HalfMinBlocks { static constexpr int value = 1; };
template <> struct HalfMinBlocks<float> { static constexpr int value = 2; };

template <typename T, bool FROM_TOD, int NT, int MCT>
__global__ void __launch_bounds__(NT, HalfMinBlocks<T>::value) k_filter_half(const FilterArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    C2<T>* s = reinterpret_cast<C2<T>*>(smraw);
    const Seg S = a.segs[blockIdx.x];
    if (!seg_active<T>(a, S)) return;
    const int M = MCT > 0 ? MCT : a.L;
    const C2<T>* tw = reinterpret_cast<const C2<T>*>(a.tw);
    if constexpr (std::is_same<T, float>::value && !FROM_TOD) half_gather_f32_map<NT>(a, S, s, M);
    else if constexpr (std::is_same<T, float>::value) half_gather_f32<FROM_TOD, NT>(a, S, s, M);
    else half_gather_t<T, FROM_TOD, NT>(a, S, s, M);
    __syncthreads();
    if constexpr (MCT > 0) {
        constexpr CtPlan pl = make_ct_plan(MCT, MaxRadix<T>::value);
        constexpr int R = pl.r[pl.np - 1];
        if constexpr ((MCT / R) % 2 == 0 && 16 % R == 0) {
            const C2<T>* tt = reinterpret_cast<const C2<T>*>(a.twp);
            ct_dif<T, MCT, NT, MaxRadix<T>::value, 0, pl.np - 1>(s, tw, tt);
            ct_fused_spectrum<T, MCT, NT, R>(s, a.items, a.Hi, (int64_t)S.band * ((MCT / R) / 2 + 1) * R);
            __syncthreads();
            if constexpr (pl.np >= 2) ct_dit<T, MCT, NT, MaxRadix<T>::value, pl.np - 2>(s, tw, tt);
            if constexpr (std::is_same<T, float>::value) half_scatter_f32<NT>(a, S, s, M);
            else half_scatter_t<T, NT>(a, S, s, M);
            return;
        }
    }
    if constexpr (MCT > 0) ct_dif<T, MCT, NT, MaxRadix<T>::value, 0>(s, tw);
    else fft_dif<T>(s, tw, a.fp);
    // paired real-spectrum filter, written conjugated for the inverse; the
    // table loads of PU pairs are issued together
    constexpr int PU = sizeof(T) == 4 ? 4 : 2;
    const int np = M / 2 + 1;
    const int64_t cb = (int64_t)S.band * np;
    for (int e0 = threadIdx.x; e0 < np; e0 += NT * PU) {
        uint32_t pr[PU];
        T aa[PU], ab[PU], be[PU];
#pragma unroll
        for (int u = 0; u < PU; ++u) {
            const int e = e0 + u * NT;
            if (e < np) {
                pr[u] = __ldg(a.pairs + e);
                ld_coef(a.H, cb + e, aa[u], ab[u], be[u]);
            }
        }
#pragma unroll
        for (int u = 0; u < PU; ++u) {
            if (e0 + u * NT < np) {
                const int pa = (int)(pr[u] & 0xffffu), pb = (int)(pr[u] >> 16);
                const C2<T> A = s[sidx(pa)], B = s[sidx(pb)];
                s[sidx(pa)] = C2<T>{aa[u] * A.x + be[u] * B.y, -(aa[u] * A.y + be[u] * B.x)};
                s[sidx(pb)] = C2<T>{ab[u] * B.x + be[u] * A.y, -(ab[u] * B.y + be[u] * A.x)};
            }
        }
    }
    __syncthreads();
    if constexpr (MCT > 0)
        ct_dit<T, MCT, NT, MaxRadix<T>::value, make_ct_plan(MCT > 0 ? MCT : 64, MaxRadix<T>::value).np - 1>(s, tw);
    else fft_dit_conj<T>(s, tw, a.fp);
    if constexpr (std::is_same<T, float>::value) half_scatter_f32<NT>(a, S, s, M);
    else half_scatter_t<T, NT>(a, S, s, M);
}

// ---------------- direct band variant, float32, four samples per thread ----------------
// For narrow bands the product is gather + scatter bound: each thread owns
// four consecutive outputs in both phases, so the pixel indices and pointing
// weights loaded for the gather stay in registers for the scatter.  The
// gathered y (with its lambda halo) is staged in shared memory for the band.
template <bool FROM_TOD, int GPT, int LMAX>
__global__ void __launch_bounds__(DIRECT_NT) k_filter_direct4(const FilterArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lam = a.lam;   // <= LMAX
    float* c = reinterpret_cast<float*>(smraw);                    // LMAX + 1 (zero beyond lam), padded to 4
    float* y = c + ((LMAX + 1 + 3) & ~3);                          // [LMAX + 4*NT*GPT + LMAX], aligned to 16 B
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        const Seg S = a.segs[2 * blockIdx.x + half];
        if (!seg_active<float>(a, S)) continue;   // uniform across the CTA
        const float* band = reinterpret_cast<const float*>(a.band) + (int64_t)S.band * (lam + 1);
        for (int k = threadIdx.x; k <= LMAX; k += blockDim.x) c[k] = k <= lam ? band[k] : 0.0f;
        V4<float>* q = reinterpret_cast<V4<float>*>(a.dst) + (int64_t)S.rhs * a.n_pix;
        const V4<float>* xm = reinterpret_cast<const V4<float>*>(a.src) + (int64_t)S.rhs * a.n_pix;
        int p[GPT][4];
        float cw[GPT][4], sw[GPT][4], yv[GPT][4];
        // outputs of this thread: groups g = threadIdx.x + k * NT, samples out0 + 4g .. +3
#pragma unroll
        for (int k = 0; k < GPT; ++k) {
            const int i0 = 4 * (threadIdx.x + k * DIRECT_NT);
            float ps[4];
            load4(a, S.out0 + i0, i0 < S.n_out, S.n_out - i0, p[k], ps);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                cw[k][j] = 0.0f;
                sw[k][j] = 0.0f;
                yv[k][j] = 0.0f;
                if (p[k][j] >= 0) weights_from(a, S.out0 + i0 + j, ps[j], cw[k][j], sw[k][j]);
            }
        }
#pragma unroll
        for (int k = 0; k < GPT; ++k) {
            const int i0 = 4 * (threadIdx.x + k * DIRECT_NT);
            if (FROM_TOD) {
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (i0 + j < S.n_out)
                        yv[k][j] = a.tod_is_float
                                       ? __ldg(reinterpret_cast<const float*>(a.src) + S.rhs * a.n_samples + S.out0 + i0 + j)
                                       : (float)__ldg(reinterpret_cast<const double*>(a.src) + S.rhs * a.n_samples + S.out0 + i0 + j);
            } else {
                V4<float> m[4];
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (p[k][j] >= 0) m[j] = ldmap<float>(xm + p[k][j]);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (p[k][j] >= 0) yv[k][j] = m[j].x + cw[k][j] * m[j].y + sw[k][j] * m[j].z;
            }
        }
        if constexpr (LMAX > 0) {
            // stage y with its halo, then each thread slides over a register window
#pragma unroll
            for (int k = 0; k < GPT; ++k) {
                const int i0 = 4 * (threadIdx.x + k * DIRECT_NT);
                *reinterpret_cast<float4*>(y + LMAX + i0) = make_float4(yv[k][0], yv[k][1], yv[k][2], yv[k][3]);
            }
            __syncthreads();   // the right halo overlaps the stores of tile positions past the segment end
            for (int h = threadIdx.x; h < 2 * LMAX; h += blockDim.x) {
                // left halo y[0 .. LMAX), right halo after the segment's outputs
                const int i = h < LMAX ? h : LMAX + S.n_out + (h - LMAX);
                const int64_t t = S.out0 - LMAX + i;
                y[i] = (t >= S.lo && t < S.hi && (h < LMAX ? LMAX - h <= lam : h - LMAX < lam))
                           ? sample_value<float, FROM_TOD>(a, t, S.rhs) : 0.0f;
            }
            // outputs inside the tile but past the segment end read zeros
            for (int i = S.n_out + threadIdx.x; i < 4 * DIRECT_NT * GPT; i += blockDim.x)
                if (i >= S.n_out + LMAX) y[LMAX + i] = 0.0f;
            __syncthreads();
            float cr[LMAX + 1];
#pragma unroll
            for (int kk = 0; kk <= LMAX; ++kk) cr[kk] = c[kk];
#pragma unroll
            for (int k = 0; k < GPT; ++k) {
                const int i0 = 4 * (threadIdx.x + k * DIRECT_NT);
                float w[4 + 2 * LMAX];
#pragma unroll
                for (int e = 0; e < (4 + 2 * LMAX) / 4; ++e) {
                    const float4 v = *reinterpret_cast<const float4*>(y + i0 + 4 * e);
                    w[4 * e] = v.x;
                    w[4 * e + 1] = v.y;
                    w[4 * e + 2] = v.z;
                    w[4 * e + 3] = v.w;
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float z = cr[0] * w[LMAX + j];
#pragma unroll
                    for (int kk = 1; kk <= LMAX; ++kk) z += cr[kk] * (w[LMAX + j - kk] + w[LMAX + j + kk]);
                    yv[k][j] = z;
                }
            }
        } else {
            __syncthreads();
            const float c0 = c[0];
#pragma unroll
            for (int k = 0; k < GPT; ++k)
#pragma unroll
                for (int j = 0; j < 4; ++j) yv[k][j] *= c0;
        }
#pragma unroll
        for (int k = 0; k < GPT; ++k) {
            float v0[4], v1[4], v2[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float z = p[k][j] >= 0 ? yv[k][j] : 0.0f;
                v0[j] = z;
                v1[j] = z * cw[k][j];
                v2[j] = z * sw[k][j];
            }
            scatter4_vals(p[k], v0, v1, v2, q);
        }
        __syncthreads();
    }
}

// ---------------- direct band variant ----------------
template <typename T, bool FROM_TOD>
__global__ void __launch_bounds__(DIRECT_NT) k_filter_direct(const FilterArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lam = a.lam;
    T* c = reinterpret_cast<T*>(smraw);
    T* y = c + ((lam + 1 + 1) & ~1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        const Seg S = a.segs[2 * blockIdx.x + half];
        if (!seg_active<T>(a, S)) continue;   // uniform across the CTA
        const T* band = reinterpret_cast<const T*>(a.band) + (int64_t)S.band * (lam + 1);
        for (int k = threadIdx.x; k <= lam; k += blockDim.x) c[k] = ldval(band + k);
        const int nin = S.n_out + 2 * lam;
        for (int i = threadIdx.x; i < nin; i += blockDim.x) {
            const int64_t t = S.out0 - lam + i;
            y[i] = (t >= S.lo && t < S.hi) ? sample_value<T, FROM_TOD>(a, t, S.rhs) : T(0);
        }
        __syncthreads();
        for (int base = warp * 32; base < S.n_out; base += nwarp * 32) {
            const int i = base + lane;
            T z = T(0);
            if (i < S.n_out) {
                const T* yc = y + lam + i;
                z = c[0] * yc[0];
                for (int k = 1; k <= lam; ++k) z += c[k] * (yc[-k] + yc[k]);
            }
            scatter_one<T>(a, S, true, i, z);
        }
        __syncthreads();
    }
}


// Dynamic shared memory of a filter kernel, and a carveout (percent of the
// 228 KB per SM) just large enough for the CTAs that registers, threads and
// shared memory let reside together (1 KB reserved per CTA); the rest of the
// 256 KB stays L1 for the map entries, twiddles and tables.
template <typename K>
inline void configure_smem(K kern, size_t sm, int nt) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, kern);
    const int warps = (nt + 31) / 32;
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    int ctas = (int)((228u * 1024u) / (sm + 1024));
    ctas = std::min(ctas, 2048 / nt);
    if (regs_warp > 0) ctas = std::min(ctas, 65536 / (regs_warp * warps));
    ctas = std::max(ctas, 1);
    const double need = (double)ctas * (double)(sm + 1024);
    int pct = (int)std::ceil(100.0 * need / (228.0 * 1024.0));
    pct = pct < 1 ? 1 : (pct > 100 ? 100 : pct);
    cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
}

template <typename T, bool FROM_TOD, int NT, int LCT>
inline void launch_fft_nt(const FilterArgs& a, size_t sm, cudaStream_t s) {
    static std::atomic<size_t> configured{0};
    raise_smem_once(configured, sm, [](size_t v) { configure_smem(k_filter_fft<T, FROM_TOD, NT, LCT>, v, NT); });
    k_filter_fft<T, FROM_TOD, NT, LCT><<<a.n_work, NT, sm, s>>>(a);
    count_launches(1);
}

// 512 threads when one CTA fills an SM's shared memory (large float32
// transforms), 256 otherwise; compile-time transforms for the common lengths.
template <typename T, bool FROM_TOD>
inline void launch_fft_t(const FilterArgs& a, cudaStream_t s) {
    if (a.n_work <= 0) return;
    const size_t sm = fft_smem_bytes(a.L, sizeof(T) == 8);
    if constexpr (sizeof(T) == 4 && !FROM_TOD) {
        switch (a.L) {
            case 18432: return launch_fft_nt<T, FROM_TOD, 512, 18432>(a, sm, s);
            case 16384: return launch_fft_nt<T, FROM_TOD, 512, 16384>(a, sm, s);
            case 12288: return launch_fft_nt<T, FROM_TOD, 512, 12288>(a, sm, s);
            case 9216: return launch_fft_nt<T, FROM_TOD, 256, 9216>(a, sm, s);
            case 8192: return launch_fft_nt<T, FROM_TOD, 256, 8192>(a, sm, s);
            case 4608: return launch_fft_nt<T, FROM_TOD, 256, 4608>(a, sm, s);
            case 4096: return launch_fft_nt<T, FROM_TOD, 256, 4096>(a, sm, s);
            case 2048: return launch_fft_nt<T, FROM_TOD, 256, 2048>(a, sm, s);
            default: break;
        }
    }
    if constexpr (std::is_same<T, df>::value) {   // double-float: 512 threads, radix <= 8
        switch (a.L) {
            case 12288: return launch_fft_nt<T, FROM_TOD, 512, 12288>(a, sm, s);
            case 9216: return launch_fft_nt<T, FROM_TOD, 512, 9216>(a, sm, s);
            case 8192: return launch_fft_nt<T, FROM_TOD, 512, 8192>(a, sm, s);
            case 4608: return launch_fft_nt<T, FROM_TOD, 512, 4608>(a, sm, s);
            default: break;
        }
        return launch_fft_nt<T, FROM_TOD, 512, 0>(a, sm, s);
    } else if constexpr (sizeof(T) == 8) {
        switch (a.L) {
            case 12288: return launch_fft_nt<T, FROM_TOD, 256, 12288>(a, sm, s);
            case 9216: return launch_fft_nt<T, FROM_TOD, 256, 9216>(a, sm, s);
            case 8192: return launch_fft_nt<T, FROM_TOD, 256, 8192>(a, sm, s);
            case 4608: return launch_fft_nt<T, FROM_TOD, 256, 4608>(a, sm, s);
            default: break;
        }
    }
    if constexpr (sizeof(T) == 4) {
        if (sm > 110 * 1024) return launch_fft_nt<T, FROM_TOD, 512, 0>(a, sm, s);
    }
    launch_fft_nt<T, FROM_TOD, 256, 0>(a, sm, s);
}
template <typename T, bool FROM_TOD, int NT, int MCT>
inline void launch_half_nt(const FilterArgs& a, size_t sm, cudaStream_t s) {
    static std::atomic<size_t> configured{0};
    raise_smem_once(configured, sm, [](size_t v) { configure_smem(k_filter_half<T, FROM_TOD, NT, MCT>, v, NT); });
    k_filter_half<T, FROM_TOD, NT, MCT><<<a.n_work, NT, sm, s>>>(a);
    count_launches(1);
}

// Half-length real transforms (a.L = M complex points): float32 with two
// CTAs per SM (512 threads for the large transforms, 256 otherwise);
// double-float with 512 threads; float64 with 256.  Compile-time transforms
// for the common block shapes.
template <typename T, bool FROM_TOD>
inline void launch_half_t(const FilterArgs& a, cudaStream_t s) {
    if (a.n_work <= 0) return;
    const size_t sm = fft_smem_bytes(a.L, sizeof(T) == 8);
    if constexpr (std::is_same<T, float>::value) {
        if constexpr (!FROM_TOD) {
            switch (a.L) {
                case 9216: return launch_half_nt<T, FROM_TOD, 512, 9216>(a, sm, s);
                case 8192: return launch_half_nt<T, FROM_TOD, 512, 8192>(a, sm, s);
                case 4608: return launch_half_nt<T, FROM_TOD, 256, 4608>(a, sm, s);
                case 2304: return launch_half_nt<T, FROM_TOD, 256, 2304>(a, sm, s);
                default: break;
            }
        } else {
            if (a.L == 9216) return launch_half_nt<T, FROM_TOD, 512, 9216>(a, sm, s);
        }
        return launch_half_nt<T, FROM_TOD, 256, 0>(a, sm, s);
    } else if constexpr (std::is_same<T, df>::value) {
        if (a.L == 9216) return launch_half_nt<T, FROM_TOD, 512, 9216>(a, sm, s);
        if (a.L == 12288) return launch_half_nt<T, FROM_TOD, 512, 12288>(a, sm, s);
        return launch_half_nt<T, FROM_TOD, 512, 0>(a, sm, s);
    } else {
        if (a.L == 9216) return launch_half_nt<T, FROM_TOD, 256, 9216>(a, sm, s);
        return launch_half_nt<T, FROM_TOD, 256, 0>(a, sm, s);
    }
}

template <typename T, bool FROM_TOD>
inline void launch_direct_t(const FilterArgs& a, cudaStream_t s) {
    if (a.n_work <= 0) return;
    if constexpr (std::is_same<T, float>::value) {
        // lean kernel: tile = 4 * DIRECT_NT * GPT outputs, bands up to 16 taps each side
        if ((a.V == 4 * DIRECT_NT * 2 || a.V == 4 * DIRECT_NT) && a.lam <= 16) {
            const int gpt = a.V / (4 * DIRECT_NT);
            const int lmax = a.lam == 0 ? 0 : (a.lam <= 4 ? 4 : (a.lam <= 8 ? 8 : 16));
            const size_t sm = (size_t)(((lmax + 1 + 3) & ~3) + a.V + 2 * lmax + 4) * sizeof(float);
            auto go = [&](auto kern) {
                kern<<<a.n_work, DIRECT_NT, sm, s>>>(a);
                count_launches(1);
            };
            if (gpt == 2) {
                if (lmax == 0) go(k_filter_direct4<FROM_TOD, 2, 0>);
                else if (lmax == 4) go(k_filter_direct4<FROM_TOD, 2, 4>);
                else if (lmax == 8) go(k_filter_direct4<FROM_TOD, 2, 8>);
                else go(k_filter_direct4<FROM_TOD, 2, 16>);
            } else {
                if (lmax == 0) go(k_filter_direct4<FROM_TOD, 1, 0>);
                else if (lmax == 4) go(k_filter_direct4<FROM_TOD, 1, 4>);
                else if (lmax == 8) go(k_filter_direct4<FROM_TOD, 1, 8>);
                else go(k_filter_direct4<FROM_TOD, 1, 16>);
            }
            return;
        }
    }
    const size_t sm = direct_smem_bytes(a.V, a.lam, sizeof(T) == 8);
    static std::atomic<size_t> configured{0};
    raise_smem_once(configured, sm, [](size_t v) {
        cudaFuncSetAttribute(k_filter_direct<T, FROM_TOD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v);
    });
    k_filter_direct<T, FROM_TOD><<<a.n_work, DIRECT_NT, sm, s>>>(a);
    count_launches(1);
}


}  // namespace mm
