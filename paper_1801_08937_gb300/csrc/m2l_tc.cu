// The dense coarse products of the two-level preconditioner (Sect. 3.2,
// Eq. m2l), M_2l R = M_BD (R - AZ U) + Z U with U = E^-1 Z^T R, for a batch of
// right-hand sides R on the tensor cores (tcgen05, Blackwell), in three
// launches:
//
//   1. T = Z^T R, a reduction over the 4 n_pix map entries: the CTAs split
//      the map (split-K), each accumulates D[rhs][c] = sum R[rhs][n] Z[c][n]
//      over its share in TMEM (M = 128 right-hand-side rows, N = k) and
//      writes it out in float64;
//   2. one CTA per right-hand side adds the partials in CTA order (float64)
//      and solves U = E^-1 T (float64);
//   3. a persistent kernel forms Z U and AZ U for 128 map entries at a time
//      (M = 128 map entries, N = the right-hand sides, K = k, two accumulators
//      in TMEM) and finishes M_BD (R - AZ U) + Z U per pixel from TMEM on the
//      CUDA cores, with the fused inner product r^T z of the PCG step; Z U and
//      AZ U never reach memory.  R and Z are read twice (U depends on all of
//      the map), AZ and the output once.  The epilogue works in float32 (the
//      products it combines carry about 21 bits): the GB300's float64 pipe
//      runs about two FMAs per clock per SM, so a float64 epilogue would take
//      longer than the loads; r^T z sums a warp's 32 float32 products in
//      float32 and everything beyond in float64.
//
// Operands are TF32 (kind::tf32, float32 accumulation).  Each float64 value x
// is truncated to float32 (integer bit operations: the hardware conversions
// run on the slow float64 pipe of the GB300) and split by masking into a TF32
// high part and the TF32-truncated remainder; x y is formed as hi hi + hi lo +
// lo hi (three MMAs into the same accumulator), about 21 bits, so M_2l x
// agrees with the float64 CUDA-core kernels to a few 1e-7 (checked in the
// tests).  One elected thread issues the MMAs; operands are staged in
// shared memory by all threads in the canonical K-major layout without
// swizzle (8-row x 16-byte core matrices: LBO 128 B between core matrices
// along K, SBO between 8-row groups); tcgen05.commit signals an mbarrier.
// Every wait on it is bounded in time; a wait that gives up records the
// failure in g_tc_fault (the host reads it as MM_ERR_TIMEOUT), releases the
// TMEM the CTA holds and ends the kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"
#include "fconv.cuh"

namespace mm {

constexpr int TC_KT = 32;        // K elements per stage of the Z^T R product
constexpr int TC_MAX_RHS = 128;
constexpr int TC_MAX_K = 64;
constexpr unsigned long long TC_WAIT_NS = 1000000000ull;   // 1 s: no stage takes this long

static __device__ int g_tc_fault = 0;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long tc_now() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void tc_mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool tc_mbar_try(uint32_t a, unsigned parity) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(a), "r"(parity)
                 : "memory");
    return done != 0;
}
// true once the phase with `parity` has completed; false after TC_WAIT_NS (the timer is read only
// when the first try finds the phase still open)
__device__ __forceinline__ bool tc_mbar_wait(uint64_t* bar, unsigned parity) {
    const uint32_t a = saddr(bar);
    if (tc_mbar_try(a, parity)) return true;
    const unsigned long long t0 = tc_now();
    for (;;) {
        if (tc_mbar_try(a, parity)) return true;
        if (tc_now() - t0 > TC_WAIT_NS) return false;
    }
}

// TMEM: allocated by warp 0, address written to shared memory
__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// shared-memory stores of this thread become visible to the tensor cores
__device__ __forceinline__ void tc_fence_proxy() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Shared-memory matrix descriptor: start address, leading (K-direction) and
// stride (8-row direction) byte offsets, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}
// Instruction descriptor of kind::tf32: float32 D, TF32 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                 "l"(a), "l"(b), "r"(idesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}
// eight consecutive float32 columns of this thread's TMEM lane
__device__ __forceinline__ void tc_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// x (float64) as a TF32 high part (the float32 value with its 13 low
// significand bits cleared) and the exact float32 remainder, truncated to TF32
// the same way: hi + lo holds about 22 significant bits of x.
__device__ __forceinline__ void tf32_split(double xd, uint32_t& hi, uint32_t& lo) {
    const float x = d2f_trunc(xd);
    hi = __float_as_uint(x) & 0xFFFFE000u;
    lo = __float_as_uint(x - __uint_as_float(hi)) & 0xFFFFE000u;
}
// Byte offset of the 16-byte group kc (elements 4 kc .. 4 kc + 3) of row r in
// a K-major tile without swizzle whose 8-row groups are sbo bytes apart.
__device__ __forceinline__ uint32_t tc_off(int r, int kc, uint32_t sbo) {
    return (uint32_t)(r >> 3) * sbo + (uint32_t)kc * 128u + (uint32_t)(r & 7) * 16u;
}
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__host__ __device__ constexpr uint32_t tc_cols(int n) {   // TMEM columns: a power of two, at least 32
    return n <= 32 ? 32u : (n <= 64 ? 64u : (n <= 128 ? 128u : (n <= 256 ? 256u : 512u)));
}

// Half a stage (TC_SEG elements from kb, zero from k1 on) of a float64 row
// into registers (rows start at multiples of 4 n_pix doubles and kb at
// multiples of TC_SEG, so the segment is 16-byte aligned), and from registers
// into row r, 16-byte groups kc0 .. kc0 + TC_SEG / 4 - 1, of the TF32 high and
// low tiles.
constexpr int TC_SEG = TC_KT / 2;
__device__ __forceinline__ void load_seg(const double* row, int64_t kb, int64_t k1, double (&v)[TC_SEG]) {
    if (kb + TC_SEG <= k1) {
        const double2* p = reinterpret_cast<const double2*>(row + kb);
#pragma unroll
        for (int j = 0; j < TC_SEG / 2; ++j) {
            const double2 d = __ldg(p + j);
            v[2 * j] = d.x;
            v[2 * j + 1] = d.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < TC_SEG; ++j) v[j] = kb + j < k1 ? __ldg(row + kb + j) : 0.0;
    }
}
__device__ __forceinline__ void store_seg(const double (&v)[TC_SEG], int r, int kc0, uint32_t hi_tile,
                                          uint32_t lo_tile, uint32_t sbo) {
#pragma unroll
    for (int kc = 0; kc < TC_SEG / 4; ++kc) {
        uint32_t h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) tf32_split(v[4 * kc + j], h[j], l[j]);
        const uint32_t o = tc_off(r, kc0 + kc, sbo);
        st_shared_v4(hi_tile + o, h[0], h[1], h[2], h[3]);
        st_shared_v4(lo_tile + o, l[0], l[1], l[2], l[3]);
    }
}

// ---- 1. T = Z^T R (split-K) ----
// Dynamic shared memory: two stages of [A_hi, A_lo (128 x TC_KT), B_hi, B_lo
// (np x TC_KT)] TF32, then two mbarriers and the TMEM address.  Eight warps:
// all stage operands, warps 0-3 read the accumulator (TMEM lanes 0-127).
constexpr int TC_ZT = 256;
__global__ void __launch_bounds__(TC_ZT, 2) k_m2l_tc_ztr(const PcgArgs a, const V4<double>* r, int kchunk) {
    extern __shared__ __align__(128) unsigned char sm[];
    const int nrhs = a.nrhs, k = a.k;
    const int np = (k + 15) & ~15;
    const int64_t n4 = (int64_t)a.n_pix * 4;
    const double* R = reinterpret_cast<const double*>(r);
    const double* Z = reinterpret_cast<const double*>(a.Z);
    constexpr uint32_t a_bytes = 128 * TC_KT * 4, sbo = TC_KT / 4 * 128;
    const uint32_t b_bytes = (uint32_t)np * TC_KT * 4;
    const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * stage_bytes);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bars + 2);
    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t ncols = tc_cols(np);
    if (tid == 0) {
        tc_mbar_init(bars, 1);
        tc_mbar_init(bars + 1, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) tc_alloc(slot, ncols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const int64_t k0 = (int64_t)blockIdx.x * kchunk;
    const int64_t k1 = k0 + kchunk < n4 ? k0 + kchunk : n4;
    const int nst = (int)((k1 - k0 + TC_KT - 1) / TC_KT);
    const uint32_t idesc = tc_idesc(128, np);
    const uint32_t base = saddr(sm);
    bool ok = true;
    // Staged rows: the nrhs rows of R (A operand) then the k rows of Z (B operand), each as two
    // half-stage items (item = 2 row + half); thread t takes item t and, when there are more than
    // TC_ZT items, item t + TC_ZT.  Item t's next stage is loaded into registers while the current
    // one is converted and multiplied.
    const int n_items = 2 * (nrhs + k);
    auto item_src = [&](int it) {
        const int r = it >> 1;
        return (r < nrhs ? R + (int64_t)r * n4 : Z + (int64_t)(r - nrhs) * n4) + (it & 1) * TC_SEG;
    };
    auto item_store = [&](const double (&v)[TC_SEG], int it, uint32_t sa) {
        const int r = it >> 1, kc0 = (it & 1) * (TC_SEG / 4);
        if (r < nrhs) store_seg(v, r, kc0, sa, sa + a_bytes, sbo);
        else store_seg(v, r - nrhs, kc0, sa + 2 * a_bytes, sa + 2 * a_bytes + b_bytes, sbo);
    };
    auto item_k1 = [&](int it) { return k1 - (it & 1) * TC_SEG; };   // the row's end, shifted like its start
    const bool has1 = tid < n_items, has2 = tid + TC_ZT < n_items;
    double pre[TC_SEG];
    if (has1 && nst > 0) load_seg(item_src(tid), k0, item_k1(tid), pre);
    for (int st = 0; st < nst && ok; ++st) {
        const int b = st & 1;
        if (st >= 2) ok = tc_mbar_wait(bars + b, ((st - 2) >> 1) & 1);   // MMAs of stage st - 2 read this buffer
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        const uint32_t sa = base + b * stage_bytes;
        const int64_t kb = k0 + (int64_t)st * TC_KT;
        if (has1) item_store(pre, tid, sa);
        if (has2) {
            double v2[TC_SEG];
            load_seg(item_src(tid + TC_ZT), kb, item_k1(tid + TC_ZT), v2);
            item_store(v2, tid + TC_ZT, sa);
        }
        if (has1 && st + 1 < nst) load_seg(item_src(tid), kb + TC_KT, item_k1(tid), pre);
        tc_fence_proxy();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int ks = 0; ks < TC_KT / 8; ++ks) {
                const uint32_t off = ks * 256;   // 8 K elements = two core matrices along K
                const uint64_t ah = tc_desc(sa + off, 128, sbo), al = tc_desc(sa + a_bytes + off, 128, sbo);
                const uint64_t bh = tc_desc(sa + 2 * a_bytes + off, 128, sbo);
                const uint64_t bl = tc_desc(sa + 2 * a_bytes + b_bytes + off, 128, sbo);
                tc_mma(tmem, ah, bh, idesc, (st > 0 || ks > 0) ? 1u : 0u);
                tc_mma(tmem, ah, bl, idesc, 1u);
                tc_mma(tmem, al, bh, idesc, 1u);
            }
            tc_commit(bars + b);
        }
    }
    // the last commit completes after every earlier MMA of this CTA
    if (ok && nst > 0) ok = tc_mbar_wait(bars + ((nst - 1) & 1), ((nst - 1) >> 1) & 1);
    ok = __syncthreads_and(ok);
    tc_fence_after();
    if (ok && warp < 4) {
        // every lane of the warp executes each (warp-collective) TMEM load; only the stores are predicated
        const uint32_t lane_addr = tmem + ((uint32_t)(warp * 32) << 16);
        double* part = a.partial + ((int64_t)blockIdx.x * nrhs + tid) * k;
        for (int c0 = 0; c0 < np; c0 += 8) {
            float v[8];
            tc_ld8(lane_addr + c0, v);
            if (tid < nrhs) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    if (c0 + j < k) part[c0 + j] = (double)v[j];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, ncols);
    if (!ok && tid == 0) atomicOr(&g_tc_fault, 1);
}

// ---- 1b. T = the split-K partials summed in CTA order (float64), U = E^-1 T ----
// One CTA per right-hand side; thread (h, c) sums half h of the partials of
// coarse index c, the halves are added in order.
constexpr int TC_UT = 2 * TC_MAX_K;
__global__ void __launch_bounds__(TC_UT) k_m2l_tc_u(const PcgArgs a, const double* partial, int g) {
    __shared__ double t2[2][TC_MAX_K];
    const int rhs = blockIdx.x, k = a.k, tid = threadIdx.x;
    const int c = tid % TC_MAX_K, h = tid / TC_MAX_K;
    if (c < k) {
        const int g0 = h ? (g + 1) / 2 : 0, g1 = h ? g : (g + 1) / 2;
        const int64_t stride = (int64_t)a.nrhs * k;
        const double* p = partial + (int64_t)rhs * k + c;
        double s = 0.0;
        int j = g0;
        for (; j + 8 <= g1; j += 8) {
            double v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcg(p + (int64_t)(j + u) * stride);
#pragma unroll
            for (int u = 0; u < 8; ++u) s += v[u];
        }
        for (; j < g1; ++j) s += __ldcg(p + (int64_t)j * stride);
        t2[h][c] = s;
    }
    __syncthreads();
    if (tid < k) {
        const double* Einv = a.Einv + (int64_t)rhs * a.einv_stride + (int64_t)tid * k;
        double s = 0.0;
        for (int j = 0; j < k; ++j) s += Einv[j] * (t2[0][j] + t2[1][j]);
        a.u[(int64_t)rhs * k + tid] = s;
    }
}

// ---- 2. out = M_BD (v - AZ U) + Z U, 128 map entries (32 pixels) per tile ----
// Persistent: each CTA stages U (B operand: row = right-hand side, K = coarse
// index) once, then for each of its tiles stages Z and AZ (A operands: row =
// map entry, K = coarse index), forms D_z = Z U and D_az = AZ U in TMEM
// (columns [0, nr) and [nr, 2 nr)), and finishes on the CUDA cores: warp w
// reads TMEM lanes 32 (w % 4) .. + 31 (32 map entries = 8 pixels) for the
// 8-column chunks w / 4, w / 4 + 4, ... of the right-hand sides (sixteen warps
// also share the staging: thread t stages row t % 128 of the tile for a
// quarter of the coarse vectors), exchanges the residual's Stokes entries of a
// pixel within a quad of lanes, applies the pixel's 3x3 block of M_BD and adds
// Z U.  r^T z per right-hand side (when finalize_beta >= 0) is summed per warp
// and tile in a fixed order, then over CTAs in CTA order by the last CTA.
// Dynamic shared memory: B_hi, B_lo (nr x kp), A tiles Z_hi, Z_lo, AZ_hi,
// AZ_lo (128 x kp), r^T z sums [4][nr], one mbarrier, the TMEM address.
constexpr int TC_AT = 512;              // four groups of four warps
constexpr int TC_AG = TC_AT / 128;
__global__ void __launch_bounds__(TC_AT, 1) k_m2l_tc_zu_apply(const PcgArgs a, const V4<double>* v, V4<double>* out,
                                                              int finalize_beta, double* partial, int n_tiles) {
    extern __shared__ __align__(128) unsigned char sm[];
    const int nrhs = a.nrhs, k = a.k;
    const int nr = (nrhs + 15) & ~15, kp = (k + 7) & ~7;
    const int64_t n4 = (int64_t)a.n_pix * 4;
    const uint32_t sbo = (uint32_t)kp / 4 * 128;
    const uint32_t b_bytes = (uint32_t)nr * kp * 4, a_bytes = 128u * kp * 4;
    double* racc = reinterpret_cast<double*>(sm + 2 * b_bytes + 4 * a_bytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(racc + 4 * nr);
    uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, q = warp & 3, grp = warp >> 2;
    const uint32_t ncols = tc_cols(2 * nr);
    const double* Z = reinterpret_cast<const double*>(a.Z);
    const double* AZ = reinterpret_cast<const double*>(a.AZ);
    const double* V = reinterpret_cast<const double*>(v);
    double* O = reinterpret_cast<double*>(out);
    if (tid == 0) {
        tc_mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (warp == 0) tc_alloc(slot, ncols);
    const uint32_t base = saddr(sm);
    const int kq = kp / 4;   // 16-byte groups of four coarse indices per row
    for (int e = tid; e < nr * kq; e += TC_AT) {
        const int n = e / kq, kc = e - n * kq;
        uint32_t h[4], l[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int c = 4 * kc + j;
            tf32_split(n < nrhs && c < k ? a.u[(int64_t)n * k + c] : 0.0, h[j], l[j]);
        }
        const uint32_t o = tc_off(n, kc, sbo);
        st_shared_v4(base + o, h[0], h[1], h[2], h[3]);
        st_shared_v4(base + b_bytes + o, l[0], l[1], l[2], l[3]);
    }
    for (int e = tid; e < 4 * nr; e += TC_AT) racc[e] = 0.0;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    const uint32_t at = base + 2 * b_bytes;
    const uint32_t idesc = tc_idesc(128, nr);
    // staging: thread tid loads row (tid % 128) of the tile; the kp / 8 blocks of eight coarse
    // vectors are split between the TC_AG groups of 128 threads (tid / 128)
    const int row = tid & 127, n_oct = kp / 8, per_grp = (n_oct + TC_AG - 1) / TC_AG;
    const int oct_begin = (tid >> 7) * per_grp, oct_end = min(n_oct, oct_begin + per_grp);
    // epilogue: this thread's TMEM lane is tile row q * 32 + lane; its columns are the 8-column chunks
    // grp, grp + TC_AG, ... of the nr right-hand-side columns
    const int comp = lane & 3;
    const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
    // this thread's row of a tile, for at most TC_MAX_K / 16 blocks of eight coarse vectors
    constexpr int MAX_OCT = (TC_MAX_K / 8 + TC_AG - 1) / TC_AG;
    double zv[MAX_OCT][8], av[MAX_OCT][8];
    auto load_tile = [&](int tile) {
        const int64_t i = (int64_t)tile * 128 + row;
        const bool rin = i < n4;
#pragma unroll
        for (int o = 0; o < MAX_OCT; ++o) {
            const int oct = oct_begin + o;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int c = 8 * oct + j;
                const bool in = rin && oct < oct_end && c < k;
                zv[o][j] = in ? __ldg(Z + (int64_t)c * n4 + i) : 0.0;
                av[o][j] = in ? __ldg(AZ + (int64_t)c * n4 + i) : 0.0;
            }
        }
    };
    auto store_tile = [&]() {
#pragma unroll
        for (int o = 0; o < MAX_OCT; ++o) {
            if (oct_begin + o >= oct_end) continue;
            const int kc = 2 * (oct_begin + o);
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                uint32_t zh[4], zl[4], ah[4], al[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    tf32_split(zv[o][4 * g + j], zh[j], zl[j]);
                    tf32_split(av[o][4 * g + j], ah[j], al[j]);
                }
                const uint32_t off = tc_off(row, kc + g, sbo);
                st_shared_v4(at + off, zh[0], zh[1], zh[2], zh[3]);
                st_shared_v4(at + a_bytes + off, zl[0], zl[1], zl[2], zl[3]);
                st_shared_v4(at + 2 * a_bytes + off, ah[0], ah[1], ah[2], ah[3]);
                st_shared_v4(at + 3 * a_bytes + off, al[0], al[1], al[2], al[3]);
            }
        }
    };
    bool ok = true;
    int it = 0;
    load_tile(blockIdx.x);
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
        const int64_t i0 = (int64_t)tile * 128;
        store_tile();   // the previous tile's MMAs have completed and its TMEM has been read
        tc_fence_proxy();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            for (int ks = 0; ks < kp / 8; ++ks) {
                const uint32_t off = ks * 256;
                const uint64_t bh = tc_desc(base + off, 128, sbo), bl = tc_desc(base + b_bytes + off, 128, sbo);
                const uint64_t zh = tc_desc(at + off, 128, sbo), zl = tc_desc(at + a_bytes + off, 128, sbo);
                const uint64_t ah = tc_desc(at + 2 * a_bytes + off, 128, sbo);
                const uint64_t al = tc_desc(at + 3 * a_bytes + off, 128, sbo);
                const uint32_t first = ks > 0 ? 1u : 0u;
                tc_mma(tmem, zh, bh, idesc, first);
                tc_mma(tmem, zh, bl, idesc, 1u);
                tc_mma(tmem, zl, bh, idesc, 1u);
                tc_mma(tmem + nr, ah, bh, idesc, first);
                tc_mma(tmem + nr, ah, bl, idesc, 1u);
                tc_mma(tmem + nr, al, bh, idesc, 1u);
            }
            tc_commit(bar);
        }
        if (tile + (int)gridDim.x < n_tiles) load_tile(tile + gridDim.x);   // in flight during the MMAs and epilogue
        ok = tc_mbar_wait(bar, it & 1);
        ok = __syncthreads_and(ok);
        tc_fence_after();
        if (!ok) break;
        const int64_t i = i0 + q * 32 + lane;
        const bool in = i < n4;
        const int64_t pix = i >> 2;
        // row comp of the pixel's symmetric block [m0 m1 m2; m1 m3 m4; m2 m4 m5]
        const int r0 = comp == 0 ? 0 : (comp == 1 ? 1 : 2), r1 = comp == 0 ? 1 : (comp == 1 ? 3 : 4),
                  r2 = comp == 0 ? 2 : (comp == 1 ? 4 : 5);
        float b0 = 0.0f, b1 = 0.0f, b2 = 0.0f;
        if (in && comp < 3 && !a.bd_per_rhs) {
            const double* m = a.bd + pix * 6;
            b0 = (float)m[r0];
            b1 = (float)m[r1];
            b2 = (float)m[r2];
        }
        for (int n0 = grp * 8; n0 < nr; n0 += 8 * TC_AG) {
            // the chunk's eight inputs are requested together, before the TMEM reads
            double xs[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) xs[j] = in && n0 + j < nrhs ? __ldg(V + (int64_t)(n0 + j) * n4 + i) : 0.0;
            float dz[8], daz[8];
            tc_ld8(lane_addr + n0, dz);
            tc_ld8(lane_addr + nr + n0, daz);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int n = n0 + j;   // the same in every lane of the warp
                if (n >= nrhs) break;
                const bool active = !a.st || a.st[n].active;
                const float x = d2f_trunc(xs[j]);
                const float y = x - daz[j];
                const int qb = lane & ~3;
                const float y0 = __shfl_sync(0xffffffffu, y, qb), y1 = __shfl_sync(0xffffffffu, y, qb + 1),
                            y2 = __shfl_sync(0xffffffffu, y, qb + 2);
                float m0 = b0, m1 = b1, m2 = b2;
                if (a.bd_per_rhs && in && comp < 3) {
                    const double* m = a.bd + ((int64_t)n * a.n_pix + pix) * 6;
                    m0 = (float)m[r0];
                    m1 = (float)m[r1];
                    m2 = (float)m[r2];
                }
                const float o = comp < 3 ? fmaf(m0, y0, fmaf(m1, y1, fmaf(m2, y2, dz[j]))) : 0.0f;
                if (in && active) O[(int64_t)n * n4 + i] = f2d_exact(o);
                if (finalize_beta >= 0) {
                    // the warp's 32 products summed in float32, the warps' sums in float64
                    float d = x * o;
#pragma unroll
                    for (int s = 16; s > 0; s >>= 1) d += __shfl_down_sync(0xffffffffu, d, s);
                    if (lane == 0) racc[q * nr + n] += (double)d;
                }
            }
        }
        tc_fence_before();
        __syncthreads();   // TMEM and the A tiles are free for the next tile
        tc_fence_after();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tc_dealloc(tmem, ncols);
    if (!ok && tid == 0) atomicOr(&g_tc_fault, 2);
    if (finalize_beta < 0) return;
    // every CTA takes its ticket, so the counter is reset even after a failed wait
    if (tid < nrhs)
        partial[(int64_t)blockIdx.x * nrhs + tid] =
            racc[tid] + racc[nr + tid] + racc[2 * nr + tid] + racc[3 * nr + tid];
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(a.counter, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (tid < nrhs) {
        double rz = 0.0;
        int g = 0;
        for (; g + 8 <= (int)gridDim.x; g += 8) {
            double w[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) w[u] = __ldcg(partial + (int64_t)(g + u) * nrhs + tid);
#pragma unroll
            for (int u = 0; u < 8; ++u) rz += w[u];
        }
        for (; g < (int)gridDim.x; ++g) rz += __ldcg(partial + (int64_t)g * nrhs + tid);
        if (a.st[tid].active) {
            RhsState& st = a.st[tid];
            st.beta = finalize_beta ? rz / st.rz : 0.0;
            st.rz = rz;
        }
    }
    if (tid == 0) a.counter[0] = 0;
}

bool m2l_tc_eligible(const PcgArgs& a) {
    return a.nrhs >= 8 && a.nrhs <= TC_MAX_RHS && a.k >= 1 && a.k <= TC_MAX_K && a.az_stride == 0;
}
// Below this map size the three launches of the tensor-core path cost more than the two float64
// CUDA-core kernels save (measured: a 32x32 patch, 64 right-hand sides, k = 32).
bool m2l_tc_pays(const PcgArgs& a) { return a.n_pix >= 16384; }

// Grids: split-K CTAs of the Z^T R product (two per SM fit), persistent CTAs of the fused
// product (one per SM).
static int tc_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}
static int tc_g1(int n_pix, int sms) {
    const int64_t stages = ((int64_t)n_pix * 4 + TC_KT - 1) / TC_KT;
    return (int)std::max<int64_t>(1, std::min<int64_t>(2 * sms, stages));
}
static int tc_g2(int n_pix, int sms) {
    const int64_t tiles = ((int64_t)n_pix * 4 + 127) / 128;
    return (int)std::max<int64_t>(1, std::min<int64_t>(sms, tiles));
}

// Scratch of launch_m2l_tc: the split-K partials of Z^T R, then the r^T z partials.
size_t m2l_tc_scratch_doubles(int n_pix, int nrhs, int k) {
    const int sms = tc_sms();
    return (size_t)tc_g1(n_pix, sms) * nrhs * std::max(k, 1) + (size_t)tc_g2(n_pix, sms) * nrhs;
}

// M_2l v -> out on the tensor cores (see the top of this file); scratch holds
// m2l_tc_scratch_doubles(n_pix, nrhs, k) doubles.
void launch_m2l_tc(const PcgArgs& a, const V4<double>* v, V4<double>* out, int finalize_beta, double* scratch,
                   cudaStream_t s) {
    const int k = a.k, nrhs = a.nrhs;
    const int np = (k + 15) & ~15, nr = (nrhs + 15) & ~15, kp = (k + 7) & ~7;
    const int64_t n4 = (int64_t)a.n_pix * 4;
    const int sms = tc_sms();
    // 1. split-K over g1 CTAs, whole stages each
    const int64_t stages = (n4 + TC_KT - 1) / TC_KT;
    const int g1 = tc_g1(a.n_pix, sms);
    const int kchunk = (int)(((stages + g1 - 1) / g1) * TC_KT);
    const int g_used = (int)((n4 + kchunk - 1) / kchunk);
    const int g2 = tc_g2(a.n_pix, sms);
    const int n_tiles = (int)((n4 + 127) / 128);
    const size_t sm1 = 2 * (2 * 128 * TC_KT * 4 + 2 * (size_t)np * TC_KT * 4) + 32;
    const size_t sm2 = 2 * (size_t)nr * kp * 4 + 4 * (size_t)128 * kp * 4 + 4 * (size_t)nr * 8 + 32;
    static std::atomic<size_t> conf1{0}, conf2{0};
    raise_smem_once(conf1, sm1, [](size_t v) {
        cudaFuncSetAttribute(k_m2l_tc_ztr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v);
    });
    raise_smem_once(conf2, sm2, [](size_t v) {
        cudaFuncSetAttribute(k_m2l_tc_zu_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v);
    });
    PcgArgs a1 = a;
    a1.partial = scratch;
    k_m2l_tc_ztr<<<g_used, TC_ZT, sm1, s>>>(a1, v, kchunk);
    k_m2l_tc_u<<<nrhs, TC_UT, 0, s>>>(a, scratch, g_used);
    k_m2l_tc_zu_apply<<<g2, TC_AT, sm2, s>>>(a, v, out, finalize_beta, scratch + (size_t)g1 * nrhs * std::max(k, 1),
                                             n_tiles);
    count_launches(3);
}

// Failures recorded by the tensor-core kernels since the last call (0: none);
// clears the record.  Synchronises stream s.
cudaError_t m2l_tc_fault_take(cudaStream_t s, int* fault) {
    *fault = 0;
    cudaError_t e = cudaMemcpyFromSymbolAsync(fault, g_tc_fault, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && *fault) {
        const int zero = 0;
        e = cudaMemcpyToSymbolAsync(g_tc_fault, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    return e;
}

}  // namespace mm
