// C ABI entry points (include/mapmaker.h): context, pointing set-up, M_BD,
// coarse space, A x, preconditioners and the PCG driver.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>
#include <map>
#include <array>

#include <nvtx3/nvToolsExt.h>

#include "../../include/mapmaker.h"
#include "common.cuh"

namespace mm {

// ---------------- device buffers ----------------
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t ensure(size_t n) {
        if (n <= bytes && p) return cudaSuccess;
        release();
        if (n == 0) n = 16;
        cudaError_t e = cudaMalloc(&p, n);
        if (e != cudaSuccess) {
            p = nullptr;
            return e;
        }
        bytes = n;
        return cudaSuccess;
    }
    template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

struct FftTables {
    int L = 0;
    DevBuf tw, H;
    DevBuf pairs;      // half-length real transforms: positions of k and M - k
    DevBuf items, Hi;  // the same coefficients by butterfly pair of the last pass (fused spectrum step)
    DevBuf twp;        // per-pass twiddle powers W_S^(j q) of the compile-time transforms
};

struct Plan {
    FftTables ft;      // twiddles and band spectra for this plan's L
    int variant = 0;   // 1 direct, 2 fft
    int L = 0, logL = 0, V = 0;
    int whole = 0;     // FFT: 1 one transform per whole block (no overlap-save halo), two blocks
                       // per CTA; 2 one block per CTA as an L/2-point complex transform
    FftPasses fp{};
    int f64 = 0;
    int nrhs = 0;
    std::vector<int64_t> lens;
    std::vector<int64_t> starts;   // per right-hand side: samples before it (per detector) are inactive
    DevBuf segs;
    int n_work = 0;
};

enum Phase { PH_IDLE = 0, PH_INNER = 1, PH_DONE = 2 };

}  // namespace mm

using namespace mm;

struct mm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    mm_precision prec = MM_FP64;
    std::string err;

    // options
    int opt_filter = 0, opt_fft_log2 = 0, opt_fft_len = 0, opt_direct_tile = 1024, opt_check_every = 8, opt_graphs = 0;
    int opt_time_filter = 0;
    int opt_autotune = 1;
    int opt_half = 1;              // allow whole blocks as half-length complex transforms
    int opt_harvest = 0;           // Lanczos vectors kept from an M_BD solve (0: off)
    int opt_coarse_prefix = 1;     // uneven-length batches: A_i Z from block-prefix products (0: directly)
    int opt_apply_prec = 0;        // mm_apply_A precision: 0 context, 1 float64, 2 double-float
    double opt_inner_tol = 2e-6;   // floor of the float32-operator PCG tolerance between refinements
    double last_apply_ms = 0.0;
    // CUDA-event pairs around filter launches (when timing is on)
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> fev;
    size_t fev_used = 0;
    bool capturing = false;

    // pointing
    bool have_pointing = false;
    int64_t n_samples = 0, n_t = 0;
    int n_det = 1, n_pix = 0, n_blocks = 0, n_bands = 0, lam = 0;
    std::vector<int64_t> block_off;
    std::vector<int32_t> block_band;
    std::vector<double> band;
    DevBuf d_pix, d_psi, d_cs64, d_block_off, d_block_band, d_band64, d_band32, d_banddf, d_csdf;
    bool have_csdf = false;
    int p64 = 1;   // precision of the float64-accurate products: 1 native, 2 double-float
    std::vector<std::unique_ptr<Plan>> plans;

    // M_BD
    bool have_bd = false;
    DevBuf d_good, d_bd, d_sums, d_dropped;
    DevBuf d_bd_rhs;   // per right-hand side, [nrhs][n_pix][6]

    // coarse space
    int k = 0;
    DevBuf d_Z, d_AZ, d_Einv, d_W, d_h;
    std::vector<double> ritz;

    // workspace
    DevBuf w_a, w_b, w_src, w_q, w_partial, w_counter, w_norms, d_lastb;
    bool have_lastb = false;
    int grid_x = 1;

    // solve state
    int phase = PH_IDLE;
    int nrhs = 0;
    mm_precond precond = MM_PRECOND_BD;
    double tol = 1e-8;
    int max_iter = 0;
    bool use_lens = false;
    std::vector<int64_t> lens;
    const void* tod_dev = nullptr;   // device timeline of the current solve (mixed precision), in s_tod
    DevBuf s_tod, s_b, s_x, s_r, s_z, s_p, s_src, s_q, s_st, s_hist, s_u, s_xtot, s_rtrue, s_q64, s_mask;
    Plan* plan_op = nullptr;
    Plan* plan_64 = nullptr;
    std::vector<RhsState> h_st;
    std::vector<int32_t> tot_iters, refinements, final_status;
    std::vector<double> true_res, rec_res, bnorm;
    int outer = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int graph_iters = 0;
    // Lanczos harvest of the last M_BD solve (right-hand side 0)
    bool harvest_on = false;
    int harvest_count = 0;
    DevBuf d_harv, d_ahist, d_bhist;
    std::vector<double> harv_alpha, harv_beta;
    // per right-hand-side coarse operators for batches of uneven length
    bool coarse_per_rhs = false;
    int64_t coarse_len = 0;          // samples per detector of the operator the basis Z was built from
    int64_t harvest_len = 0;         // samples per detector of the harvested right-hand side
    int opt_coarse_fallback = 1;     // uneven batches: M_BD for right-hand sides of another length
    int opt_tc_coarse = 1;           // M_2l coarse products on the tensor cores: 0 never, 1 large maps, 2 always
    DevBuf w_zu;                     // scratch of the tensor-core M_2l (split-K and r^T z partials)
    DevBuf w_u;                      // U = E^-1 Z^T x of mm_apply_precond
    std::vector<int32_t> precond_used;
    // cross-rank sum of partial products (timeline split across processes)
    mm_reduce_fn reduce_fn = nullptr;
    void* reduce_user = nullptr;
    int reduce_dev = 0;
    bool tuning = false;               // autotuner runs: products are timed, not used
    void* reduce_host = nullptr;       // pinned staging buffer
    size_t reduce_host_bytes = 0;
    DevBuf d_AZr, d_Einvr;
    // template filters (mm_set_templates): F = F_B W^-1 F_G W^-1 F_B
    bool tmpl_on = false;
    int tmpl_order = -1, tmpl_bins = 0, tmpl_qu = 0;
    int64_t tmpl_max_block = 0;
    DevBuf d_tsub, d_tblk, d_tginv, d_taz, d_twb;
    std::vector<int64_t> tmpl_sub;   // host copy of the subscan offsets
    // block-prefix coarse products T[m] = A_(first m blocks of every detector) Z,
    // [(blocks per detector + 1)][k][n_pix][4], for uneven-length batches
    DevBuf d_Tpref;
    bool tpref_valid = false;
    DevBuf d_Z32, d_AZ32;              // float32 copies of Z and AZ for mixed-precision M_2l
    bool z32_valid = false;
    int coarse_rank_min = 0;           // smallest coarse rank a right-hand side of the last uneven batch kept
    // asynchronous stepping
    RhsState* h_st_pinned = nullptr;
    int h_st_pinned_n = 0;
    cudaEvent_t ev_state = nullptr;
    bool launched = false;
};

namespace {

// NVTX range around one phase (entry point, PCG iterations, refinement,
// coarse-space build): visible on a profiler timeline, free when none is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

mm_status fail(mm_ctx* c, mm_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

#define CK(call)                                                                                  \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? MM_ERR_OOM : MM_ERR_CUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                      \
    } while (0)

#define CKL()                                                                                     \
    do {                                                                                          \
        cudaError_t e_ = cudaGetLastError();                                                      \
        if (e_ != cudaSuccess) return fail(ctx, MM_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
    } while (0)

#define TRY(expr)                      \
    do {                               \
        mm_status s_ = (expr);         \
        if (s_ != MM_OK) return s_;    \
    } while (0)

// Sum of a partial product over the ranks that share the problem (see
// mm_set_reduction); nothing without a reduction or while plans are tuned.
mm_status reduce_sum(mm_ctx* ctx, void* dev, int64_t count, int elem) {
    if (!ctx->reduce_fn || ctx->tuning || count <= 0) return MM_OK;
    if (ctx->capturing) return fail(ctx, MM_ERR_STATE, "a cross-rank reduction cannot run inside a graph capture");
    CK(cudaStreamSynchronize(ctx->stream));
    const size_t bytes = (size_t)count * elem;
    int rc = 0;
    if (ctx->reduce_dev) {
        rc = ctx->reduce_fn(dev, count, elem, ctx->reduce_user);
    } else {
        if (ctx->reduce_host_bytes < bytes) {
            if (ctx->reduce_host) cudaFreeHost(ctx->reduce_host);
            ctx->reduce_host = nullptr;
            ctx->reduce_host_bytes = 0;
            CK(cudaMallocHost(&ctx->reduce_host, bytes));
            ctx->reduce_host_bytes = bytes;
        }
        CK(cudaMemcpyAsync(ctx->reduce_host, dev, bytes, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        rc = ctx->reduce_fn(ctx->reduce_host, count, elem, ctx->reduce_user);
        if (rc == 0) {
            CK(cudaMemcpyAsync(dev, ctx->reduce_host, bytes, cudaMemcpyHostToDevice, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
        }
    }
    if (rc != 0) return fail(ctx, MM_ERR_REDUCE, "the cross-rank reduction returned " + std::to_string(rc));
    return MM_OK;
}

bool is_f32(const mm_ctx* c) { return c->prec == MM_FP32_MIXED; }
// Precision of the solver's operator products (PCG, Arnoldi, A Z): float32 in
// MM_FP32_MIXED; in MM_FP64 the float64-accurate kind of "fp64_products"
// (1 native float64, 2 double-float).
int op_prec(const mm_ctx* c) { return is_f32(c) ? 0 : c->p64; }

cudaError_t copy_in(void* dst, const void* src, size_t bytes, int mem, cudaStream_t s) {
    return cudaMemcpyAsync(dst, src, bytes, mem == MM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s);
}

int ilog2(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

int64_t max_block_len(const mm_ctx* c) {
    int64_t m = 0;
    for (int b = 0; b < c->n_blocks; ++b) m = std::max(m, c->block_off[b + 1] - c->block_off[b]);
    return m;
}

// Mixed-radix pass plan for L = 2^a 3^b (b <= 2): a radix-3 or radix-9 pass
// first, then radix 16 while it divides, then one radix 2, 4 or 8 pass
// (radix 8 plans end in 4, 4 instead of 8, 2, so the last pass -- fused with
// the spectrum step -- is never a radix-2 one).  maxr: largest power-of-two
// radix (8 for double-float plans, 16 otherwise), the same rule as the
// kernels' compile-time plans.
bool fft_passes(int L, FftPasses* fp, int maxr = 16) {
    int rest = L, np = 0, span = L;
    fp->L = L;
    auto add = [&](int r) {
        fp->radix[np] = r;
        fp->span[np] = span;
        span /= r;
        rest /= r;
        ++np;
    };
    if (rest % 9 == 0) add(9);
    else if (rest % 3 == 0) add(3);
    while (rest % maxr == 0 && np < 8) add(maxr);
    if (maxr == 8 && rest == 2 && np > 0 && fp->radix[np - 1] == 8 && np < 8) {
        --np;
        span *= 8;
        rest *= 8;
        add(4);
        add(4);
    } else if (rest > 1 && rest < maxr && (rest == 8 || rest == 4 || rest == 2)) {
        add(rest);
    }
    fp->npass = np;
    return rest == 1 && np <= 8;
}

size_t smem_limit_bytes() { return 220 * 1024; }

// FFT length and mode candidates: whole blocks (one block per transform, no
// halo, when L >= n_b + lambda) or overlap-save segments of V = L - 2 lambda
// outputs.  Cost model: transform points x passes plus gathered and
// scattered samples, with a penalty when the grid cannot fill the GPU.
struct FftCand {
    int L, whole;
    double cost;
};

std::vector<FftCand> fft_candidates(const mm_ctx* c, int f64, int forced_log2, int forced_len) {
    const int64_t nb = std::max<int64_t>(1, max_block_len(c));
    const int lam = c->lam;
    std::vector<FftCand> out;
    for (int b3 = 0; b3 <= 2; ++b3) {
        for (int lg = 5; lg <= 15; ++lg) {
            const int L = (1 << lg) * (b3 == 0 ? 1 : (b3 == 1 ? 3 : 9));
            if (L < 64) continue;
            if (forced_log2 > 0 && L != (1 << forced_log2)) continue;
            if (forced_len > 0 && L != forced_len) continue;
            // a whole block as an L/2-point complex transform, one block per CTA
            FftPasses fh;
            if (L >= nb + lam && c->opt_half && L % 4 == 0 && L / 2 <= 65535 &&
                fft_smem_bytes(L / 2, f64 != 0) <= smem_limit_bytes() && fft_passes(L / 2, &fh, f64 == 2 ? 8 : 16)) {
                const size_t smh = fft_smem_bytes(L / 2, f64 != 0);
                const double fit = std::floor(228.0 * 1024 / (double)(smh + 1024));
                const double per_smh = std::max(1.0, std::min(fit, f64 ? 1.0 : 2.0));
                const double ctash = c->n_blocks;
                const double per_ctah = (double)(L / 2) * fh.npass * 44.0 + 2.0 * (double)c->n_samples / ctash * 45.0;
                const double wavesh = std::ceil(ctash / (152.0 * per_smh));
                out.push_back({L, 2, wavesh * per_ctah + 1e-3 * ((double)c->n_blocks * (L / 2) * fh.npass * 44.0)});
            }
            const size_t sm = fft_smem_bytes(L, f64 != 0);
            if (sm > smem_limit_bytes()) continue;
            FftPasses fp;
            if (!fft_passes(L, &fp, f64 == 2 ? 8 : 16)) continue;
            double points = 0, gathered = 0, ctas = 0;
            int whole = 0;
            if (L >= nb + lam) {
                whole = 1;
                points = (double)c->n_blocks * L * 0.5;
                gathered = (double)c->n_samples;
                ctas = c->n_blocks * 0.5;
            } else {
                const int V = L - 2 * lam;
                if (V < 32) continue;
                double segs = 0;
                for (int b = 0; b < c->n_blocks; ++b) {
                    const int64_t n = c->block_off[b + 1] - c->block_off[b];
                    segs += (double)((n + V - 1) / V);
                }
                points = segs * L * 0.5;
                gathered = std::min<double>(segs * L, 2.0 * c->n_samples + segs * 2.0 * lam);
                ctas = segs * 0.5;
            }
            // waves of CTAs times the work of one CTA (transform passes plus its gathers and scatters)
            const double per_sm = std::max(1.0, std::floor(228.0 * 1024 / (double)(sm + 1024)));
            const double slots = 152.0 * per_sm;
            const double per_cta = (double)L * fp.npass * 44.0 + (gathered + (double)c->n_samples) / std::max(1.0, ctas) * 45.0;
            const double waves = std::ceil(std::max(1.0, ctas) / slots);
            double cost = waves * per_cta + 1e-3 * (points * fp.npass * 44.0);
            out.push_back({L, whole, cost});
        }
    }
    std::sort(out.begin(), out.end(), [](const FftCand& a, const FftCand& b) { return a.cost < b.cost; });
    return out;
}

bool choose_fft(const mm_ctx* c, int f64, int forced_log2, int forced_len, int* L_out, int* whole_out) {
    auto cands = fft_candidates(c, f64, forced_log2, forced_len);
    if (cands.empty()) return false;
    *L_out = cands[0].L;
    *whole_out = cands[0].whole;
    return true;
}

mm_status build_fft_tables(mm_ctx* ctx, FftTables& ft, const FftPasses& fp, int f64) {
    const int L = fp.L;
    if (ft.L == L) return MM_OK;
    // twiddles exp(-2 pi i e / L) in float64 on the host
    std::vector<double> tw64(2 * (size_t)L);
    for (int e = 0; e < L; ++e) {
        const double ang = -2.0 * M_PI * (double)e / (double)L;
        tw64[2 * e] = std::cos(ang);
        tw64[2 * e + 1] = std::sin(ang);
    }
    // circular placement of each band: h[i] = c_i, h[L - i] = c_i
    std::vector<double> h((size_t)ctx->n_bands * L, 0.0);
    for (int b = 0; b < ctx->n_bands; ++b) {
        const double* c = &ctx->band[(size_t)b * (ctx->lam + 1)];
        double* hb = &h[(size_t)b * L];
        hb[0] = c[0];
        for (int i = 1; i <= ctx->lam; ++i) {
            hb[i] = c[i];
            hb[L - i] = c[i];
        }
    }
    DevBuf d_tw64, d_h, d_H64, d_work;
    CK(d_tw64.ensure(tw64.size() * 8));
    CK(d_h.ensure(h.size() * 8));
    CK(d_H64.ensure(h.size() * 8));
    CK(d_work.ensure((size_t)ctx->n_bands * (L + (L >> 4)) * 16));
    CK(cudaMemcpyAsync(d_tw64.p, tw64.data(), tw64.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(d_h.p, h.data(), h.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    launch_fft_spectrum(d_h.as<double>(), d_H64.as<double>(), d_work.as<double2>(), d_tw64.as<double2>(),
                        ctx->n_bands, fp, ctx->stream);
    CKL();
    if (f64 == 1) {
        CK(ft.tw.ensure(tw64.size() * 8));
        CK(ft.H.ensure(h.size() * 8));
        CK(cudaMemcpyAsync(ft.tw.p, d_tw64.p, tw64.size() * 8, cudaMemcpyDeviceToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ft.H.p, d_H64.p, h.size() * 8, cudaMemcpyDeviceToDevice, ctx->stream));
    } else if (f64 == 2) {
        // double-float: each value as (hi, lo) float32 pair
        std::vector<double> H64(h.size());
        CK(cudaMemcpyAsync(H64.data(), d_H64.p, h.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        std::vector<float> Hdf(2 * h.size()), twdf(2 * tw64.size());
        auto split = [](double d, float* o) {
            o[0] = (float)d;
            o[1] = (float)(d - (double)o[0]);
        };
        for (size_t i = 0; i < h.size(); ++i) split(H64[i], &Hdf[2 * i]);
        for (size_t i = 0; i < tw64.size(); ++i) split(tw64[i], &twdf[2 * i]);
        CK(ft.tw.ensure(twdf.size() * 4));
        CK(ft.H.ensure(Hdf.size() * 4));
        CK(cudaMemcpyAsync(ft.tw.p, twdf.data(), twdf.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ft.H.p, Hdf.data(), Hdf.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    } else {
        std::vector<double> H64(h.size());
        CK(cudaMemcpyAsync(H64.data(), d_H64.p, h.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        std::vector<float> H32(h.size()), tw32(tw64.size());
        for (size_t i = 0; i < h.size(); ++i) H32[i] = (float)H64[i];
        for (size_t i = 0; i < tw64.size(); ++i) tw32[i] = (float)tw64[i];
        CK(ft.tw.ensure(tw32.size() * 4));
        CK(ft.H.ensure(H32.size() * 4));
        CK(cudaMemcpyAsync(ft.tw.p, tw32.data(), tw32.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(ft.H.p, H32.data(), H32.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    ft.L = L;
    return MM_OK;
}

// Frequency index held at each position after the DIF passes of fp: with
// position p = sum_i d_i (span_i / radix_i), the frequency is
// d_0 + radix_0 (d_1 + radix_1 (d_2 + ...)) (mixed-radix digit reversal).
std::vector<int> dif_frequency(const FftPasses& fp) {
    std::vector<int> k(fp.L);
    for (int p = 0; p < fp.L; ++p) {
        int rem = p, mult = 1, f = 0;
        for (int i = 0; i < fp.npass; ++i) {
            const int sr = fp.span[i] / fp.radix[i];
            const int d = rem / sr;
            rem -= d * sr;
            f += d * mult;
            mult *= fp.radix[i];
        }
        k[p] = f;
    }
    return k;
}

// Tables of a whole-block plan run as an M = N/2 point complex transform:
// twiddles of length M, the pair positions (k, M - k) and, per band, the
// coefficients (alpha_k, alpha_{M-k}, beta_k) of the paired real-spectrum
// filter, from the band's length-N spectrum, with 1/M folded in.
mm_status build_half_tables(mm_ctx* ctx, FftTables& ft, const FftPasses& fpM, int N, int f64) {
    const int M = fpM.L;
    if (ft.L == M && ft.pairs.p) return MM_OK;
    FftPasses fpN;
    if (!fft_passes(N, &fpN, 16)) return fail(ctx, MM_ERR_ARG, "no transform plan for the block spectrum");
    // length-N spectra of the bands (digit-reversed, scaled by 1/N) on the device
    std::vector<double> twN(2 * (size_t)N);
    for (int e = 0; e < N; ++e) {
        const double ang = -2.0 * M_PI * (double)e / (double)N;
        twN[2 * e] = std::cos(ang);
        twN[2 * e + 1] = std::sin(ang);
    }
    std::vector<double> h((size_t)ctx->n_bands * N, 0.0);
    for (int b = 0; b < ctx->n_bands; ++b) {
        const double* c = &ctx->band[(size_t)b * (ctx->lam + 1)];
        double* hb = &h[(size_t)b * N];
        hb[0] = c[0];
        for (int i = 1; i <= ctx->lam; ++i) {
            hb[i] = c[i];
            hb[N - i] = c[i];
        }
    }
    std::vector<double> Hp(h.size());
    {
        DevBuf d_tw, d_h, d_H, d_work;
        CK(d_tw.ensure(twN.size() * 8));
        CK(d_h.ensure(h.size() * 8));
        CK(d_H.ensure(h.size() * 8));
        CK(d_work.ensure((size_t)ctx->n_bands * (N + (N >> 4)) * 16));
        CK(cudaMemcpyAsync(d_tw.p, twN.data(), twN.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
        CK(cudaMemcpyAsync(d_h.p, h.data(), h.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
        launch_fft_spectrum(d_h.as<double>(), d_H.as<double>(), d_work.as<double2>(), d_tw.as<double2>(),
                            ctx->n_bands, fpN, ctx->stream);
        CKL();
        CK(cudaMemcpyAsync(Hp.data(), d_H.p, Hp.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    const std::vector<int> kN = dif_frequency(fpN), kM = dif_frequency(fpM);
    std::vector<int> posM(M);
    for (int p = 0; p < M; ++p) posM[kM[p]] = p;
    const int np = M / 2 + 1;
    // pairs in the order of their first position: neighbouring threads then
    // touch neighbouring points (the frequency order would stride by M/r_0
    // and put a warp's accesses on one bank)
    std::vector<int> order(np);
    for (int k = 0; k < np; ++k) order[k] = k;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return posM[x] < posM[y]; });
    std::vector<uint32_t> pairs(np);
    for (int e = 0; e < np; ++e) {
        const int k = order[e];
        pairs[e] = (uint32_t)posM[k] | ((uint32_t)posM[(M - k) % M] << 16);
    }
    // The last pass of radix R works on butterflies c of R consecutive
    // positions; butterfly c holds the frequencies kc + (M/R) q and its partner
    // c' (frequency digits M/R - kc) holds their mirror images M - k, at output
    // R - 1 - q (kc = 0 and kc = M/(2R) pair with themselves).  One item per
    // pair {c, c'}, kc = 0 .. M/(2R).
    const int R = fpM.radix[fpM.npass - 1];
    const int NB = M / R;
    const bool fused = fpM.span[fpM.npass - 1] == R && NB % 2 == 0 && 16 % R == 0;
    const int ni = fused ? NB / 2 + 1 : 0;
    std::vector<uint32_t> items(std::max(ni, 1), 0u);
    std::vector<int> item_kc;
    if (fused) {
        std::vector<int> bfly(NB, -1);
        for (int c = 0; c < NB; ++c) {
            const int kc = kM[c * R];
            for (int q = 0; q < R; ++q)
                if (kM[c * R + q] != kc + NB * q) return fail(ctx, MM_ERR_STATE, "unexpected digit order of the last pass");
            bfly[kc] = c;
        }
        // items in the order of their first butterfly's position: neighbouring
        // threads then touch neighbouring points (2-way bank conflicts at most),
        // where the frequency order would put a warp on one bank; bit 31 marks
        // the kc = 0 item
        std::vector<int> kcs(ni);
        for (int i = 0; i < ni; ++i) kcs[i] = i;
        std::sort(kcs.begin(), kcs.end(), [&](int x, int y) { return bfly[x] < bfly[y]; });
        for (int i = 0; i < ni; ++i) {
            const int kc = kcs[i];
            items[i] = (uint32_t)bfly[kc] | ((uint32_t)bfly[(NB - kc) % NB] << 16) | (kc == 0 ? 0x80000000u : 0u);
        }
        item_kc.swap(kcs);
    }
    // coefficients in float64: H_k / M = 2 (H_k / N)
    std::vector<double> coef((size_t)ctx->n_bands * np * 3), coefi((size_t)ctx->n_bands * std::max(ni, 1) * R * 3);
    std::vector<double> Hn(N);
    auto pair_coef = [&](int k, double* o) {
        const double h1 = Hn[k], h2 = Hn[M - k];
        const double th = 2.0 * M_PI * (double)k / (double)N;
        const double sn = std::sin(th), cs = std::cos(th);
        o[0] = 0.5 * ((h1 + h2) + (h2 - h1) * sn);
        o[1] = 0.5 * ((h1 + h2) - (h2 - h1) * sn);
        o[2] = -0.5 * (h2 - h1) * cs;
    };
    for (int b = 0; b < ctx->n_bands; ++b) {
        for (int p = 0; p < N; ++p) Hn[kN[p]] = 2.0 * Hp[(size_t)b * N + p];
        for (int e = 0; e < np; ++e) pair_coef(order[e], &coef[((size_t)b * np + e) * 3]);
        for (int i = 0; i < ni; ++i)
            for (int q = 0; q < R; ++q) pair_coef(item_kc[i] + NB * q, &coefi[(((size_t)b * ni + i) * R + q) * 3]);
    }
    std::vector<double> twM(2 * (size_t)M);
    for (int e = 0; e < M; ++e) {
        const double ang = -2.0 * M_PI * (double)e / (double)M;
        twM[2 * e] = std::cos(ang);
        twM[2 * e + 1] = std::sin(ang);
    }
    // device layouts per element type: float64 (a, b, c, 0) as two double2;
    // double-float (hi, lo) pairs as two float4; float32 (a, b, c, 0) as float4
    auto upload = [&](DevBuf& dst, const std::vector<double>& src) -> cudaError_t {
        const size_t n = src.size() / 3;
        if (f64 == 1) {
            std::vector<double> C(n * 4, 0.0);
            for (size_t i = 0; i < n; ++i)
                for (int j = 0; j < 3; ++j) C[4 * i + j] = src[3 * i + j];
            cudaError_t e = dst.ensure(C.size() * 8);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dst.p, C.data(), C.size() * 8, cudaMemcpyHostToDevice, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            return e;
        } else if (f64 == 2) {
            std::vector<float> C(n * 8, 0.0f);
            for (size_t i = 0; i < n; ++i)
                for (int j = 0; j < 3; ++j) {
                    const double d = src[3 * i + j];
                    C[8 * i + 2 * j] = (float)d;
                    C[8 * i + 2 * j + 1] = (float)(d - (double)(float)d);
                }
            cudaError_t e = dst.ensure(C.size() * 4);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dst.p, C.data(), C.size() * 4, cudaMemcpyHostToDevice, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            return e;
        }
        std::vector<float> C(n * 4, 0.0f);
        for (size_t i = 0; i < n; ++i)
            for (int j = 0; j < 3; ++j) C[4 * i + j] = (float)src[3 * i + j];
        cudaError_t e = dst.ensure(C.size() * 4);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst.p, C.data(), C.size() * 4, cudaMemcpyHostToDevice, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        return e;
    };
    CK(upload(ft.H, coef));
    if (fused) CK(upload(ft.Hi, coefi));
    if (f64 == 1) {
        CK(ft.tw.ensure(twM.size() * 8));
        CK(cudaMemcpyAsync(ft.tw.p, twM.data(), twM.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    } else if (f64 == 2) {
        std::vector<float> tw(2 * twM.size());
        for (size_t i = 0; i < twM.size(); ++i) {
            tw[2 * i] = (float)twM[i];
            tw[2 * i + 1] = (float)(twM[i] - (double)(float)twM[i]);
        }
        CK(ft.tw.ensure(tw.size() * 4));
        CK(cudaMemcpyAsync(ft.tw.p, tw.data(), tw.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    } else {
        std::vector<float> tw(twM.size());
        for (size_t i = 0; i < twM.size(); ++i) tw[i] = (float)twM[i];
        CK(ft.tw.ensure(tw.size() * 4));
        CK(cudaMemcpyAsync(ft.tw.p, tw.data(), tw.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    // per-pass twiddle powers: pass p (radix R, span S, Sr = S/R > 1) holds
    // W_S^(j q) at [(q - 1) Sr + j], passes concatenated in order
    {
        std::vector<double> t;
        for (int i = 0; i < fpM.npass; ++i) {
            const int Rp = fpM.radix[i], S = fpM.span[i], Sr = S / Rp;
            for (int q = 1; q < Rp; ++q)
                for (int j = 0; j < Sr; ++j) {
                    const double ang = -2.0 * M_PI * (double)((int64_t)j * q % S) / (double)S;
                    t.push_back(std::cos(ang));
                    t.push_back(std::sin(ang));
                }
        }
        if (t.empty()) t.assign(2, 0.0);
        if (f64 == 1) {
            CK(ft.twp.ensure(t.size() * 8));
            CK(cudaMemcpyAsync(ft.twp.p, t.data(), t.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
        } else {
            const bool dfp = f64 == 2;
            std::vector<float> tf(t.size() * (dfp ? 2 : 1));
            for (size_t i = 0; i < t.size(); ++i) {
                if (dfp) {
                    tf[2 * i] = (float)t[i];
                    tf[2 * i + 1] = (float)(t[i] - (double)(float)t[i]);
                } else {
                    tf[i] = (float)t[i];
                }
            }
            CK(ft.twp.ensure(tf.size() * 4));
            CK(cudaMemcpyAsync(ft.twp.p, tf.data(), tf.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
        }
        CK(cudaStreamSynchronize(ctx->stream));
    }
    if (fused) {
        CK(ft.items.ensure(items.size() * 4));
        CK(cudaMemcpyAsync(ft.items.p, items.data(), items.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(ft.pairs.ensure(pairs.size() * 4));
    CK(cudaMemcpyAsync(ft.pairs.p, pairs.data(), pairs.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ft.L = M;
    return MM_OK;
}

// Segment list: for every block, chunk and right-hand side, pairs of segments
// that share a band (and halo).
// starts (optional, per right-hand side): the first starts[r] samples of every
// detector are inactive; each start must fall on a block boundary (whole
// blocks are skipped), as the block-prefix coarse products use it.
mm_status make_plan(mm_ctx* ctx, int f64, int nrhs, const std::vector<int64_t>& lens, int variant, int L,
                    int whole, int V, Plan** out, const std::vector<int64_t>& starts = {}) {
    FftPasses fp{};
    int logL = 0;
    if (variant == 2) {
        fft_passes(whole == 2 ? L / 2 : L, &fp, f64 == 2 ? 8 : 16);
        logL = ilog2(whole == 2 ? L / 2 : L);
    }
    for (auto& p : ctx->plans)
        if (p->variant == variant && p->L == L && p->V == V && p->whole == whole && p->f64 == f64 &&
            p->nrhs == nrhs && p->lens == lens && p->starts == starts) {
            *out = p.get();
            return MM_OK;
        }
    std::vector<Seg> segs;
    const bool single = (variant == 2 && whole == 2);   // one segment per CTA
    auto push = [&](const Seg& s) {
        if (!single && segs.size() % 2 == 1 && (segs.back().band != s.band || segs.back().shift != s.shift)) {
            Seg e{};
            e.n_out = 0;
            e.band = segs.back().band;
            e.shift = segs.back().shift;
            segs.push_back(e);
        }
        segs.push_back(s);
    };
    for (int b = 0; b < ctx->n_blocks; ++b) {
        const int64_t o0 = ctx->block_off[b], o1 = ctx->block_off[b + 1];
        const int64_t det0 = (o0 / ctx->n_t) * ctx->n_t;
        const int64_t step = whole ? (o1 - o0) : V;
        for (int64_t c0 = o0; c0 < o1; c0 += step) {
            for (int r = 0; r < nrhs; ++r) {
                int64_t hi = o1;
                if (!lens.empty()) hi = std::min(hi, det0 + lens[r]);
                if (c0 >= hi) continue;
                if (!starts.empty() && o0 < det0 + starts[r]) continue;
                Seg s{};
                s.out0 = c0;
                s.lo = o0;
                s.hi = hi;
                s.rhs = r;
                s.n_out = (int32_t)std::min<int64_t>(step, hi - c0);
                s.band = ctx->block_band[b];
                s.shift = whole ? 0 : ctx->lam;
                push(s);
            }
        }
    }
    if (!single && segs.size() % 2 == 1) {
        Seg e{};
        e.band = segs.back().band;
        e.shift = segs.back().shift;
        segs.push_back(e);
    }
    auto p = std::make_unique<Plan>();
    p->variant = variant;
    p->L = L;
    p->logL = logL;
    p->V = V;
    p->whole = whole;
    p->fp = fp;
    p->f64 = f64;
    p->nrhs = nrhs;
    p->lens = lens;
    p->starts = starts;
    p->n_work = (int)(single ? segs.size() : segs.size() / 2);
    CK(p->segs.ensure(std::max<size_t>(1, segs.size()) * sizeof(Seg)));
    if (!segs.empty())
        CK(cudaMemcpyAsync(p->segs.p, segs.data(), segs.size() * sizeof(Seg), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (variant == 2 && whole == 2) TRY(build_half_tables(ctx, p->ft, fp, L, f64));
    else if (variant == 2) TRY(build_fft_tables(ctx, p->ft, fp, f64));
    if (f64 == 2 && !ctx->have_csdf) {
        CK(ctx->d_csdf.ensure((size_t)ctx->n_samples * 16));
        launch_weights_df(ctx->d_cs64.as<double2>(), ctx->d_csdf.as<float4>(), ctx->n_samples, ctx->stream);
        CKL();
        ctx->have_csdf = true;
    }
    ctx->plans.push_back(std::move(p));
    *out = ctx->plans.back().get();
    return MM_OK;
}

mm_status run_filter(mm_ctx* ctx, Plan* plan, bool from_tod, const void* src, void* dst, const RhsState* st,
                     int tod_is_float, const void* xmap = nullptr);

// Process-wide record of tuned choices, keyed by problem shape.
struct TuneKey {
    int f64, lam, n_blocks, nrhs;
    int64_t n_samples, max_block, lens_sum;
    int n_pix;
    bool operator==(const TuneKey& o) const {
        return f64 == o.f64 && lam == o.lam && n_blocks == o.n_blocks && nrhs == o.nrhs && n_samples == o.n_samples &&
               max_block == o.max_block && lens_sum == o.lens_sum && n_pix == o.n_pix;
    }
};
struct TuneVal {
    int variant, L, whole, V;
    double ms;
};
// Optional persistence: when MM_TUNE_CACHE names a file, tuned choices are
// read from it at first use and appended to it as JSON lines.
const char* tune_file() { return std::getenv("MM_TUNE_CACHE"); }

// The plan cache is shared by every context of the process (contexts may be
// set up on several host threads): it is read and extended under this lock.
std::mutex& tune_mutex() {
    static std::mutex m;
    return m;
}

// Callers hold tune_mutex().
std::vector<std::pair<TuneKey, TuneVal>>& tune_cache() {
    static std::vector<std::pair<TuneKey, TuneVal>> c;
    static bool loaded = false;
    if (!loaded) {
        loaded = true;
        if (const char* path = tune_file()) {
            if (FILE* f = std::fopen(path, "r")) {
                char line[512];
                while (std::fgets(line, sizeof line, f)) {
                    TuneKey k{};
                    TuneVal v{};
                    long long ns = 0, mb = 0, ls = 0;
                    if (std::sscanf(line,
                                    "{\"f64\": %d, \"lam\": %d, \"n_blocks\": %d, \"nrhs\": %d, \"n_samples\": %lld, "
                                    "\"max_block\": %lld, \"lens_sum\": %lld, \"n_pix\": %d, \"variant\": %d, \"L\": %d, "
                                    "\"whole\": %d, \"V\": %d, \"ms\": %lf}",
                                    &k.f64, &k.lam, &k.n_blocks, &k.nrhs, &ns, &mb, &ls, &k.n_pix, &v.variant, &v.L,
                                    &v.whole, &v.V, &v.ms) == 13) {
                        k.n_samples = ns;
                        k.max_block = mb;
                        k.lens_sum = ls;
                        c.push_back({k, v});
                    }
                }
                std::fclose(f);
            }
        }
    }
    return c;
}

bool tune_lookup(const TuneKey& k, bool allow_half, TuneVal* v) {
    std::lock_guard<std::mutex> lock(tune_mutex());
    for (auto& kv : tune_cache())
        if (kv.first == k && (allow_half || kv.second.whole != 2)) {
            *v = kv.second;
            return true;
        }
    return false;
}

void tune_record(const TuneKey& k, const TuneVal& v) {
    std::lock_guard<std::mutex> lock(tune_mutex());
    tune_cache().push_back({k, v});
    if (const char* path = tune_file()) {
        if (FILE* f = std::fopen(path, "a")) {
            std::fprintf(f,
                         "{\"f64\": %d, \"lam\": %d, \"n_blocks\": %d, \"nrhs\": %d, \"n_samples\": %lld, "
                         "\"max_block\": %lld, \"lens_sum\": %lld, \"n_pix\": %d, \"variant\": %d, \"L\": %d, "
                         "\"whole\": %d, \"V\": %d, \"ms\": %.6f}\n",
                         k.f64, k.lam, k.n_blocks, k.nrhs, (long long)k.n_samples, (long long)k.max_block,
                         (long long)k.lens_sum, k.n_pix, v.variant, v.L, v.whole, v.V, v.ms);
            std::fclose(f);
        }
    }
}

// Time each candidate plan once (after one warm-up launch) on the current
// pointing and keep the fastest.  Candidates: the six cheapest FFT plans of
// the cost model and, for narrow bands, the direct band at two tile sizes.
mm_status autotune_plan(mm_ctx* ctx, int f64, int nrhs, const std::vector<int64_t>& lens, TuneVal* best) {
    struct Opt { int variant, L, whole, V; };
    std::vector<Opt> opts;
    auto cands = fft_candidates(ctx, f64, 0, 0);
    for (size_t i = 0; i < cands.size() && i < 6; ++i)
        opts.push_back({2, cands[i].L, cands[i].whole, cands[i].whole ? cands[i].L - ctx->lam : cands[i].L - 2 * ctx->lam});
    if (ctx->lam <= 256)
        for (int tile : {1024, 2048})
            if (direct_smem_bytes(tile, ctx->lam, f64 != 0) <= 200 * 1024) opts.push_back({1, 0, 0, tile});
    if (opts.empty()) return fail(ctx, MM_ERR_ARG, "no filter plan fits this band");
    const size_t esz = f64 ? sizeof(V4<double>) : sizeof(V4<float>);   // V4<df> is 32 bytes too
    const size_t nv = (size_t)ctx->n_pix * nrhs;
    DevBuf src, dst;
    CK(src.ensure(nv * esz));
    CK(dst.ensure(nv * esz));
    CK(cudaMemsetAsync(src.p, 0, nv * esz, ctx->stream));
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    best->ms = 1e300;
    const int saved_time = ctx->opt_time_filter;
    ctx->opt_time_filter = 0;
    ctx->tuning = true;
    for (const Opt& o : opts) {
        Plan* p = nullptr;
        TRY(make_plan(ctx, f64, nrhs, lens, o.variant, o.L, o.whole, o.V, &p));
        TRY(run_filter(ctx, p, false, src.p, dst.p, nullptr, 0));
        // best of up to three timed launches (one when a launch is long)
        double ms_best = 1e300;
        for (int rep = 0; rep < 3; ++rep) {
            CK(cudaEventRecord(e0, ctx->stream));
            TRY(run_filter(ctx, p, false, src.p, dst.p, nullptr, 0));
            CK(cudaEventRecord(e1, ctx->stream));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            ms_best = std::min(ms_best, (double)ms);
            if (ms > 2.0) break;
        }
        if (ms_best < best->ms) *best = TuneVal{o.variant, o.L, o.whole, o.V, ms_best};
    }
    ctx->opt_time_filter = saved_time;
    ctx->tuning = false;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return MM_OK;
}

mm_status get_plan(mm_ctx* ctx, int f64, int nrhs, const std::vector<int64_t>& lens, Plan** out,
                   const std::vector<int64_t>& starts = {}) {
    int variant = ctx->opt_filter;
    int L = 0, V = 0, whole = 0;
    if (variant == 0 && ctx->opt_fft_len == 0 && ctx->opt_fft_log2 == 0 && ctx->opt_autotune && !ctx->capturing) {
        // tuned once per precision and geometry on a single right-hand side: the
        // per-CTA work of a plan does not depend on how many right-hand sides share it
        TuneKey key{f64, ctx->lam, ctx->n_blocks, 1, ctx->n_samples, max_block_len(ctx), 0, ctx->n_pix};
        TuneVal hit{};
        if (tune_lookup(key, ctx->opt_half != 0, &hit))
            return make_plan(ctx, f64, nrhs, lens, hit.variant, hit.L, hit.whole, hit.V, out, starts);
        TuneVal best{};
        TRY(autotune_plan(ctx, f64, 1, {}, &best));
        tune_record(key, best);
        return make_plan(ctx, f64, nrhs, lens, best.variant, best.L, best.whole, best.V, out, starts);
    }
    if (variant == 0) variant = (ctx->lam <= 32) ? 1 : 2;
    if (variant == 2) {
        if (!choose_fft(ctx, f64, ctx->opt_fft_log2, ctx->opt_fft_len, &L, &whole)) {
            if (ctx->opt_filter == 2) return fail(ctx, MM_ERR_ARG, "no FFT length fits the band half-width");
            variant = 1;
        } else {
            V = whole ? L - ctx->lam : L - 2 * ctx->lam;
        }
    }
    if (variant == 1) {
        V = std::max(32, ctx->opt_direct_tile);
        L = 0;
        whole = 0;
        const size_t sm = direct_smem_bytes(V, ctx->lam, f64 != 0);
        if (sm > 200 * 1024) return fail(ctx, MM_ERR_ARG, "direct filter tile plus halo exceeds shared memory");
    }
    return make_plan(ctx, f64, nrhs, lens, variant, L, whole, V, out, starts);
}

// dst (V4<T>[nrhs][n_pix], zeroed by the caller) += P^T W (P src | d).
mm_status run_filter(mm_ctx* ctx, Plan* plan, bool from_tod, const void* src, void* dst, const RhsState* st,
                     int tod_is_float, const void* xmap) {
    FilterArgs a{};
    a.xmap = xmap;
    a.segs = plan->segs.as<Seg>();
    a.n_work = plan->n_work;
    a.pix = ctx->d_pix.as<int32_t>();
    a.psi = ctx->d_psi.as<float>();
    a.cs64 = ctx->d_cs64.as<double2>();
    a.src = src;
    a.n_samples = ctx->n_samples;
    a.dst = dst;
    a.n_pix = ctx->n_pix;
    a.lam = ctx->lam;
    a.L = plan->L;
    a.logL = plan->logL;
    a.V = plan->V;
    a.fp = plan->fp;
    a.state = st;
    a.tod_is_float = tod_is_float;
    cudaEvent_t e1 = nullptr;
    if (ctx->opt_time_filter && !ctx->capturing) {
        if (ctx->fev_used == ctx->fev.size()) {
            std::pair<cudaEvent_t, cudaEvent_t> pr;
            CK(cudaEventCreate(&pr.first));
            CK(cudaEventCreate(&pr.second));
            ctx->fev.push_back(pr);
        }
        auto& pr = ctx->fev[ctx->fev_used++];
        CK(cudaEventRecord(pr.first, ctx->stream));
        e1 = pr.second;
    }
    a.csdf = ctx->d_csdf.as<float4>();
    if (ctx->tmpl_on) {
        if (!plan->lens.empty() || !plan->starts.empty())
            return fail(ctx, MM_ERR_ARG, "template filters: right-hand sides of uneven length are not supported");
        TmplArgs t{};
        t.block_off = ctx->d_block_off.as<int64_t>();
        t.n_blocks = ctx->n_blocks;
        t.max_block = ctx->tmpl_max_block;
        t.w_block = ctx->d_twb.as<double>();
        t.sub_off = ctx->d_tsub.as<int64_t>();
        t.blk_sub = ctx->d_tblk.as<int32_t>();
        t.ginv = ctx->d_tginv.as<double>();
        t.order = ctx->tmpl_order;
        t.az = ctx->tmpl_bins > 0 ? ctx->d_taz.as<int32_t>() : nullptr;
        t.n_bins = ctx->tmpl_bins;
        t.stokes = ctx->tmpl_qu;
        launch_filter_tmpl(a, t, plan->nrhs, plan->f64, from_tod, ctx->stream);
    } else if (plan->variant == 2) {
        FftTables& ft = plan->ft;
        a.H = ft.H.p;
        a.tw = ft.tw.p;
        if (plan->whole == 2) {
            a.half = 1;
            a.L = plan->L / 2;
            a.pairs = ft.pairs.as<uint32_t>();
            a.items = ft.items.as<uint32_t>();
            a.Hi = ft.Hi.p;
            a.twp = ft.twp.p;
        }
        if (plan->f64 == 2) launch_filter_fft_df(a, from_tod, ctx->stream);
        else if (plan->f64 == 1) launch_filter_fft_f64(a, from_tod, ctx->stream);
        else launch_filter_fft_f32(a, from_tod, ctx->stream);
    } else {
        a.band = plan->f64 == 2 ? ctx->d_banddf.p : (plan->f64 ? ctx->d_band64.p : ctx->d_band32.p);
        if (plan->f64 == 2) launch_filter_direct_df(a, from_tod, ctx->stream);
        else if (plan->f64 == 1) launch_filter_direct_f64(a, from_tod, ctx->stream);
        else launch_filter_direct_f32(a, from_tod, ctx->stream);
    }
    CKL();
    if (e1) CK(cudaEventRecord(e1, ctx->stream));
    if (ctx->reduce_fn && !ctx->tuning)
        TRY(reduce_sum(ctx, dst, (int64_t)4 * ctx->n_pix * plan->nrhs, plan->f64 ? 8 : 4));
    return MM_OK;
}

mm_status ensure_work(mm_ctx* ctx, int nrhs, int kmax) {
    const size_t nv = (size_t)ctx->n_pix * std::max(1, nrhs);
    CK(ctx->w_a.ensure(nv * sizeof(V4<double>)));
    CK(ctx->w_b.ensure(nv * sizeof(V4<double>)));
    CK(ctx->w_src.ensure(nv * sizeof(V4<double>)));
    CK(ctx->w_q.ensure(nv * sizeof(V4<double>)));
    const size_t per = (size_t)std::max({2, kmax, 1}) * std::max(1, nrhs);
    CK(ctx->w_partial.ensure((size_t)ctx->grid_x * std::max<size_t>(per, 512) * sizeof(double)));
    if (ctx->w_counter.bytes < (size_t)std::max(1, nrhs) * sizeof(unsigned)) {
        CK(ctx->w_counter.ensure((size_t)std::max(1, nrhs) * sizeof(unsigned) + 64));
        CK(cudaMemsetAsync(ctx->w_counter.p, 0, ctx->w_counter.bytes, ctx->stream));
    }
    CK(ctx->w_norms.ensure((size_t)std::max(1, nrhs) * sizeof(double) + 64));
    return MM_OK;
}

// out (V4<double>) = A in (V4<double>) for nrhs vectors, operator precision
// f64 or the context's.
mm_status apply_A_dev(mm_ctx* ctx, int f64, const V4<double>* in, V4<double>* out, int nrhs, const Plan* forced = nullptr) {
    Plan* plan = nullptr;
    if (forced) plan = const_cast<Plan*>(forced);
    else TRY(get_plan(ctx, f64, nrhs, {}, &plan));
    TRY(ensure_work(ctx, nrhs, ctx->k));
    const int64_t nv = (int64_t)ctx->n_pix * nrhs;
    if (f64 == 1) {
        CK(cudaMemsetAsync(out, 0, nv * sizeof(V4<double>), ctx->stream));
        TRY(run_filter(ctx, plan, false, in, out, nullptr, 0));
    } else if (f64 == 2) {
        launch_map_to_df(in, ctx->w_src.p, nv, ctx->stream);
        CK(cudaMemsetAsync(out, 0, nv * sizeof(V4<double>), ctx->stream));
        TRY(run_filter(ctx, plan, false, ctx->w_src.p, out, nullptr, 0));
    } else {
        V4<float>* src = ctx->w_src.as<V4<float>>();
        V4<float>* q = ctx->w_q.as<V4<float>>();
        launch_to_f32(in, src, nv, ctx->stream);
        CK(cudaMemsetAsync(q, 0, nv * sizeof(V4<float>), ctx->stream));
        TRY(run_filter(ctx, plan, false, src, q, nullptr, 0));
        launch_from_f32(q, out, nv, ctx->stream);
        CKL();
    }
    return MM_OK;
}

PcgArgs pcg_args(mm_ctx* ctx) {
    PcgArgs a{};
    a.n_pix = ctx->n_pix;
    a.nrhs = ctx->nrhs;
    a.st = ctx->s_st.as<RhsState>();
    a.x = ctx->s_x.as<V4<double>>();
    a.r = ctx->s_r.as<V4<double>>();
    a.z = ctx->s_z.as<V4<double>>();
    a.p = ctx->s_p.as<V4<double>>();
    if (is_f32(ctx)) {
        a.q32 = ctx->s_q.as<V4<float>>();
        a.src_f32 = 1;
    } else {
        a.q64 = ctx->s_q.as<V4<double>>();
        a.src_f32 = op_prec(ctx) == 2 ? 2 : 0;   // 2: double-float operator input
    }
    a.src = ctx->s_src.p;
    a.qacc = ctx->s_q.p;
    a.bd = ctx->use_lens ? ctx->d_bd_rhs.as<double>() : ctx->d_bd.as<double>();
    a.bd_per_rhs = ctx->use_lens ? 1 : 0;
    a.k = ctx->k;
    a.Z = ctx->d_Z.as<V4<double>>();
    a.AZ = ctx->d_AZ.as<V4<double>>();
    a.Einv = ctx->d_Einv.as<double>();
    a.u = ctx->s_u.as<double>();
    a.partial = ctx->w_partial.as<double>();
    a.counter = ctx->w_counter.as<unsigned>();
    a.hist = ctx->s_hist.as<double>();
    a.hist_stride = ctx->max_iter + 1;
    a.grid_x = ctx->grid_x;
    if (is_f32(ctx) && ctx->z32_valid && !ctx->coarse_per_rhs) {
        a.Z32 = ctx->d_Z32.as<V4<float>>();
        a.AZ32 = ctx->d_AZ32.as<V4<float>>();
    }
    if (ctx->coarse_per_rhs && ctx->precond == MM_PRECOND_2L) {
        a.AZ = ctx->d_AZr.as<V4<double>>();
        a.Einv = ctx->d_Einvr.as<double>();
        a.az_stride = (int64_t)ctx->k * ctx->n_pix;
        a.einv_stride = ctx->k * ctx->k;
    }
    if (ctx->harvest_on) {
        a.ahist = ctx->d_ahist.as<double>();
        a.bhist = ctx->d_bhist.as<double>();
        a.harvest = ctx->d_harv.as<V4<double>>();
        a.harvest_m = ctx->opt_harvest;
    }
    return a;
}

// M_2l v -> out: on the tensor cores for a batch of right-hand sides sharing
// the coarse space (the scratch w_zu must be in place), else on the CUDA cores.
// The coarse products go to the tensor cores when the option asks for it and the batch fits them.
bool tc_wanted(const mm_ctx* ctx, const PcgArgs& a) {
    return ctx->opt_tc_coarse && m2l_tc_eligible(a) && (ctx->opt_tc_coarse == 2 || m2l_tc_pays(a));
}
bool use_tc(const mm_ctx* ctx, const PcgArgs& a) {
    return tc_wanted(ctx, a) && ctx->w_zu.bytes >= m2l_tc_scratch_doubles(a.n_pix, a.nrhs, a.k) * sizeof(double);
}
mm_status ensure_tc_scratch(mm_ctx* ctx, const PcgArgs& a) {
    CK(ctx->w_zu.ensure(m2l_tc_scratch_doubles(a.n_pix, a.nrhs, a.k) * sizeof(double)));
    return MM_OK;
}
void m2l_apply(mm_ctx* ctx, const PcgArgs& a, const V4<double>* v, V4<double>* out, int finalize_beta) {
    if (use_tc(ctx, a)) {
        launch_m2l_tc(a, v, out, finalize_beta, ctx->w_zu.as<double>(), ctx->stream);
    } else {
        launch_m2l_ztr(a, v, ctx->stream);
        launch_m2l_apply(a, v, out, finalize_beta, ctx->stream);
    }
}

// Preconditioner on r -> z with rz (and beta when finalize_beta).
void precond_step(mm_ctx* ctx, const PcgArgs& a, int finalize_beta) {
    if (ctx->precond == MM_PRECOND_2L) {
        m2l_apply(ctx, a, a.r, a.z, finalize_beta);
    } else {
        launch_precond_bd_dot(a, finalize_beta, ctx->stream);
    }
}

mm_status pcg_iteration(mm_ctx* ctx) {
    PcgArgs a = pcg_args(ctx);
    launch_pcg_src(a, 0, ctx->stream);
    TRY(run_filter(ctx, ctx->plan_op, false, ctx->s_src.p, ctx->s_q.p, a.st, 0));
    launch_pcg_pq(a, ctx->stream);
    const int two = ctx->precond == MM_PRECOND_2L;
    launch_pcg_update(a, two, ctx->stream);
    if (two) {
        m2l_apply(ctx, a, a.r, a.z, 1);
    } else if (ctx->harvest_on) {
        launch_harvest(a, ctx->stream);
    }
    CKL();
    return MM_OK;
}

// Start PCG on right-hand sides b (V4<double>), per-RHS tolerances and iteration budgets.
mm_status pcg_start(mm_ctx* ctx, const V4<double>* b, const std::vector<double>& tols, const std::vector<int>& budgets) {
    std::vector<RhsState> st(ctx->nrhs);
    for (int i = 0; i < ctx->nrhs; ++i) {
        st[i] = RhsState{};
        st[i].tol = tols[i];
        st[i].max_iter = budgets[i];
    }
    CK(cudaMemcpyAsync(ctx->s_st.p, st.data(), st.size() * sizeof(RhsState), cudaMemcpyHostToDevice, ctx->stream));
    PcgArgs a = pcg_args(ctx);
    launch_pcg_init(a, b, ctx->stream);
    precond_step(ctx, a, 0);
    if (ctx->harvest_on && ctx->precond == MM_PRECOND_BD) launch_harvest(a, ctx->stream);
    CKL();
    return MM_OK;
}

mm_status tc_fault_check(mm_ctx* ctx) {
    int fault = 0;
    CK(m2l_tc_fault_take(ctx->stream, &fault));
    if (fault)
        return fail(ctx, MM_ERR_TIMEOUT,
                    "tensor-core M_2l: a bounded wait for the tensor cores gave up (code " + std::to_string(fault) + ")");
    return MM_OK;
}

mm_status read_state(mm_ctx* ctx) {
    ctx->h_st.resize(ctx->nrhs);
    CK(cudaMemcpyAsync(ctx->h_st.data(), ctx->s_st.p, ctx->nrhs * sizeof(RhsState), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (ctx->precond == MM_PRECOND_2L) TRY(tc_fault_check(ctx));
    return MM_OK;
}

// float64 residual b - A x per right-hand side (x in s_xtot or s_x), written to
// s_rtrue; norms to host.  With the float32 operator (mixed precision) it is
// formed in one float64-accurate pass from the timeline, P^T W (d - P x), so b
// itself is needed only to float32 accuracy; otherwise as b - A x.
mm_status true_residual(mm_ctx* ctx, const V4<double>* x, std::vector<double>& rr) {
    NvtxRange nvtx_range("true_residual");
    if (is_f32(ctx) && ctx->tod_dev) {
        TRY(ensure_work(ctx, ctx->nrhs, ctx->k));
        const int64_t nv = (int64_t)ctx->n_pix * ctx->nrhs;
        const void* xm = x;
        if (ctx->p64 == 2) {
            launch_map_to_df(x, ctx->w_src.p, nv, ctx->stream);
            xm = ctx->w_src.p;
        }
        CK(cudaMemsetAsync(ctx->s_rtrue.p, 0, nv * sizeof(V4<double>), ctx->stream));
        TRY(run_filter(ctx, ctx->plan_64, true, ctx->tod_dev, ctx->s_rtrue.p, nullptr, 1, xm));
        CK(cudaMemsetAsync(ctx->s_q64.p, 0, nv * sizeof(V4<double>), ctx->stream));
        launch_residual(ctx->s_rtrue.as<V4<double>>(), ctx->s_q64.as<V4<double>>(), nullptr, ctx->w_norms.as<double>(),
                        ctx->n_pix, ctx->nrhs, ctx->w_partial.as<double>(), ctx->w_counter.as<unsigned>(),
                        ctx->grid_x, ctx->stream);
    } else {
        TRY(apply_A_dev(ctx, ctx->p64, x, ctx->s_q64.as<V4<double>>(), ctx->nrhs, ctx->plan_64));
        launch_residual(ctx->s_b.as<V4<double>>(), ctx->s_q64.as<V4<double>>(), ctx->s_rtrue.as<V4<double>>(),
                        ctx->w_norms.as<double>(), ctx->n_pix, ctx->nrhs, ctx->w_partial.as<double>(),
                        ctx->w_counter.as<unsigned>(), ctx->grid_x, ctx->stream);
    }
    CKL();
    rr.resize(ctx->nrhs);
    CK(cudaMemcpyAsync(rr.data(), ctx->w_norms.p, ctx->nrhs * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (auto& v : rr) v = std::sqrt(std::max(0.0, v));
    return MM_OK;
}

void destroy_graph(mm_ctx* ctx) {
    if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
    ctx->graph_exec = nullptr;
    ctx->graph_iters = 0;
}

mm_status bd_for_lens(mm_ctx* ctx) {
    // per right-hand side M_BD over its active samples; pixel selection stays the full-scan one
    const int R = ctx->nrhs;
    std::vector<int64_t> sorted(ctx->lens);
    std::vector<int> order(R);
    for (int i = 0; i < R; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ctx->lens[a] < ctx->lens[b]; });
    for (int i = 0; i < R; ++i) sorted[i] = ctx->lens[order[i]];
    DevBuf d_sorted, sums, bdsorted;
    CK(d_sorted.ensure(R * sizeof(int64_t)));
    CK(cudaMemcpyAsync(d_sorted.p, sorted.data(), R * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
    CK(sums.ensure((size_t)R * ctx->n_pix * 7 * sizeof(double)));
    CK(cudaMemsetAsync(sums.p, 0, sums.bytes, ctx->stream));
    launch_bd_accumulate(ctx->d_pix.as<int32_t>(), ctx->d_psi.as<float>(), ctx->d_block_off.as<int64_t>(),
                         ctx->d_block_band.as<int32_t>(), ctx->d_band64.as<double>(), ctx->lam + 1, ctx->n_blocks, 0,
                         ctx->n_t, d_sorted.as<int64_t>(), R, sums.as<double>(), ctx->n_pix, ctx->stream);
    CK(bdsorted.ensure((size_t)R * ctx->n_pix * 6 * sizeof(double)));
    launch_bd_invert(sums.as<double>(), bdsorted.as<double>(), ctx->d_good.as<uint8_t>(), nullptr, ctx->n_pix, R, 0.0, 0,
                     ctx->stream, ctx->tmpl_on ? ctx->tmpl_qu : 0);
    CKL();
    CK(ctx->d_bd_rhs.ensure((size_t)R * ctx->n_pix * 6 * sizeof(double)));
    const size_t per = (size_t)ctx->n_pix * 6 * sizeof(double);
    for (int i = 0; i < R; ++i)
        CK(cudaMemcpyAsync(ctx->d_bd_rhs.as<char>() + (size_t)order[i] * per, bdsorted.as<char>() + (size_t)i * per, per,
                           cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}

// Orthonormalise the columns of X [kin][n] (kept columns only) into Y, twice (CholQR2).
mm_status orthonormalise(mm_ctx* ctx, DevBuf& X, int kin, int* kout) {
    const int64_t n = (int64_t)ctx->n_pix * 4;
    int kcur = kin;
    for (int pass = 0; pass < 2; ++pass) {
        DevBuf dG;
        CK(dG.ensure((size_t)kcur * kcur * sizeof(double)));
        TRY(ensure_work(ctx, 1, std::max(kcur, ctx->k)));
        CK(ctx->w_partial.ensure((size_t)ctx->grid_x * std::max(kcur, 2) * sizeof(double) + 64));
        launch_gram(X.as<double>(), kcur, X.as<double>(), kcur, n, n, dG.as<double>(), ctx->w_partial.as<double>(),
                    ctx->w_counter.as<unsigned>(), ctx->grid_x, ctx->stream);
        CKL();
        std::vector<double> G((size_t)kcur * kcur);
        CK(cudaMemcpyAsync(G.data(), dG.p, G.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        // Cholesky with column dropping on near-dependence
        std::vector<int> keep;
        std::vector<double> L;
        for (int j = 0; j < kcur; ++j) {
            std::vector<int> trial = keep;
            trial.push_back(j);
            const int t = (int)trial.size();
            std::vector<double> S((size_t)t * t);
            for (int a = 0; a < t; ++a)
                for (int b = 0; b < t; ++b) S[(size_t)a * t + b] = 0.5 * (G[(size_t)trial[a] * kcur + trial[b]] + G[(size_t)trial[b] * kcur + trial[a]]);
            std::vector<double> Sc = S;
            const double dj = G[(size_t)j * kcur + j];
            if (host_cholesky(Sc, t) && Sc[(size_t)(t - 1) * t + (t - 1)] > 1e-7 * std::sqrt(std::max(dj, 1e-300))) {
                keep = trial;
                L = Sc;
            }
        }
        const int kk = (int)keep.size();
        if (kk == 0) return fail(ctx, MM_ERR_SINGULAR, "deflation basis has no independent column");
        // C = L^-T (upper) mapped back to the input columns
        std::vector<double> Lt((size_t)kk * kk), Rinv;
        for (int a = 0; a < kk; ++a)
            for (int b = 0; b < kk; ++b) Lt[(size_t)a * kk + b] = L[(size_t)b * kk + a];
        host_upper_inverse(Lt, kk, Rinv);
        std::vector<double> C((size_t)kcur * kk, 0.0);
        for (int a = 0; a < kk; ++a)
            for (int c = 0; c < kk; ++c) C[(size_t)keep[a] * kk + c] = Rinv[(size_t)a * kk + c];
        DevBuf dC, Y;
        CK(dC.ensure(C.size() * 8));
        CK(cudaMemcpyAsync(dC.p, C.data(), C.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
        CK(Y.ensure((size_t)kk * n * 8));
        launch_combo(X.as<double>(), n, kcur, dC.as<double>(), kk, Y.as<double>(), n, n, ctx->stream);
        CKL();
        CK(cudaStreamSynchronize(ctx->stream));
        std::swap(X.p, Y.p);
        std::swap(X.bytes, Y.bytes);
        kcur = kk;
    }
    *kout = kcur;
    return MM_OK;
}

// Given Z (ctx->d_Z, k columns), form AZ, E = Z^T A Z and E^-1.
mm_status finish_coarse(mm_ctx* ctx) {
    NvtxRange nvtx_range("coarse_AZ_E");
    ctx->tpref_valid = false;
    ctx->z32_valid = false;
    const int k = ctx->k;
    const int64_t n = (int64_t)ctx->n_pix * 4;
    CK(ctx->d_AZ.ensure((size_t)k * n * 8));
    TRY(apply_A_dev(ctx, op_prec(ctx), ctx->d_Z.as<V4<double>>(), ctx->d_AZ.as<V4<double>>(), k));
    DevBuf dG;
    CK(dG.ensure((size_t)k * k * 8));
    CK(ctx->w_partial.ensure((size_t)ctx->grid_x * std::max(k, 2) * sizeof(double) + 64));
    launch_gram(ctx->d_Z.as<double>(), k, ctx->d_AZ.as<double>(), k, n, n, dG.as<double>(), ctx->w_partial.as<double>(),
                ctx->w_counter.as<unsigned>(), ctx->grid_x, ctx->stream);
    CKL();
    std::vector<double> G((size_t)k * k), E((size_t)k * k);
    CK(cudaMemcpyAsync(G.data(), dG.p, G.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) E[(size_t)i * k + j] = 0.5 * (G[(size_t)j * k + i] + G[(size_t)i * k + j]);
    std::vector<double> L = E, Einv;
    if (!host_cholesky(L, k)) {
        ctx->k = 0;
    ctx->tpref_valid = false;
    ctx->z32_valid = false;
        return fail(ctx, MM_ERR_SINGULAR, "coarse operator E = Z^T A Z is not positive definite");
    }
    host_spd_inverse_from_chol(L, k, Einv);
    CK(ctx->d_Einv.ensure(Einv.size() * 8));
    CK(cudaMemcpyAsync(ctx->d_Einv.p, Einv.data(), Einv.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}


// ---- scan fingerprint for exported coarse spaces ----
// A coarse space (Z, A Z, E^-1) is valid only for the operator it was built
// with: the same pointing after pixel selection, weights, block structure,
// filters and operator precision.  The fingerprint is a 64-bit sum, modulo
// 2^64, of splitmix64 hashes of every (position, word) pair, so it is the same
// whatever order the device threads add their terms in.
__host__ __device__ inline uint64_t splitmix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__global__ void k_hash_words(const uint32_t* __restrict__ w, int64_t n, uint64_t salt, unsigned long long* out) {
    uint64_t acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += splitmix64(((uint64_t)w[i] << 32 | (uint64_t)(i & 0xffffffff)) ^ splitmix64(salt + (uint64_t)(i >> 32)));
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, (unsigned long long)acc);
}

uint64_t host_hash_bytes(const void* p, size_t bytes, uint64_t h) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < bytes; ++i) h = (h ^ c[i]) * 0x100000001b3ull;   // FNV-1a
    return h;
}

mm_status scan_fingerprint(mm_ctx* ctx, uint64_t* out) {
    DevBuf acc;
    CK(acc.ensure(8));
    CK(cudaMemsetAsync(acc.p, 0, 8, ctx->stream));
    auto dev_hash = [&](const void* p, int64_t words, uint64_t salt) {
        if (p && words > 0) {
            k_hash_words<<<152 * 4, 256, 0, ctx->stream>>>(static_cast<const uint32_t*>(p), words, salt,
                                                          acc.as<unsigned long long>());
            count_launches(1);
        }
    };
    dev_hash(ctx->d_pix.p, ctx->n_samples, 1);   // after pixel selection: dropped pixels' samples are -1
    dev_hash(ctx->d_psi.p, ctx->n_samples, 2);
    if (ctx->tmpl_on && ctx->tmpl_bins > 0) dev_hash(ctx->d_taz.p, ctx->n_samples, 3);
    CKL();
    uint64_t dh = 0;
    CK(cudaMemcpyAsync(&dh, acc.p, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    uint64_t h = 0xcbf29ce484222325ull;
    const int64_t dims[] = {ctx->n_samples, ctx->n_det, ctx->n_pix, ctx->n_blocks, ctx->n_bands, ctx->lam,
                            op_prec(ctx), ctx->tmpl_on, ctx->tmpl_order, ctx->tmpl_bins, ctx->tmpl_qu};
    h = host_hash_bytes(dims, sizeof(dims), h);
    h = host_hash_bytes(ctx->block_off.data(), ctx->block_off.size() * 8, h);
    h = host_hash_bytes(ctx->block_band.data(), ctx->block_band.size() * 4, h);
    h = host_hash_bytes(ctx->band.data(), ctx->band.size() * 8, h);
    if (ctx->tmpl_on) h = host_hash_bytes(ctx->tmpl_sub.data(), ctx->tmpl_sub.size() * 8, h);
    *out = splitmix64(h ^ dh);
    return MM_OK;
}

// Layout of an exported coarse space: this header, then Z [k][n_pix][3],
// A Z [k][n_pix][3], E^-1 [k][k] and the Ritz values [k], all float64.
struct CoarseFileHeader {
    char magic[8];       // "MMCOARS1"
    int32_t version;     // 1
    int32_t n_pix;
    int32_t k;
    int32_t op_prec;     // precision of the products A Z was formed with
    uint64_t fingerprint;
    int64_t payload_bytes;
};
constexpr char kCoarseMagic[8] = {'M', 'M', 'C', 'O', 'A', 'R', 'S', '1'};
int64_t coarse_payload_bytes(int64_t n_pix, int64_t k) { return (2 * k * n_pix * 3 + k * k + k) * 8; }
}  // namespace

namespace {
// Per right-hand side coarse operators for a batch of uneven lengths: the
// basis Z is shared, AZ_i = A_i Z and E_i = Z^T A_i Z use each right-hand
// side's own A_i (its first rhs_len[i] samples per detector), so that
// M_2l,i A_i Z = Z holds for every i (Sect. 3.2, Eq. ident).
// Block boundaries relative to the detector start when every detector has the
// same ones (then the first L samples of each detector cover the same blocks).
static bool uniform_block_bounds(const mm_ctx* ctx, std::vector<int64_t>* rel) {
    rel->clear();
    if (ctx->n_t <= 0 || ctx->n_samples % ctx->n_t != 0) return false;
    const int64_t n_det = ctx->n_samples / ctx->n_t;
    std::vector<std::vector<int64_t>> per(n_det);
    for (int b = 0; b < ctx->n_blocks; ++b) {
        const int64_t o0 = ctx->block_off[b], d = o0 / ctx->n_t;
        if (d < 0 || d >= n_det || ctx->block_off[b + 1] > (d + 1) * ctx->n_t) return false;
        per[d].push_back(o0 - d * ctx->n_t);
    }
    for (int64_t d = 0; d < n_det; ++d)
        if (per[d] != per[0]) return false;
    *rel = per[0];
    if (rel->empty() || (*rel)[0] != 0) return false;
    rel->push_back(ctx->n_t);
    return true;
}

// A_i Z for right-hand sides of uneven length.  W is block diagonal, so with
// the same block boundaries in every detector A_i Z is the product over the
// blocks that lie wholly inside the first L_i samples, T[m_i] (computed once
// per coarse space: one product per block column, then prefix sums), plus the
// product over the one partly covered block of each detector.  Otherwise the
// products are formed directly for every right-hand side.
mm_status coarse_products_for_lens(mm_ctx* ctx, int f64) {
    const int k = ctx->k, R = ctx->nrhs;
    const int64_t n = (int64_t)ctx->n_pix * 4;
    std::vector<int64_t> rel;
    const bool prefix = ctx->opt_coarse_prefix && uniform_block_bounds(ctx, &rel) &&
                        (double)(rel.size() + 1) * k * n * 8 * 3 <= 6.0e9;   // D, T and a replicated Z
    std::vector<int64_t> lens_rep, starts_rep;
    std::vector<int> full(R, 0);
    for (int r = 0; r < R; ++r) {
        if (prefix)
            while (full[r] + 1 < (int)rel.size() && rel[full[r] + 1] <= ctx->lens[r]) ++full[r];
        for (int c = 0; c < k; ++c) {
            lens_rep.push_back(ctx->lens[r]);
            starts_rep.push_back(prefix ? rel[full[r]] : 0);
        }
    }
    if (prefix && !ctx->tpref_valid) {
        const int nbd = (int)rel.size() - 1;
        std::vector<int64_t> lc, sc;
        for (int m = 0; m < nbd; ++m)
            for (int c = 0; c < k; ++c) {
                lc.push_back(rel[m + 1]);
                sc.push_back(rel[m]);
            }
        DevBuf zcol, D;
        CK(zcol.ensure((size_t)nbd * k * n * 8));
        for (int m = 0; m < nbd; ++m)
            CK(cudaMemcpyAsync(zcol.as<double>() + (size_t)m * k * n, ctx->d_Z.p, (size_t)k * n * 8,
                               cudaMemcpyDeviceToDevice, ctx->stream));
        CK(D.ensure((size_t)nbd * k * n * 8));
        Plan* pcol = nullptr;
        TRY(get_plan(ctx, f64, nbd * k, lc, &pcol, sc));
        TRY(apply_A_dev(ctx, f64, zcol.as<V4<double>>(), D.as<V4<double>>(), nbd * k, pcol));
        // T[0] = 0, T[m + 1] = T[m] + D[m]
        CK(ctx->d_Tpref.ensure((size_t)(nbd + 1) * k * n * 8));
        CK(cudaMemsetAsync(ctx->d_Tpref.p, 0, (size_t)k * n * 8, ctx->stream));
        CK(cudaMemcpyAsync(ctx->d_Tpref.as<double>() + (size_t)k * n, D.p, (size_t)nbd * k * n * 8,
                           cudaMemcpyDeviceToDevice, ctx->stream));
        for (int m = 1; m < nbd; ++m)
            launch_axpy_masked(ctx->d_Tpref.as<double>() + (size_t)(m + 1) * k * n,
                               ctx->d_Tpref.as<double>() + (size_t)m * k * n, (int64_t)k * n, 1, nullptr, ctx->stream);
        CKL();
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->tpref_valid = true;
    }
    DevBuf zrep;
    CK(zrep.ensure((size_t)R * k * n * 8));
    for (int r = 0; r < R; ++r)
        CK(cudaMemcpyAsync(zrep.as<double>() + (size_t)r * k * n, ctx->d_Z.p, (size_t)k * n * 8,
                           cudaMemcpyDeviceToDevice, ctx->stream));
    CK(ctx->d_AZr.ensure((size_t)R * k * n * 8));
    Plan* plan = nullptr;
    TRY(get_plan(ctx, f64, R * k, lens_rep, &plan, prefix ? starts_rep : std::vector<int64_t>{}));
    TRY(apply_A_dev(ctx, f64, zrep.as<V4<double>>(), ctx->d_AZr.as<V4<double>>(), R * k, plan));
    if (prefix) {
        for (int r = 0; r < R; ++r)
            if (full[r] > 0)
                launch_axpy_masked(ctx->d_AZr.as<double>() + (size_t)r * k * n,
                                   ctx->d_Tpref.as<double>() + (size_t)full[r] * k * n, (int64_t)k * n, 1, nullptr,
                                   ctx->stream);
        CKL();
    }
    return MM_OK;
}

mm_status coarse_for_lens(mm_ctx* ctx, const std::vector<uint8_t>& deflate) {
    const int k = ctx->k, R = ctx->nrhs;
    const int64_t n = (int64_t)ctx->n_pix * 4;
    TRY(coarse_products_for_lens(ctx, op_prec(ctx)));
    DevBuf dG;
    CK(dG.ensure((size_t)R * k * k * 8));
    CK(ctx->w_partial.ensure((size_t)ctx->grid_x * std::max(k, 2) * sizeof(double) + 64));
    for (int r = 0; r < R; ++r)
        launch_gram(ctx->d_Z.as<double>(), k, ctx->d_AZr.as<double>() + (size_t)r * k * n, k, n, n,
                    dG.as<double>() + (size_t)r * k * k, ctx->w_partial.as<double>(), ctx->w_counter.as<unsigned>(),
                    ctx->grid_x, ctx->stream);
    CKL();
    std::vector<double> G((size_t)R * k * k), Einv_all((size_t)R * k * k);
    CK(cudaMemcpyAsync(G.data(), dG.p, G.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    // A prefix of the scan may leave part of the map unobserved, and with it directions of span Z
    // on which A_i vanishes: E_i is then only semi-definite.  Its inverse is taken on the columns a
    // pivoted Cholesky keeps (all of them when E_i is well conditioned; otherwise the coarse
    // correction of the basis reduced to what the prefix sees, for which M_2l,i A_i Z_S = Z_S
    // holds).  The cut-off sits above the products' rounding level.
    const double piv_tol = op_prec(ctx) == 0 ? 1e-5 : 1e-10;
    ctx->coarse_rank_min = k;
    for (int r = 0; r < R; ++r) {
        const double* g = &G[(size_t)r * k * k];
        std::vector<double> E((size_t)k * k), Einv;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) E[(size_t)i * k + j] = 0.5 * (g[(size_t)j * k + i] + g[(size_t)i * k + j]);
        if (deflate[r]) {
            // pivoted even when a plain Cholesky would pass: a direction at the rounding level must
            // not decide the preconditioner through the rounding of the float64 atomics
            const int rank = host_pivoted_spd_inverse(E, k, piv_tol, Einv);
            if (rank <= 0) return fail(ctx, MM_ERR_SINGULAR, "a per-RHS coarse operator E_i is not semi-definite");
            ctx->coarse_rank_min = std::min(ctx->coarse_rank_min, rank);
        } else {
            Einv.assign((size_t)k * k, 0.0);   // M_2l,r = M_BD,r
        }
        std::copy(Einv.begin(), Einv.end(), Einv_all.begin() + (size_t)r * k * k);
    }
    CK(ctx->d_Einvr.ensure(Einv_all.size() * 8));
    CK(cudaMemcpyAsync(ctx->d_Einvr.p, Einv_all.data(), Einv_all.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->coarse_per_rhs = true;
    return MM_OK;
}
}  // namespace

namespace mm {
// Read-only view of a context's M_BD and coarse space for other translation units.
bool ctx_coarse_view(mm_ctx* ctx, CoarseView* v) {
    if (!ctx) return false;
    v->device = ctx->device;
    v->stream = ctx->stream;
    v->n_pix = ctx->n_pix;
    v->k = ctx->k;
    v->grid_x = ctx->grid_x;
    v->have_bd = ctx->have_bd;
    v->bd = ctx->d_bd.as<double>();
    v->Z = ctx->d_Z.as<V4<double>>();
    v->AZ = ctx->d_AZ.as<V4<double>>();
    v->Einv = ctx->d_Einv.as<double>();
    return true;
}
void ctx_set_error(mm_ctx* ctx, const std::string& msg) {
    if (ctx) ctx->err = msg;
}
}  // namespace mm

// =====================================================================
extern "C" {

mm_status mm_create(mm_ctx** out, int device, void* cuda_stream, mm_precision prec) {
    if (!out) return MM_ERR_ARG;
    *out = nullptr;
    if (prec != MM_FP64 && prec != MM_FP32_MIXED) return MM_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return MM_ERR_CUDA;
    // the kernels' launch configuration is kept once per process: one device per process
    static std::atomic<int> process_device{-1};
    int expect = -1;
    if (!process_device.compare_exchange_strong(expect, device) && expect != device) return MM_ERR_ARG;
    DeviceScope dev_scope(device);
    if (dev_scope.err != cudaSuccess) return MM_ERR_CUDA;
    mm_ctx* ctx = new mm_ctx();
    ctx->device = device;
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    ctx->prec = prec;
    ctx->p64 = prec == MM_FP32_MIXED ? 2 : 1;
    cudaEventCreate(&ctx->ev0);
    cudaEventCreate(&ctx->ev1);
    *out = ctx;
    return MM_OK;
}

mm_status mm_destroy(mm_ctx* ctx) {
    if (!ctx) return MM_OK;
    DeviceScope dev_scope(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    destroy_graph(ctx);
    for (auto& pr : ctx->fev) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    if (ctx->h_st_pinned) cudaFreeHost(ctx->h_st_pinned);
    if (ctx->reduce_host) cudaFreeHost(ctx->reduce_host);
    if (ctx->ev_state) cudaEventDestroy(ctx->ev_state);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    delete ctx;
    return MM_OK;
}

const char* mm_last_error(const mm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

mm_status mm_setup_pointing(mm_ctx* ctx, int64_t n_samples, int32_t n_det, int32_t n_pix, const int32_t* pix,
                            const float* psi, int32_t n_blocks, const int64_t* block_off, const int32_t* block_band,
                            int32_t n_bands, int32_t half_bw, const double* band, int mem) {
    if (!ctx) return MM_ERR_ARG;
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    if (n_samples <= 0 || n_pix <= 0 || n_blocks <= 0 || n_bands <= 0 || half_bw < 0 || n_det <= 0)
        return fail(ctx, MM_ERR_ARG, "sizes must be positive (half_bw >= 0)");
    if (n_samples % n_det != 0) return fail(ctx, MM_ERR_ARG, "n_samples must be a multiple of n_det");
    if (!pix || !psi || !block_off || !block_band || !band) return fail(ctx, MM_ERR_ARG, "null array");
    if (mem != MM_HOST && mem != MM_DEVICE) return fail(ctx, MM_ERR_ARG, "mem must be MM_HOST or MM_DEVICE");
    const int64_t n_t = n_samples / n_det;
    if (block_off[0] != 0 || block_off[n_blocks] != n_samples)
        return fail(ctx, MM_ERR_ARG, "block_off must start at 0 and end at n_samples");
    for (int b = 0; b < n_blocks; ++b) {
        if (block_off[b + 1] <= block_off[b]) return fail(ctx, MM_ERR_ARG, "block_off must be strictly increasing");
        if (block_off[b] / n_t != (block_off[b + 1] - 1) / n_t)
            return fail(ctx, MM_ERR_ARG, "a block straddles two detector timelines");
        if (block_band[b] < 0 || block_band[b] >= n_bands) return fail(ctx, MM_ERR_ARG, "block_band out of range");
        if (block_off[b + 1] - block_off[b] > (int64_t)INT32_MAX) return fail(ctx, MM_ERR_ARG, "block too long");
    }
    if (n_pix > (1 << 26)) return fail(ctx, MM_ERR_ARG, "n_pix too large");
    for (size_t i = 0; i < (size_t)n_bands * (half_bw + 1); ++i)
        if (!std::isfinite(band[i])) return fail(ctx, MM_ERR_ARG, "band holds a non-finite value");
    {
        // the kernels index the map by pix: its range is checked for host and device arrays (a device
        // array through a bounded host buffer, once per pointing set-up)
        auto in_range = [n_pix](const int32_t* p, int64_t c) {
            int32_t lo = 0, hi = -1;
            for (int64_t i = 0; i < c; ++i) {
                lo = std::min(lo, p[i]);
                hi = std::max(hi, p[i]);
            }
            return lo >= -1 && hi < n_pix;
        };
        if (mem == MM_HOST) {
            if (!in_range(pix, n_samples)) return fail(ctx, MM_ERR_ARG, "pix out of range [-1, n_pix)");
        } else {
            const int64_t chunk = (int64_t)1 << 22;
            std::vector<int32_t> hb((size_t)std::min<int64_t>(chunk, n_samples));
            for (int64_t t0 = 0; t0 < n_samples; t0 += chunk) {
                const int64_t c = std::min<int64_t>(chunk, n_samples - t0);
                CK(cudaMemcpyAsync(hb.data(), pix + t0, (size_t)c * 4, cudaMemcpyDeviceToHost, ctx->stream));
                CK(cudaStreamSynchronize(ctx->stream));
                if (!in_range(hb.data(), c)) return fail(ctx, MM_ERR_ARG, "pix out of range [-1, n_pix)");
            }
        }
    }
    destroy_graph(ctx);
    ctx->have_pointing = ctx->have_bd = false;
    ctx->k = 0;
    ctx->tpref_valid = false;
    ctx->z32_valid = false;
    ctx->have_lastb = false;
    ctx->plans.clear();
    ctx->n_samples = n_samples;
    ctx->n_det = n_det;
    ctx->n_t = n_t;
    ctx->n_pix = n_pix;
    ctx->n_blocks = n_blocks;
    ctx->n_bands = n_bands;
    ctx->lam = half_bw;
    ctx->block_off.assign(block_off, block_off + n_blocks + 1);
    ctx->block_band.assign(block_band, block_band + n_blocks);
    ctx->band.assign(band, band + (size_t)n_bands * (half_bw + 1));
    const int64_t gb = (n_pix + 255) / 256;
    ctx->grid_x = (int)std::min<int64_t>(gb, 304);
    CK(ctx->d_pix.ensure(n_samples * 4));
    CK(ctx->d_psi.ensure(n_samples * 4));
    CK(ctx->d_cs64.ensure(n_samples * 16));
    CK(copy_in(ctx->d_pix.p, pix, n_samples * 4, mem, ctx->stream));
    CK(copy_in(ctx->d_psi.p, psi, n_samples * 4, mem, ctx->stream));
    launch_weights64(ctx->d_psi.as<float>(), ctx->d_cs64.as<double2>(), n_samples, ctx->stream);
    CKL();
    CK(ctx->d_block_off.ensure((n_blocks + 1) * 8));
    CK(ctx->d_block_band.ensure(n_blocks * 4));
    CK(cudaMemcpyAsync(ctx->d_block_off.p, block_off, (n_blocks + 1) * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_block_band.p, block_band, n_blocks * 4, cudaMemcpyHostToDevice, ctx->stream));
    std::vector<float> b32(ctx->band.size());
    for (size_t i = 0; i < b32.size(); ++i) b32[i] = (float)ctx->band[i];
    CK(ctx->d_band64.ensure(ctx->band.size() * 8));
    CK(ctx->d_band32.ensure(b32.size() * 4));
    CK(cudaMemcpyAsync(ctx->d_band64.p, ctx->band.data(), ctx->band.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_band32.p, b32.data(), b32.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    std::vector<float> bdf(2 * ctx->band.size());
    for (size_t i = 0; i < ctx->band.size(); ++i) {
        bdf[2 * i] = (float)ctx->band[i];
        bdf[2 * i + 1] = (float)(ctx->band[i] - (double)bdf[2 * i]);
    }
    CK(ctx->d_banddf.ensure(bdf.size() * 4));
    CK(cudaMemcpyAsync(ctx->d_banddf.p, bdf.data(), bdf.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    ctx->have_csdf = false;
    ctx->tmpl_on = false;
    ctx->tmpl_qu = 0;
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->have_pointing = true;
    return MM_OK;
}

// Template filters of ground-based scans (Sect. 2.1, Eq. filtnoise; Sect. 4;
// Sect. 5.1): subscan polynomials and azimuth-bin ground templates, white
// block weights, optionally the differenced timeline's (0, cos, sin) rows.
mm_status mm_set_templates(mm_ctx* ctx, int32_t poly_order, int32_t n_subscans, const int64_t* subscan_off,
                           const int32_t* az_bin, int32_t n_az_bins, int32_t stokes, int mem) {
    if (!ctx) return MM_ERR_ARG;
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    if (!ctx->have_pointing) return fail(ctx, MM_ERR_STATE, "mm_set_templates: set the pointing first");
    if (ctx->reduce_fn) return fail(ctx, MM_ERR_ARG, "mm_set_templates: not supported with a cross-rank reduction");
    if (mem != MM_HOST && mem != MM_DEVICE) return fail(ctx, MM_ERR_ARG, "mem must be MM_HOST or MM_DEVICE");
    ctx->have_bd = false;   // M_BD and any coarse space belong to the previous operator
    ctx->k = 0;
    ctx->tpref_valid = false;
    ctx->z32_valid = false;
    if (stokes < 0 || stokes > 2) return fail(ctx, MM_ERR_ARG, "stokes must be 0 (I, Q, U), 1 (Q, U) or 2 (I)");
    if (poly_order < 0 && !az_bin && stokes == 0) {
        ctx->tmpl_on = false;
        ctx->tmpl_qu = 0;
        return MM_OK;
    }
    if (ctx->lam != 0)
        return fail(ctx, MM_ERR_ARG, "template filters need white block weights: set the pointing with half_bw = 0");
    if (poly_order < -1 || poly_order > 3) return fail(ctx, MM_ERR_ARG, "poly_order must be -1..3");
    if (az_bin && (n_az_bins <= 0 || n_az_bins > 8192)) return fail(ctx, MM_ERR_ARG, "n_az_bins must be 1..8192");
    const int64_t N = ctx->n_samples;
    std::vector<int64_t> so;
    if (poly_order >= 0) {
        if (n_subscans <= 0 || !subscan_off) return fail(ctx, MM_ERR_ARG, "subscan offsets needed for poly_order >= 0");
        so.assign(subscan_off, subscan_off + n_subscans + 1);
    } else {
        so = ctx->block_off;   // unused without polynomials
    }
    const int ns = (int)so.size() - 1;
    if (so[0] != 0 || so[ns] != N) return fail(ctx, MM_ERR_ARG, "subscan_off must start at 0 and end at n_samples");
    std::vector<int32_t> blk_sub;
    std::vector<double> ginv;
    std::string lerr;
    if (!host_template_layout(ctx->block_off, so, poly_order, blk_sub, ginv, lerr)) return fail(ctx, MM_ERR_ARG, lerr);
    std::vector<double> wb(ctx->n_blocks);
    int64_t maxb = 0;
    for (int b = 0; b < ctx->n_blocks; ++b) {
        wb[b] = ctx->band[(size_t)ctx->block_band[b] * (ctx->lam + 1)];
        maxb = std::max(maxb, ctx->block_off[b + 1] - ctx->block_off[b]);
    }
    const int nbins = az_bin ? n_az_bins : 0;
    if (tmpl_smem_bytes(maxb, nbins, true) > smem_limit_bytes())
        return fail(ctx, MM_ERR_ARG, "template filters: longest block plus azimuth bins exceed shared memory");
    CK(ctx->d_tsub.ensure(so.size() * 8));
    ctx->tmpl_sub = so;
    CK(ctx->d_tblk.ensure(blk_sub.size() * 4));
    CK(ctx->d_tginv.ensure(ginv.size() * 8));
    CK(ctx->d_twb.ensure(wb.size() * 8));
    CK(cudaMemcpyAsync(ctx->d_tsub.p, so.data(), so.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_tblk.p, blk_sub.data(), blk_sub.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_tginv.p, ginv.data(), ginv.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->d_twb.p, wb.data(), wb.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    if (az_bin) {
        CK(ctx->d_taz.ensure((size_t)N * 4));
        CK(copy_in(ctx->d_taz.p, az_bin, (size_t)N * 4, mem, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->tmpl_on = true;
    ctx->tmpl_order = poly_order;
    ctx->tmpl_bins = nbins;
    ctx->tmpl_qu = stokes;
    ctx->tmpl_max_block = maxb;
    ctx->p64 = 1;   // native float64 by default; "fp64_products" = 2 selects double-float afterwards
    return MM_OK;
}

mm_status mm_build_bd(mm_ctx* ctx, double rcond_min, int32_t* n_dropped_out) {
    if (!ctx) return MM_ERR_ARG;
    if (!ctx->have_pointing) return fail(ctx, MM_ERR_STATE, "mm_setup_pointing first");
    if (!(rcond_min >= 0.0) || rcond_min > 1.0) return fail(ctx, MM_ERR_ARG, "rcond_min must lie in [0, 1]");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    const int n_pix = ctx->n_pix;
    CK(ctx->d_sums.ensure((size_t)n_pix * 7 * 8));
    CK(ctx->d_good.ensure(n_pix));
    CK(ctx->d_bd.ensure((size_t)n_pix * 6 * 8));
    CK(ctx->d_dropped.ensure(16));
    CK(cudaMemsetAsync(ctx->d_sums.p, 0, ctx->d_sums.bytes, ctx->stream));
    CK(cudaMemsetAsync(ctx->d_dropped.p, 0, 16, ctx->stream));
    DevBuf d_len;
    CK(d_len.ensure(8));
    const int64_t full = ctx->n_t;
    CK(cudaMemcpyAsync(d_len.p, &full, 8, cudaMemcpyHostToDevice, ctx->stream));
    launch_bd_accumulate(ctx->d_pix.as<int32_t>(), ctx->d_psi.as<float>(), ctx->d_block_off.as<int64_t>(),
                         ctx->d_block_band.as<int32_t>(), ctx->d_band64.as<double>(), ctx->lam + 1, ctx->n_blocks, 0,
                         ctx->n_t, d_len.as<int64_t>(), 1, ctx->d_sums.as<double>(), n_pix, ctx->stream);
    CKL();
    TRY(reduce_sum(ctx, ctx->d_sums.p, (int64_t)n_pix * 7, 8));
    launch_bd_invert(ctx->d_sums.as<double>(), ctx->d_bd.as<double>(), ctx->d_good.as<uint8_t>(),
                     ctx->d_dropped.as<int>(), n_pix, 1, rcond_min, 1, ctx->stream, ctx->tmpl_on ? ctx->tmpl_qu : 0);
    launch_flag_samples(ctx->d_pix.as<int32_t>(), ctx->d_good.as<uint8_t>(), ctx->n_samples, ctx->stream);
    CKL();
    int dropped = 0;
    CK(cudaMemcpyAsync(&dropped, ctx->d_dropped.p, 4, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (n_dropped_out) *n_dropped_out = dropped;
    ctx->have_bd = true;
    ctx->k = 0;
    ctx->tpref_valid = false;
    ctx->z32_valid = false;
    return MM_OK;
}

mm_status mm_rhs(mm_ctx* ctx, const void* tod, double* b_out, int32_t nrhs, int mem) {
    if (!ctx) return MM_ERR_ARG;
    if (!ctx->have_pointing) return fail(ctx, MM_ERR_STATE, "mm_setup_pointing first");
    if (!tod || !b_out || nrhs <= 0) return fail(ctx, MM_ERR_ARG, "null array or nrhs <= 0");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    const size_t esz = is_f32(ctx) ? 4 : 8;
    DevBuf d_tod;
    const void* src = tod;
    if (mem == MM_HOST) {
        CK(d_tod.ensure((size_t)nrhs * ctx->n_samples * esz));
        CK(cudaMemcpyAsync(d_tod.p, tod, d_tod.bytes, cudaMemcpyHostToDevice, ctx->stream));
        src = d_tod.p;
    }
    Plan* plan = nullptr;
    TRY(get_plan(ctx, ctx->p64, nrhs, {}, &plan));
    TRY(ensure_work(ctx, nrhs, ctx->k));
    DevBuf q;
    CK(q.ensure((size_t)nrhs * ctx->n_pix * sizeof(V4<double>)));
    CK(cudaMemsetAsync(q.p, 0, q.bytes, ctx->stream));
    TRY(run_filter(ctx, plan, true, src, q.p, nullptr, is_f32(ctx) ? 1 : 0));
    CK(ctx->d_lastb.ensure((size_t)ctx->n_pix * sizeof(V4<double>)));
    CK(cudaMemcpyAsync(ctx->d_lastb.p, q.p, (size_t)ctx->n_pix * sizeof(V4<double>), cudaMemcpyDeviceToDevice, ctx->stream));
    ctx->have_lastb = true;
    if (mem == MM_HOST) {
        DevBuf o;
        CK(o.ensure((size_t)nrhs * ctx->n_pix * 3 * 8));
        launch_map_out(q.as<V4<double>>(), o.as<double>(), (int64_t)nrhs * ctx->n_pix, ctx->stream);
        CKL();
        CK(cudaMemcpyAsync(b_out, o.p, o.bytes, cudaMemcpyDeviceToHost, ctx->stream));
    } else {
        launch_map_out(q.as<V4<double>>(), b_out, (int64_t)nrhs * ctx->n_pix, ctx->stream);
        CKL();
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return MM_OK;
}

mm_status mm_apply_A(mm_ctx* ctx, const double* x, double* y, int32_t nrhs, int mem) {
    if (!ctx) return MM_ERR_ARG;
    if (!ctx->have_pointing) return fail(ctx, MM_ERR_STATE, "mm_setup_pointing first");
    if (!x || !y || nrhs <= 0) return fail(ctx, MM_ERR_ARG, "null array or nrhs <= 0");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    TRY(ensure_work(ctx, nrhs, ctx->k));
    const int64_t nv = (int64_t)nrhs * ctx->n_pix;
    // the context's work vectors (sized for nrhs by ensure_work) hold the 4-wide copies, so repeated
    // calls allocate nothing on the device
    DevBuf in3;
    DevBuf& in4 = ctx->w_a;
    DevBuf& out4 = ctx->w_b;
    const double* xsrc = x;
    if (mem == MM_HOST) {
        CK(in3.ensure(nv * 3 * 8));
        CK(cudaMemcpyAsync(in3.p, x, nv * 24, cudaMemcpyHostToDevice, ctx->stream));
        xsrc = in3.as<double>();
    }
    launch_map_in(xsrc, in4.as<V4<double>>(), nv, ctx->stream);
    CKL();
    Plan* plan = nullptr;
    const int aprec = ctx->opt_apply_prec ? ctx->opt_apply_prec : op_prec(ctx);
    TRY(get_plan(ctx, aprec, nrhs, {}, &plan));
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    TRY(apply_A_dev(ctx, aprec, in4.as<V4<double>>(), out4.as<V4<double>>(), nrhs, plan));
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    if (mem == MM_HOST) {
        DevBuf o;
        CK(o.ensure(nv * 24));
        launch_map_out(out4.as<V4<double>>(), o.as<double>(), nv, ctx->stream);
        CKL();
        CK(cudaMemcpyAsync(y, o.p, nv * 24, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    } else {
        launch_map_out(out4.as<V4<double>>(), y, nv, ctx->stream);
        CKL();
        CK(cudaStreamSynchronize(ctx->stream));
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    ctx->last_apply_ms = ms;
    return MM_OK;
}

mm_status mm_apply_precond(mm_ctx* ctx, mm_precond which, const double* x, double* y, int32_t nrhs, int mem) {
    if (!ctx) return MM_ERR_ARG;
    if (!ctx->have_bd) return fail(ctx, MM_ERR_STATE, "mm_build_bd first");
    if (which == MM_PRECOND_2L && ctx->k <= 0) return fail(ctx, MM_ERR_STATE, "no coarse space");
    if (which != MM_PRECOND_BD && which != MM_PRECOND_2L) return fail(ctx, MM_ERR_ARG, "unknown preconditioner");
    if (!x || !y || nrhs <= 0) return fail(ctx, MM_ERR_ARG, "null array or nrhs <= 0");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    TRY(ensure_work(ctx, nrhs, ctx->k));
    const int64_t nv = (int64_t)nrhs * ctx->n_pix;
    // the context's work vectors (sized for nrhs by ensure_work) hold the 4-wide copies, so repeated
    // calls allocate nothing on the device
    DevBuf in3;
    DevBuf& in4 = ctx->w_a;
    DevBuf& out4 = ctx->w_b;
    DevBuf& u = ctx->w_u;
    const double* xsrc = x;
    if (mem == MM_HOST) {
        CK(in3.ensure(nv * 24));
        CK(cudaMemcpyAsync(in3.p, x, nv * 24, cudaMemcpyHostToDevice, ctx->stream));
        xsrc = in3.as<double>();
    }
    launch_map_in(xsrc, in4.as<V4<double>>(), nv, ctx->stream);
    if (which == MM_PRECOND_BD) {
        launch_bd_apply(ctx->d_bd.as<double>(), 0, in4.as<V4<double>>(), out4.as<V4<double>>(), ctx->n_pix, nrhs,
                        ctx->stream);
    } else {
        CK(u.ensure((size_t)nrhs * ctx->k * 8));
        CK(ctx->w_partial.ensure((size_t)ctx->grid_x * nrhs * ctx->k * 8 + 64));
        PcgArgs a{};
        a.n_pix = ctx->n_pix;
        a.nrhs = nrhs;
        a.st = nullptr;
        a.bd = ctx->d_bd.as<double>();
        a.bd_per_rhs = 0;
        a.k = ctx->k;
        a.Z = ctx->d_Z.as<V4<double>>();
        a.AZ = ctx->d_AZ.as<V4<double>>();
        a.Einv = ctx->d_Einv.as<double>();
        a.u = u.as<double>();
        a.partial = ctx->w_partial.as<double>();
        a.counter = ctx->w_counter.as<unsigned>();
        a.grid_x = ctx->grid_x;
        if (tc_wanted(ctx, a)) TRY(ensure_tc_scratch(ctx, a));
        m2l_apply(ctx, a, in4.as<V4<double>>(), out4.as<V4<double>>(), -1);
    }
    CKL();
    if (mem == MM_HOST) {
        DevBuf o;
        CK(o.ensure(nv * 24));
        launch_map_out(out4.as<V4<double>>(), o.as<double>(), nv, ctx->stream);
        CK(cudaMemcpyAsync(y, o.p, nv * 24, cudaMemcpyDeviceToHost, ctx->stream));
    } else {
        launch_map_out(out4.as<V4<double>>(), y, nv, ctx->stream);
    }
    CKL();
    CK(cudaStreamSynchronize(ctx->stream));
    if (which == MM_PRECOND_2L) TRY(tc_fault_check(ctx));
    return MM_OK;
}

mm_status mm_build_coarse(mm_ctx* ctx, const double* b_or_null, int32_t m_max, double eps_arn, int32_t k,
                          double eps_lambda, int32_t* k_out, int mem) {
    if (!ctx) return MM_ERR_ARG;
    if (!ctx->have_bd) return fail(ctx, MM_ERR_STATE, "mm_build_bd first");
    if (m_max <= 0 || m_max > 1024) return fail(ctx, MM_ERR_ARG, "m_max must lie in [1, 1024]");
    if (k > MM_K_MAX) return fail(ctx, MM_ERR_ARG, "k must be at most 512");
    if (!b_or_null && !ctx->have_lastb) return fail(ctx, MM_ERR_STATE, "no right-hand side: pass b or call mm_rhs");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    const int n_pix = ctx->n_pix;
    const int64_t n = (int64_t)n_pix * 4;
    ctx->k = 0;
    ctx->tpref_valid = false;
    ctx->z32_valid = false;
    TRY(ensure_work(ctx, 1, MM_K_MAX));
    CK(ctx->w_partial.ensure((size_t)ctx->grid_x * (m_max + 2) * 8 + 64));
    CK(ctx->d_W.ensure((size_t)(m_max + 1) * n * 8));
    CK(ctx->d_h.ensure((size_t)(m_max + 2) * 8 * 2));
    V4<double>* bvec = ctx->w_a.as<V4<double>>();
    if (b_or_null) {
        DevBuf in3;
        const double* src = b_or_null;
        if (mem == MM_HOST) {
            CK(in3.ensure(n_pix * 24));
            CK(cudaMemcpyAsync(in3.p, b_or_null, n_pix * 24, cudaMemcpyHostToDevice, ctx->stream));
            src = in3.as<double>();
        }
        launch_map_in(src, bvec, n_pix, ctx->stream);
        CK(cudaStreamSynchronize(ctx->stream));
    } else {
        CK(cudaMemcpyAsync(bvec, ctx->d_lastb.p, n_pix * sizeof(V4<double>), cudaMemcpyDeviceToDevice, ctx->stream));
    }
    double* W = ctx->d_W.as<double>();
    // w_1 = M_BD b / ||M_BD b||
    launch_bd_apply(ctx->d_bd.as<double>(), 0, bvec, reinterpret_cast<V4<double>*>(W), n_pix, 1, ctx->stream);
    double* h = ctx->d_h.as<double>();
    launch_multidot(W, n, 1, W, n, h, ctx->w_partial.as<double>(), ctx->w_counter.as<unsigned>(), ctx->grid_x, ctx->stream);
    double nrm2 = 0.0;
    CK(cudaMemcpyAsync(&nrm2, h, 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (!(nrm2 > 0.0)) return fail(ctx, MM_ERR_ARG, "M_BD b is zero: no Krylov space");
    launch_scale_host(W, n, 1.0 / std::sqrt(nrm2), ctx->stream);
    std::vector<double> H((size_t)(m_max + 1) * m_max, 0.0);   // row-major (m_max+1) x m_max
    Plan* plan = nullptr;
    const int f64 = op_prec(ctx);
    TRY(get_plan(ctx, f64, 1, {}, &plan));
    V4<double>* q = ctx->w_b.as<V4<double>>();
    int m = m_max;
    std::vector<double> hcol(m_max + 2);
    for (int j = 0; j < m_max; ++j) {
        double* wj = W + (int64_t)j * n;
        double* v = W + (int64_t)(j + 1) * n;
        TRY(apply_A_dev(ctx, f64, reinterpret_cast<V4<double>*>(wj), q, 1, plan));
        launch_bd_apply(ctx->d_bd.as<double>(), 0, q, reinterpret_cast<V4<double>*>(v), n_pix, 1, ctx->stream);
        // two classical Gram-Schmidt passes
        for (int pass = 0; pass < 2; ++pass) {
            launch_multidot(W, n, j + 1, v, n, h + (size_t)pass * (m_max + 2), ctx->w_partial.as<double>(),
                            ctx->w_counter.as<unsigned>(), ctx->grid_x, ctx->stream);
            launch_sub_combo(W, n, j + 1, h + (size_t)pass * (m_max + 2), v, n, ctx->stream);
        }
        launch_multidot(v, n, 1, v, n, h + (size_t)(m_max + 1), ctx->w_partial.as<double>(), ctx->w_counter.as<unsigned>(),
                        ctx->grid_x, ctx->stream);
        CKL();
        std::vector<double> h2(2 * (size_t)(m_max + 2));
        CK(cudaMemcpyAsync(h2.data(), h, h2.size() * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        for (int i = 0; i <= j; ++i) H[(size_t)i * m_max + j] = h2[i] + h2[(size_t)(m_max + 2) + i];
        const double hn = std::sqrt(std::max(0.0, h2[m_max + 1]));
        H[(size_t)(j + 1) * m_max + j] = hn;
        if (!(hn > eps_arn)) {
            m = j + 1;
            break;
        }
        launch_scale_host(v, n, 1.0 / hn, ctx->stream);
    }
    // Ritz pairs of H_m
    std::vector<double> Hm((size_t)m * m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) Hm[(size_t)i * m + j] = H[(size_t)i * m_max + j];
    // Ritz values first; Ritz vectors (inverse iteration) only for the selected ones
    std::vector<double> C, vals;
    const int rs = host_ritz_hess(Hm, m, k, MM_K_MAX, eps_lambda, C, vals);
    if (rs == 1) return fail(ctx, MM_ERR_SINGULAR, "eigen-solve of H_m failed");
    if (rs == 2) return fail(ctx, MM_ERR_ARG, "no Ritz value selected");
    const int ksel = (int)vals.size();
    DevBuf dC;
    CK(dC.ensure(C.size() * 8));
    CK(cudaMemcpyAsync(dC.p, C.data(), C.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(ctx->d_Z.ensure((size_t)ksel * n * 8));
    launch_combo(W, n, m, dC.as<double>(), ksel, ctx->d_Z.as<double>(), n, n, ctx->stream);
    CKL();
    CK(cudaStreamSynchronize(ctx->stream));
    int kk = 0;
    TRY(orthonormalise(ctx, ctx->d_Z, ksel, &kk));
    ctx->k = kk;
    ctx->ritz.assign(vals.begin(), vals.begin() + std::min<size_t>(vals.size(), kk));
    ctx->coarse_len = ctx->n_t;
    TRY(finish_coarse(ctx));
    if (k_out) *k_out = ctx->k;
    return MM_OK;
}

mm_status mm_build_coarse_from_solve(mm_ctx* ctx, int32_t k, double eps_lambda, int32_t* k_out) {
    if (!ctx) return MM_ERR_ARG;
    if (!ctx->have_bd) return fail(ctx, MM_ERR_STATE, "mm_build_bd first");
    if (ctx->harvest_count < 2) return fail(ctx, MM_ERR_STATE, "no harvested M_BD solve (set option harvest > 1)");
    if (k > MM_K_MAX) return fail(ctx, MM_ERR_ARG, "k must be at most 512");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    const int m = ctx->harvest_count;
    const int64_t n = (int64_t)ctx->n_pix * 4;
    std::vector<double> td, te;
    host_lanczos_tridiag(ctx->harv_alpha, ctx->harv_beta, m, td, te);
    std::vector<double> C, vals;
    const int rs = host_ritz_tridiag(td, te, m, k, MM_K_MAX, eps_lambda, C, vals);
    if (rs == 1) return fail(ctx, MM_ERR_SINGULAR, "eigen-solve of the Lanczos matrix failed");
    if (rs == 2) return fail(ctx, MM_ERR_ARG, "no Ritz value selected");
    const int ksel = (int)vals.size();
    DevBuf dC;
    CK(dC.ensure(C.size() * 8));
    CK(cudaMemcpyAsync(dC.p, C.data(), C.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    ctx->k = 0;
    ctx->tpref_valid = false;
    ctx->z32_valid = false;
    TRY(ensure_work(ctx, 1, MM_K_MAX));
    CK(ctx->d_Z.ensure((size_t)ksel * n * 8));
    launch_combo(ctx->d_harv.as<double>(), n, m, dC.as<double>(), ksel, ctx->d_Z.as<double>(), n, n, ctx->stream);
    CKL();
    CK(cudaStreamSynchronize(ctx->stream));
    int kk = 0;
    TRY(orthonormalise(ctx, ctx->d_Z, ksel, &kk));
    ctx->k = kk;
    ctx->ritz.assign(vals.begin(), vals.begin() + std::min<size_t>(vals.size(), kk));
    ctx->coarse_len = ctx->harvest_len > 0 ? ctx->harvest_len : ctx->n_t;
    TRY(finish_coarse(ctx));
    if (k_out) *k_out = ctx->k;
    return MM_OK;
}

mm_status mm_set_coarse(mm_ctx* ctx, int32_t k, const double* Z, int mem) {
    if (!ctx) return MM_ERR_ARG;
    if (!ctx->have_bd) return fail(ctx, MM_ERR_STATE, "mm_build_bd first");
    if (k <= 0 || k > MM_K_MAX || !Z) return fail(ctx, MM_ERR_ARG, "k must lie in [1, 512] and Z non-null");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    const int64_t n = (int64_t)ctx->n_pix * 4;
    ctx->k = 0;
    ctx->tpref_valid = false;
    ctx->z32_valid = false;
    DevBuf in3;
    const double* src = Z;
    if (mem == MM_HOST) {
        CK(in3.ensure((size_t)k * ctx->n_pix * 24));
        CK(cudaMemcpyAsync(in3.p, Z, in3.bytes, cudaMemcpyHostToDevice, ctx->stream));
        src = in3.as<double>();
    }
    CK(ctx->d_Z.ensure((size_t)k * n * 8));
    launch_map_in(src, ctx->d_Z.as<V4<double>>(), (int64_t)k * ctx->n_pix, ctx->stream);
    CKL();
    CK(cudaStreamSynchronize(ctx->stream));
    int kk = 0;
    TRY(orthonormalise(ctx, ctx->d_Z, k, &kk));
    ctx->k = kk;
    ctx->ritz.assign(kk, 0.0);
    ctx->coarse_len = ctx->n_t;
    TRY(finish_coarse(ctx));
    return MM_OK;
}

mm_status mm_get_coarse(mm_ctx* ctx, double* Z_out, double* ritz_out, int32_t* k_out) {
    if (!ctx) return MM_ERR_ARG;
    if (ctx->k <= 0) return fail(ctx, MM_ERR_STATE, "no coarse space");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    if (k_out) *k_out = ctx->k;
    if (ritz_out)
        for (int i = 0; i < ctx->k; ++i) ritz_out[i] = i < (int)ctx->ritz.size() ? ctx->ritz[i] : 0.0;
    if (Z_out) {
        DevBuf o;
        const int64_t nv = (int64_t)ctx->k * ctx->n_pix;
        CK(o.ensure(nv * 24));
        launch_map_out(ctx->d_Z.as<V4<double>>(), o.as<double>(), nv, ctx->stream);
        CKL();
        CK(cudaMemcpyAsync(Z_out, o.p, nv * 24, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
    }
    return MM_OK;
}

mm_status mm_export_coarse(mm_ctx* ctx, void* buf, int64_t* bytes) {
    if (!ctx || !bytes) return MM_ERR_ARG;
    if (ctx->k <= 0) return fail(ctx, MM_ERR_STATE, "no coarse space");
    const int k = ctx->k;
    const int64_t need = (int64_t)sizeof(CoarseFileHeader) + coarse_payload_bytes(ctx->n_pix, k);
    if (!buf) {
        *bytes = need;
        return MM_OK;
    }
    if (*bytes < need) return fail(ctx, MM_ERR_ARG, "buffer smaller than the exported coarse space");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    CoarseFileHeader hd{};
    std::memcpy(hd.magic, kCoarseMagic, 8);
    hd.version = 1;
    hd.n_pix = ctx->n_pix;
    hd.k = k;
    hd.op_prec = op_prec(ctx);
    TRY(scan_fingerprint(ctx, &hd.fingerprint));
    hd.payload_bytes = coarse_payload_bytes(ctx->n_pix, k);
    unsigned char* o = static_cast<unsigned char*>(buf);
    std::memcpy(o, &hd, sizeof(hd));
    double* z3 = reinterpret_cast<double*>(o + sizeof(hd));
    const int64_t nv = (int64_t)k * ctx->n_pix;
    DevBuf t;
    CK(t.ensure(nv * 24));
    launch_map_out(ctx->d_Z.as<V4<double>>(), t.as<double>(), nv, ctx->stream);
    CKL();
    CK(cudaMemcpyAsync(z3, t.p, nv * 24, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    launch_map_out(ctx->d_AZ.as<V4<double>>(), t.as<double>(), nv, ctx->stream);
    CKL();
    CK(cudaMemcpyAsync(z3 + nv * 3, t.p, nv * 24, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(z3 + nv * 6, ctx->d_Einv.p, (size_t)k * k * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double* rz = z3 + nv * 6 + (int64_t)k * k;
    for (int i = 0; i < k; ++i) rz[i] = i < (int)ctx->ritz.size() ? ctx->ritz[i] : 0.0;
    *bytes = need;
    return MM_OK;
}

mm_status mm_import_coarse(mm_ctx* ctx, const void* buf, int64_t bytes) {
    if (!ctx) return MM_ERR_ARG;
    if (!ctx->have_bd) return fail(ctx, MM_ERR_STATE, "mm_build_bd first");
    if (!buf || bytes < (int64_t)sizeof(CoarseFileHeader)) return fail(ctx, MM_ERR_ARG, "buffer too small");
    CoarseFileHeader hd{};
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, kCoarseMagic, 8) != 0 || hd.version != 1)
        return fail(ctx, MM_ERR_ARG, "not an exported coarse space (magic or version)");
    if (hd.k <= 0 || hd.k > MM_K_MAX || hd.n_pix != ctx->n_pix ||
        hd.payload_bytes != coarse_payload_bytes(hd.n_pix, hd.k) ||
        bytes < (int64_t)sizeof(hd) + hd.payload_bytes)
        return fail(ctx, MM_ERR_ARG, "exported coarse space does not match this problem's size or is truncated");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    uint64_t fp = 0;
    TRY(scan_fingerprint(ctx, &fp));
    if (fp != hd.fingerprint || hd.op_prec != op_prec(ctx))
        return fail(ctx, MM_ERR_ARG,
                    "exported coarse space belongs to another scan, filter or operator precision (fingerprint)");
    const int k = hd.k;
    const int64_t n4 = (int64_t)ctx->n_pix * 4, nv = (int64_t)k * ctx->n_pix;
    const double* z3 = reinterpret_cast<const double*>(static_cast<const unsigned char*>(buf) + sizeof(hd));
    ctx->k = 0;
    ctx->tpref_valid = false;
    ctx->z32_valid = false;
    DevBuf t;
    CK(t.ensure(nv * 24));
    CK(ctx->d_Z.ensure((size_t)k * n4 * 8));
    CK(ctx->d_AZ.ensure((size_t)k * n4 * 8));
    CK(ctx->d_Einv.ensure((size_t)k * k * 8));
    CK(cudaMemcpyAsync(t.p, z3, nv * 24, cudaMemcpyHostToDevice, ctx->stream));
    launch_map_in(t.as<double>(), ctx->d_Z.as<V4<double>>(), nv, ctx->stream);
    CKL();
    CK(cudaStreamSynchronize(ctx->stream));
    CK(cudaMemcpyAsync(t.p, z3 + nv * 3, nv * 24, cudaMemcpyHostToDevice, ctx->stream));
    launch_map_in(t.as<double>(), ctx->d_AZ.as<V4<double>>(), nv, ctx->stream);
    CKL();
    CK(cudaMemcpyAsync(ctx->d_Einv.p, z3 + nv * 6, (size_t)k * k * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    const double* rz = z3 + nv * 6 + (int64_t)k * k;
    ctx->ritz.assign(rz, rz + k);
    ctx->coarse_len = ctx->n_t;
    ctx->k = k;
    return MM_OK;
}

mm_status mm_set_reduction(mm_ctx* ctx, mm_reduce_fn fn, void* user, int on_device) {
    if (!ctx) return MM_ERR_ARG;
    if (ctx->phase != PH_IDLE) return fail(ctx, MM_ERR_STATE, "mm_set_reduction: a solve is in progress");
    if (fn && ctx->tmpl_on) return fail(ctx, MM_ERR_ARG, "mm_set_reduction: not supported with template filters");
    ctx->reduce_fn = fn;
    ctx->reduce_user = user;
    ctx->reduce_dev = on_device ? 1 : 0;
    destroy_graph(ctx);
    return MM_OK;
}

mm_status mm_solve_begin(mm_ctx* ctx, const void* tod, int32_t nrhs, const int64_t* rhs_len, mm_precond precond,
                         double tol, int32_t max_iter, int mem) {
    if (!ctx) return MM_ERR_ARG;
    if (!ctx->have_bd) return fail(ctx, MM_ERR_STATE, "mm_build_bd first");
    if (!tod || nrhs <= 0) return fail(ctx, MM_ERR_ARG, "null TOD or nrhs <= 0");
    if (precond != MM_PRECOND_BD && precond != MM_PRECOND_2L) return fail(ctx, MM_ERR_ARG, "unknown preconditioner");
    if (precond == MM_PRECOND_2L && ctx->k <= 0) return fail(ctx, MM_ERR_STATE, "no coarse space for M_2l");
    if (!(tol >= 0.0) || max_iter < 0) return fail(ctx, MM_ERR_ARG, "tol must be >= 0 and max_iter >= 0");
    if (rhs_len)
        for (int i = 0; i < nrhs; ++i)
            if (rhs_len[i] <= 0 || rhs_len[i] > ctx->n_t) return fail(ctx, MM_ERR_ARG, "rhs_len out of (0, n_t]");
    if (rhs_len && ctx->reduce_fn)
        return fail(ctx, MM_ERR_ARG, "right-hand sides of uneven length are not supported with a cross-rank reduction");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    destroy_graph(ctx);
    ctx->nrhs = nrhs;
    ctx->precond = precond;
    ctx->tol = tol;
    ctx->max_iter = max_iter;
    ctx->use_lens = rhs_len != nullptr;
    ctx->lens.clear();
    if (rhs_len) ctx->lens.assign(rhs_len, rhs_len + nrhs);
    const int64_t nv = (int64_t)nrhs * ctx->n_pix;
    const size_t v4 = nv * sizeof(V4<double>);
    const bool f32 = is_f32(ctx);
    TRY(ensure_work(ctx, nrhs, ctx->k));
    CK(ctx->w_partial.ensure((size_t)ctx->grid_x * nrhs * std::max(2, ctx->k) * 8 + 64));
    CK(ctx->s_b.ensure(v4));
    CK(ctx->s_x.ensure(v4));
    CK(ctx->s_r.ensure(v4));
    CK(ctx->s_z.ensure(v4));
    CK(ctx->s_p.ensure(v4));
    CK(ctx->s_src.ensure(f32 ? nv * sizeof(V4<float>) : v4));
    CK(ctx->s_q.ensure(f32 ? nv * sizeof(V4<float>) : v4));
    CK(ctx->s_q64.ensure(v4));
    CK(ctx->s_xtot.ensure(v4));
    CK(ctx->s_rtrue.ensure(v4));
    CK(ctx->s_st.ensure(nrhs * sizeof(RhsState)));
    CK(ctx->s_hist.ensure((size_t)nrhs * (max_iter + 1) * 8));
    CK(ctx->s_u.ensure((size_t)nrhs * std::max(1, ctx->k) * 8));
    CK(ctx->s_mask.ensure((size_t)nrhs * 4 + 16));
    if (ctx->use_lens) TRY(bd_for_lens(ctx));
    ctx->harvest_on = false;
    if (ctx->opt_harvest > 0 && precond == MM_PRECOND_BD) {
        CK(ctx->d_harv.ensure((size_t)ctx->opt_harvest * ctx->n_pix * sizeof(V4<double>)));
        CK(ctx->d_ahist.ensure((size_t)nrhs * (max_iter + 1) * 8));
        CK(ctx->d_bhist.ensure((size_t)nrhs * (max_iter + 1) * 8));
        ctx->harvest_on = true;
        ctx->harvest_count = 0;
        ctx->harvest_len = ctx->use_lens ? ctx->lens[0] : ctx->n_t;
    }
    ctx->coarse_per_rhs = false;
    ctx->precond_used.assign(nrhs, precond);
    std::vector<uint8_t> deflate(nrhs, 1);
    if (ctx->use_lens && precond == MM_PRECOND_2L && ctx->opt_coarse_fallback) {
        // A basis deflates the small eigenmodes of the operator it was built from.  A prefix of
        // another length covers the patch differently (other pixels are poorly hit), its small
        // modes are not in span Z, and M_2l then costs more than M_BD for the same products: such
        // right-hand sides run M_BD (E_i^-1 = 0 makes M_2l,i = M_BD,i); a batch with none left runs
        // M_BD throughout.
        const int64_t tolen = std::max<int64_t>(1, ctx->coarse_len / 100);
        int n_defl = 0;
        for (int i = 0; i < nrhs; ++i) {
            deflate[i] = std::llabs(ctx->lens[i] - ctx->coarse_len) <= tolen;
            n_defl += deflate[i];
            if (!deflate[i]) ctx->precond_used[i] = MM_PRECOND_BD;
        }
        if (n_defl == 0) ctx->precond = MM_PRECOND_BD;
    }
    if (ctx->use_lens && ctx->precond == MM_PRECOND_2L) TRY(coarse_for_lens(ctx, deflate));
    if (ctx->precond == MM_PRECOND_2L && is_f32(ctx) && !ctx->z32_valid && ctx->k > 0) {
        // the coarse sums of M_2l in float32 read float32 copies, made once per coarse space
        const int64_t nz = (int64_t)ctx->k * ctx->n_pix;
        CK(ctx->d_Z32.ensure(nz * sizeof(V4<float>)));
        CK(ctx->d_AZ32.ensure(nz * sizeof(V4<float>)));
        launch_to_f32(ctx->d_Z.as<V4<double>>(), ctx->d_Z32.as<V4<float>>(), nz, ctx->stream);
        launch_to_f32(ctx->d_AZ.as<V4<double>>(), ctx->d_AZ32.as<V4<float>>(), nz, ctx->stream);
        CKL();
        ctx->z32_valid = true;
    }
    if (ctx->precond == MM_PRECOND_2L) {
        const PcgArgs a = pcg_args(ctx);
        if (tc_wanted(ctx, a)) TRY(ensure_tc_scratch(ctx, a));
    }
    TRY(get_plan(ctx, op_prec(ctx), nrhs, ctx->lens, &ctx->plan_op));
    TRY(get_plan(ctx, ctx->p64, nrhs, ctx->lens, &ctx->plan_64));
    CK(cudaEventRecord(ctx->ev0, ctx->stream));
    const size_t esz = f32 ? 4 : 8;
    const void* src = tod;
    ctx->tod_dev = nullptr;
    if (mem == MM_HOST || f32) {
        // the mixed-precision refinement reads the timeline again (residuals
        // P^T W (d - P x)), so it keeps its own device copy
        CK(ctx->s_tod.ensure((size_t)nrhs * ctx->n_samples * esz));
        CK(cudaMemcpyAsync(ctx->s_tod.p, tod, (size_t)nrhs * ctx->n_samples * esz,
                           mem == MM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, ctx->stream));
        src = ctx->s_tod.p;
        ctx->tod_dev = ctx->s_tod.p;
    }
    CK(cudaMemsetAsync(ctx->s_b.p, 0, v4, ctx->stream));
    if (f32) {
        // b = P^T W d with the float32 operator: the inner solve stops at
        // float32 accuracy anyway, and every refinement residual comes from d
        TRY(ensure_work(ctx, nrhs, ctx->k));
        V4<float>* q = ctx->w_q.as<V4<float>>();
        CK(cudaMemsetAsync(q, 0, (size_t)ctx->n_pix * nrhs * sizeof(V4<float>), ctx->stream));
        TRY(run_filter(ctx, ctx->plan_op, true, src, q, nullptr, 1));
        launch_from_f32(q, ctx->s_b.as<V4<double>>(), (int64_t)ctx->n_pix * nrhs, ctx->stream);
        CKL();
    } else {
        // b = P^T W d in float64
        TRY(run_filter(ctx, ctx->plan_64, true, src, ctx->s_b.p, nullptr, 0));
    }
    CK(ctx->d_lastb.ensure((size_t)ctx->n_pix * sizeof(V4<double>)));
    CK(cudaMemcpyAsync(ctx->d_lastb.p, ctx->s_b.p, (size_t)ctx->n_pix * sizeof(V4<double>), cudaMemcpyDeviceToDevice,
                       ctx->stream));
    ctx->have_lastb = true;
    CK(cudaMemsetAsync(ctx->s_xtot.p, 0, v4, ctx->stream));
    ctx->tot_iters.assign(nrhs, 0);
    ctx->refinements.assign(nrhs, 0);
    ctx->final_status.assign(nrhs, 0);
    ctx->true_res.assign(nrhs, 1.0);
    ctx->rec_res.assign(nrhs, 1.0);
    ctx->outer = 0;
    // ||b|| on the host for the refinement tolerances
    std::vector<double> bb;
    {
        CK(cudaMemsetAsync(ctx->s_q64.p, 0, v4, ctx->stream));
        launch_residual(ctx->s_b.as<V4<double>>(), ctx->s_q64.as<V4<double>>(), nullptr, ctx->w_norms.as<double>(),
                        ctx->n_pix, nrhs, ctx->w_partial.as<double>(), ctx->w_counter.as<unsigned>(), ctx->grid_x,
                        ctx->stream);
        CKL();
        bb.resize(nrhs);
        CK(cudaMemcpyAsync(bb.data(), ctx->w_norms.p, nrhs * 8, cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        ctx->bnorm.resize(nrhs);
        for (int i = 0; i < nrhs; ++i) ctx->bnorm[i] = std::sqrt(bb[i]);
    }
    std::vector<double> tols(nrhs);
    std::vector<int> budgets(nrhs, max_iter);
    for (int i = 0; i < nrhs; ++i) tols[i] = f32 ? std::max(tol, ctx->opt_inner_tol) : tol;
    TRY(pcg_start(ctx, ctx->s_b.as<V4<double>>(), tols, budgets));
    ctx->phase = PH_INNER;
    return MM_OK;
}

static mm_status finish_inner(mm_ctx* ctx, int32_t* done, bool allow_refine) {
    // all inner PCG runs have stopped: accumulate and (mixed) refine
    const int R = ctx->nrhs;
    if (ctx->harvest_on) {
        // the Lanczos sequence is the first inner solve's; restarts would begin a new one
        ctx->harvest_on = false;
        const int m = std::min(ctx->h_st[0].iters, ctx->opt_harvest);
        ctx->harvest_count = m;
        ctx->harv_alpha.assign(m, 0.0);
        ctx->harv_beta.assign(m, 0.0);
        if (m > 0) {
            CK(cudaMemcpyAsync(ctx->harv_alpha.data(), ctx->d_ahist.p, m * 8, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaMemcpyAsync(ctx->harv_beta.data(), ctx->d_bhist.p, m * 8, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
        }
    }
    std::vector<int32_t> mask(R, 1);
    for (int i = 0; i < R; ++i) {
        ctx->tot_iters[i] += ctx->h_st[i].iters;
        if (ctx->h_st[i].iters > 0 || ctx->outer == 0) ctx->rec_res[i] = ctx->h_st[i].relres;
        if (ctx->h_st[i].status == 6) ctx->final_status[i] = MM_ERR_BREAKDOWN;
    }
    CK(cudaMemcpyAsync(ctx->s_mask.p, mask.data(), R * 4, cudaMemcpyHostToDevice, ctx->stream));
    launch_axpy_masked(ctx->s_xtot.as<double>(), ctx->s_x.as<double>(), (int64_t)ctx->n_pix * 4, R,
                       ctx->s_mask.as<int32_t>(), ctx->stream);
    CKL();
    std::vector<double> rr;
    TRY(true_residual(ctx, ctx->s_xtot.as<V4<double>>(), rr));
    bool again = false;
    std::vector<double> tols(R, 0.0);
    std::vector<int> budgets(R, 0);
    for (int i = 0; i < R; ++i) {
        ctx->true_res[i] = ctx->bnorm[i] > 0 ? rr[i] / ctx->bnorm[i] : 0.0;
        if (!is_f32(ctx)) continue;
        const int left = ctx->max_iter - ctx->tot_iters[i];
        if (ctx->final_status[i] == MM_ERR_BREAKDOWN) continue;
        if (allow_refine && ctx->true_res[i] > ctx->tol && left > 0 && ctx->outer < 8 && rr[i] > 0) {
            again = true;
            budgets[i] = left;
            tols[i] = std::max(0.5 * ctx->tol * ctx->bnorm[i] / rr[i], ctx->opt_inner_tol);
        }
    }
    if (again) {
        ctx->outer += 1;
        for (int i = 0; i < R; ++i)
            if (budgets[i] > 0) ctx->refinements[i] += 1;
        TRY(pcg_start(ctx, ctx->s_rtrue.as<V4<double>>(), tols, budgets));
        *done = 0;
        return MM_OK;
    }
    for (int i = 0; i < R; ++i) {
        if (ctx->final_status[i] != 0) continue;
        const double target = is_f32(ctx) ? ctx->true_res[i] : ctx->rec_res[i];
        if (!(target <= ctx->tol)) ctx->final_status[i] = MM_ERR_NOT_CONVERGED;
        // float64 products: the recurrence stops the solve, but a true residual far above it means the
        // recurrence drifted (an inconsistent preconditioner): not converged either
        if (!is_f32(ctx) && !(ctx->true_res[i] <= 100.0 * ctx->tol)) ctx->final_status[i] = MM_ERR_NOT_CONVERGED;
    }
    ctx->phase = PH_DONE;
    *done = 1;
    return MM_OK;
}

static mm_status launch_iters(mm_ctx* ctx, int32_t n_iter) {
    if (n_iter <= 0) return MM_OK;
    NvtxRange nvtx_range("pcg_iterations");
    const bool capturable = ctx->stream != nullptr && ctx->stream != cudaStreamLegacy &&
                            ctx->stream != cudaStreamPerThread;
    if (ctx->opt_graphs && capturable && !ctx->reduce_fn && n_iter == ctx->opt_check_every) {
        if (!ctx->graph_exec) {
            // one eager iteration first so every kernel attribute is configured
            TRY(pcg_iteration(ctx));
            cudaGraph_t g;
            CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
            ctx->capturing = true;
            mm_status s = MM_OK;
            for (int i = 0; i < n_iter && s == MM_OK; ++i) s = pcg_iteration(ctx);
            ctx->capturing = false;
            cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
            if (s != MM_OK) return s;
            CK(e);
            CK(cudaGraphInstantiate(&ctx->graph_exec, g, 0));
            cudaGraphDestroy(g);
            ctx->graph_iters = n_iter;
        }
        CK(cudaGraphLaunch(ctx->graph_exec, ctx->stream));
    } else {
        for (int i = 0; i < n_iter; ++i) TRY(pcg_iteration(ctx));
    }
    return MM_OK;
}

static mm_status evaluate_state(mm_ctx* ctx, int32_t* done) {
    bool any = false;
    for (int i = 0; i < ctx->nrhs; ++i) any = any || ctx->h_st[i].active;
    int32_t d = 0;
    if (!any) TRY(finish_inner(ctx, &d, true));
    if (done) *done = d;
    return MM_OK;
}

mm_status mm_solve_step(mm_ctx* ctx, int32_t n_iter, int32_t* done) {
    if (!ctx) return MM_ERR_ARG;
    if (ctx->phase == PH_DONE) {
        if (done) *done = 1;
        return MM_OK;
    }
    if (ctx->phase != PH_INNER) return fail(ctx, MM_ERR_STATE, "mm_solve_begin first");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    TRY(launch_iters(ctx, n_iter));
    TRY(read_state(ctx));
    return evaluate_state(ctx, done);
}

mm_status mm_solve_launch(mm_ctx* ctx, int32_t n_iter) {
    if (!ctx) return MM_ERR_ARG;
    if (ctx->phase == PH_DONE) return MM_OK;
    if (ctx->phase != PH_INNER) return fail(ctx, MM_ERR_STATE, "mm_solve_begin first");
    if (n_iter < 0) return fail(ctx, MM_ERR_ARG, "n_iter must be >= 0");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    TRY(launch_iters(ctx, n_iter));
    if (!ctx->h_st_pinned || ctx->h_st_pinned_n < ctx->nrhs) {
        if (ctx->h_st_pinned) cudaFreeHost(ctx->h_st_pinned);
    if (ctx->reduce_host) cudaFreeHost(ctx->reduce_host);
        ctx->h_st_pinned = nullptr;
        CK(cudaMallocHost(reinterpret_cast<void**>(&ctx->h_st_pinned), ctx->nrhs * sizeof(RhsState)));
        ctx->h_st_pinned_n = ctx->nrhs;
    }
    if (!ctx->ev_state) CK(cudaEventCreateWithFlags(&ctx->ev_state, cudaEventDisableTiming));
    CK(cudaMemcpyAsync(ctx->h_st_pinned, ctx->s_st.p, ctx->nrhs * sizeof(RhsState), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CK(cudaEventRecord(ctx->ev_state, ctx->stream));
    ctx->launched = true;
    return MM_OK;
}

mm_status mm_solve_poll(mm_ctx* ctx, int32_t* ready, int32_t* done) {
    if (!ctx || !ready || !done) return MM_ERR_ARG;
    *ready = 0;
    *done = 0;
    if (ctx->phase == PH_DONE) {
        *ready = *done = 1;
        return MM_OK;
    }
    if (ctx->phase != PH_INNER || !ctx->launched) return fail(ctx, MM_ERR_STATE, "mm_solve_launch first");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    const cudaError_t q = cudaEventQuery(ctx->ev_state);
    if (q == cudaErrorNotReady) return MM_OK;
    CK(q);
    ctx->launched = false;
    ctx->h_st.assign(ctx->h_st_pinned, ctx->h_st_pinned + ctx->nrhs);
    *ready = 1;
    return evaluate_state(ctx, done);
}

mm_status mm_solve_end(mm_ctx* ctx, double* map_out, mm_solve_info* info, int mem) {
    if (!ctx) return MM_ERR_ARG;
    if (ctx->phase == PH_IDLE) return fail(ctx, MM_ERR_STATE, "mm_solve_begin first");
    DeviceScope dev_scope(ctx->device);
    CK(dev_scope.err);
    NvtxRange nvtx_range(__func__);
    if (ctx->phase == PH_INNER) {
        // stopped early by the caller: account for what ran, no further refinement
        TRY(read_state(ctx));
        int32_t d = 0;
        TRY(finish_inner(ctx, &d, false));
        for (int i = 0; i < ctx->nrhs; ++i)
            if (ctx->final_status[i] == 0 && !(ctx->true_res[i] <= ctx->tol)) ctx->final_status[i] = MM_ERR_NOT_CONVERGED;
    }
    CK(cudaEventRecord(ctx->ev1, ctx->stream));
    const int R = ctx->nrhs;
    const int64_t nv = (int64_t)R * ctx->n_pix;
    if (map_out) {
        if (mem == MM_HOST) {
            DevBuf o;
            CK(o.ensure(nv * 24));
            launch_map_out(ctx->s_xtot.as<V4<double>>(), o.as<double>(), nv, ctx->stream);
            CKL();
            CK(cudaMemcpyAsync(map_out, o.p, nv * 24, cudaMemcpyDeviceToHost, ctx->stream));
            CK(cudaStreamSynchronize(ctx->stream));
        } else {
            launch_map_out(ctx->s_xtot.as<V4<double>>(), map_out, nv, ctx->stream);
            CKL();
        }
    }
    CK(cudaStreamSynchronize(ctx->stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1);
    mm_status overall = MM_OK;
    for (int i = 0; i < R; ++i) {
        if (ctx->final_status[i] == MM_ERR_BREAKDOWN) overall = MM_ERR_BREAKDOWN;
        else if (ctx->final_status[i] == MM_ERR_NOT_CONVERGED && overall == MM_OK) overall = MM_ERR_NOT_CONVERGED;
        if (info) {
            info[i].iters = ctx->tot_iters[i];
            info[i].status = ctx->final_status[i];
            info[i].rel_res = ctx->rec_res[i];
            info[i].true_rel_res = ctx->true_res[i];
            info[i].t_solve_ms = ms;
            info[i].refinements = ctx->refinements[i];
            info[i].precond_used = i < (int)ctx->precond_used.size() ? ctx->precond_used[i] : (int32_t)ctx->precond;
        }
    }
    ctx->phase = PH_IDLE;
    destroy_graph(ctx);
    if (overall == MM_ERR_NOT_CONVERGED) ctx->err = "at least one right-hand side did not converge";
    if (overall == MM_ERR_BREAKDOWN) ctx->err = "PCG breakdown (p^T A p <= 0 or NaN)";
    return overall;
}

mm_status mm_solve(mm_ctx* ctx, const void* tod, double* map_out, int32_t nrhs, const int64_t* rhs_len,
                   mm_precond precond, double tol, int32_t max_iter, mm_solve_info* info, int mem) {
    TRY(mm_solve_begin(ctx, tod, nrhs, rhs_len, precond, tol, max_iter, mem));
    int32_t done = 0;
    while (!done) TRY(mm_solve_step(ctx, ctx->opt_check_every, &done));
    return mm_solve_end(ctx, map_out, info, mem);
}

mm_status mm_set_option(mm_ctx* ctx, const char* name, double value) {
    if (!ctx || !name) return MM_ERR_ARG;
    const std::string n(name);
    const int v = (int)value;
    if (n == "filter") {
        if (v < 0 || v > 2) return fail(ctx, MM_ERR_ARG, "filter must be 0, 1 or 2");
        ctx->opt_filter = v;
    } else if (n == "fft_log2") {
        if (v != 0 && (v < 6 || v > 14)) return fail(ctx, MM_ERR_ARG, "fft_log2 must be 0 or in [6, 14]");
        ctx->opt_fft_log2 = v;
    } else if (n == "fft_len") {
        FftPasses fp;
        if (v != 0 && (v < 64 || !fft_passes(v, &fp))) return fail(ctx, MM_ERR_ARG, "fft_len must be 0 or 2^a 3^b >= 64, b <= 2");
        ctx->opt_fft_len = v;
    } else if (n == "direct_tile") {
        if (v < 32 || v > 65536) return fail(ctx, MM_ERR_ARG, "direct_tile must lie in [32, 65536]");
        ctx->opt_direct_tile = v;
    } else if (n == "check_every") {
        if (v < 1 || v > 100000) return fail(ctx, MM_ERR_ARG, "check_every must be >= 1");
        ctx->opt_check_every = v;
    } else if (n == "graphs") {
        ctx->opt_graphs = v ? 1 : 0;
    } else if (n == "autotune") {
        ctx->opt_autotune = v ? 1 : 0;
    } else if (n == "half_transform") {
        ctx->opt_half = v ? 1 : 0;
    } else if (n == "coarse_prefix") {
        ctx->opt_coarse_prefix = v ? 1 : 0;
    } else if (n == "coarse_fallback") {
        ctx->opt_coarse_fallback = v ? 1 : 0;
    } else if (n == "tc_coarse") {
        if (ctx->phase != PH_IDLE) return fail(ctx, MM_ERR_STATE, "tc_coarse: a solve is in progress");
        if (v < 0 || v > 2) return fail(ctx, MM_ERR_ARG, "tc_coarse must be 0, 1 or 2");
        ctx->opt_tc_coarse = v;
    } else if (n == "inner_tol") {
        if (!(value > 0.0) || value > 1e-2) return fail(ctx, MM_ERR_ARG, "inner_tol must lie in (0, 1e-2]");
        ctx->opt_inner_tol = value;
    } else if (n == "apply_precision") {
        if (v < 0 || v > 2) return fail(ctx, MM_ERR_ARG, "apply_precision must be 0, 1 or 2");
        ctx->opt_apply_prec = v;
    } else if (n == "fp64_products") {
        if (v != 1 && v != 2) return fail(ctx, MM_ERR_ARG, "fp64_products must be 1 (float64) or 2 (double-float)");
        if (ctx->phase == PH_INNER) return fail(ctx, MM_ERR_STATE, "fp64_products cannot change during a solve");
        ctx->p64 = v;
    } else if (n == "harvest") {
        if (v < 0 || v > 4096) return fail(ctx, MM_ERR_ARG, "harvest must lie in [0, 4096]");
        ctx->opt_harvest = v;
    } else if (n == "time_filter") {
        ctx->opt_time_filter = v ? 1 : 0;
        ctx->fev_used = 0;
    } else {
        return fail(ctx, MM_ERR_ARG, "unknown option " + n);
    }
    return MM_OK;
}

mm_status mm_get_option(mm_ctx* ctx, const char* name, double* value) {
    if (!ctx || !name || !value) return MM_ERR_ARG;
    const std::string n(name);
    if (n == "filter") *value = ctx->opt_filter;
    else if (n == "fft_log2") *value = ctx->opt_fft_log2;
    else if (n == "fft_len") *value = ctx->opt_fft_len;
    else if (n == "direct_tile") *value = ctx->opt_direct_tile;
    else if (n == "check_every") *value = ctx->opt_check_every;
    else if (n == "graphs") *value = ctx->opt_graphs;
    else if (n == "last_apply_ms") *value = ctx->last_apply_ms;
    else if (n == "kernel_launches") *value = (double)launches_total();
    else if (n == "time_filter") *value = ctx->opt_time_filter;
    else if (n == "autotune") *value = ctx->opt_autotune;
    else if (n == "half_transform") *value = ctx->opt_half;
    else if (n == "coarse_prefix") *value = ctx->opt_coarse_prefix;
    else if (n == "coarse_rank_min") *value = ctx->coarse_rank_min;
    else if (n == "coarse_fallback") *value = ctx->opt_coarse_fallback;
    else if (n == "tc_coarse") *value = ctx->opt_tc_coarse;
    else if (n == "coarse_len") *value = (double)ctx->coarse_len;
    else if (n == "harvest") *value = ctx->opt_harvest;
    else if (n == "fp64_products") *value = ctx->p64;
    else if (n == "apply_precision") *value = ctx->opt_apply_prec;
    else if (n == "inner_tol") *value = ctx->opt_inner_tol;
    else if (n == "harvested") *value = ctx->harvest_count;
    else if (n == "filter_ms" || n == "filter_launches") {
        // total device time of the filter launches timed since the last read; resets the record
        CK(cudaStreamSynchronize(ctx->stream));
        double tot = 0.0;
        for (size_t i = 0; i < ctx->fev_used; ++i) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, ctx->fev[i].first, ctx->fev[i].second));
            tot += ms;
        }
        *value = n == "filter_ms" ? tot : (double)ctx->fev_used;
        if (n == "filter_ms") ctx->fev_used = 0;
    }
    else if (n == "plan_fft_log2") {
        Plan* p = nullptr;
        if (!ctx->have_pointing) return fail(ctx, MM_ERR_STATE, "no pointing");
        TRY(get_plan(ctx, op_prec(ctx), 1, {}, &p));
        *value = p->variant == 2 ? p->logL : 0;
    } else if (n == "plan_fft_len" || n == "plan_whole") {
        Plan* p = nullptr;
        if (!ctx->have_pointing) return fail(ctx, MM_ERR_STATE, "no pointing");
        TRY(get_plan(ctx, op_prec(ctx), 1, {}, &p));
        *value = n == "plan_whole" ? p->whole : (p->variant == 2 ? p->L : 0);
    } else if (n == "device_bytes") {
        size_t f = 0, t = 0;
        cudaMemGetInfo(&f, &t);
        *value = (double)(t - f);
    } else return fail(ctx, MM_ERR_ARG, "unknown option " + n);
    return MM_OK;
}

int64_t mm_estimate_bytes(int64_t n_samples, int32_t n_pix, int32_t n_bands, int32_t half_bw, int32_t nrhs,
                          int32_t m_max, int32_t k, mm_precision prec) {
    const int64_t esz = prec == MM_FP32_MIXED ? 4 : 8;
    int64_t b = n_samples * (4 + 4 + 16);              // pix, psi, float64 weights
    if (prec == MM_FP32_MIXED) b += n_samples * 16;    // double-float weights
    b += (int64_t)nrhs * n_samples * esz;              // timelines
    b += (int64_t)n_pix * 32 * (12 + 2 * (int64_t)nrhs * 6);  // maps and PCG state
    b += (int64_t)(m_max + 1) * n_pix * 32;            // Arnoldi basis
    b += (int64_t)2 * k * n_pix * 32;                  // Z, AZ
    b += (int64_t)n_bands * (int64_t)16384 * 12;       // spectra
    b += (int64_t)n_pix * 7 * 8 * std::max(1, nrhs);   // M_BD sums
    b += n_samples / 64 * 40 * std::max(1, nrhs);      // segment lists
    (void)half_bw;
    return b;
}

}  // extern "C"
