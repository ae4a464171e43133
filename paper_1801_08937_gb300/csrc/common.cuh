// Shared types and launcher declarations of the map-making library.
//
// Layouts in device memory
//   pointing   pix int32[N], psi float32[N] (and, for float64 products, the
//              weights (cos 2psi, sin 2psi) as double2[N] precomputed once)
//   maps       [nrhs][n_pix] of 4-wide vectors (I, Q, U, 0); float4 for the
//              float32 operator, V4<double> (32-byte aligned) elsewhere.  The
//              fourth lane keeps every pixel one aligned vector load.
//   segments   the timeline is cut into output segments inside stationary
//              blocks; each CTA of the filter kernels processes one pair of
//              segments (see Seg).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

namespace mm {

// Largest coarse space (number of deflation vectors k) the M_2l kernels hold.
constexpr int MM_K_MAX = 512;

// Kernels launched by this library since load (every launcher adds its count).
long long launches_total();
void count_launches(int n);

// Raises a kernel's dynamic shared-memory configuration to at least sm bytes,
// never lowering it: set(sm) runs once per larger size, under a lock, so
// contexts set up on several host threads cannot leave a kernel configured
// below a size another thread already launches with.
std::mutex& smem_config_mutex();
template <typename F>
inline void raise_smem_once(std::atomic<size_t>& configured, size_t sm, F&& set) {
    if (sm <= configured.load(std::memory_order_acquire)) return;
    std::lock_guard<std::mutex> lock(smem_config_mutex());
    if (sm <= configured.load(std::memory_order_relaxed)) return;
    set(sm);
    configured.store(sm, std::memory_order_release);
}

// Makes `device` current for one entry point and gives the caller back the
// device that was current before, so a call on this library's device never
// leaves a caller working on another device switched over.
struct DeviceScope {
    int prev = -1;
    int dev;
    cudaError_t err;
    explicit DeviceScope(int device) : dev(device) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        err = (prev == device) ? cudaSuccess : cudaSetDevice(device);
    }
    ~DeviceScope() {
        if (prev >= 0 && prev != dev) cudaSetDevice(prev);
    }
    DeviceScope(const DeviceScope&) = delete;
    DeviceScope& operator=(const DeviceScope&) = delete;
};

template <typename T> struct __align__(sizeof(T) * 4) V4 { T x, y, z, w; };
template <typename T> struct __align__(sizeof(T) * 2) C2 { T x, y; };

// One output segment of one stationary block for one right-hand side.
//   outputs  t in [out0, out0 + n_out)
//   inputs   t in [out0 - lambda, out0 + n_out + lambda) clipped to [lo, hi),
//            the block's active range for this right-hand side.
// Segments are stored in pairs; a pair shares one band (one filter) so two
// real timelines travel as the real and imaginary parts of one complex FFT.
// n_out == 0 marks an empty slot.
struct Seg {
    int64_t out0;
    int64_t lo, hi;
    int32_t rhs;
    int32_t n_out;
    int32_t band;
    int32_t shift;   // left halo in the transform buffer: lambda, or 0 for a whole block
};

// Mixed-radix FFT plan: L = product of radix[p]; pass p works on spans of
// span[p] points (span[0] = L, span[p+1] = span[p] / radix[p]).
struct FftPasses {
    int L, npass;
    int radix[8];
    int span[8];
};

// Per-right-hand-side PCG scalars kept on the device (float64).
struct RhsState {
    double rz;       // r^T z of the current iterate
    double pq;       // p^T A p
    double alpha, beta;
    double bnorm;    // ||b||
    double relres;   // ||r_k|| / ||b||
    double tol;
    int32_t active;  // 1 while iterating
    int32_t iters;
    int32_t status;  // 0 ok/running, 5 not converged, 6 breakdown
    int32_t max_iter;
};

// ---------------- filter (A x, b) ----------------
struct FilterArgs {
    const Seg* segs;       // [2 * n_work] (pairs), or [n_work] for half-length real transforms
    int n_work;
    const int32_t* pix;
    const float* psi;
    const double2* cs64;   // float64 weights, may be null for float32
    const float4* csdf;    // double-float weights (hi, lo of cos 2psi; hi, lo of sin 2psi)
    const void* src;       // maps [nrhs][n_pix] (V4<T>) or TOD [nrhs][n_samples] (T)
    int64_t n_samples;
    void* dst;             // accumulators [nrhs][n_pix] (V4<T>)
    int n_pix;
    const void* H;         // FFT: [n_bands][L] real spectrum (digit-reversed, 1/L folded in);
                           // half: [n_bands][L/2 + 1] pair coefficients (alpha_k, alpha_{L-k}, beta_k)
    const void* tw;        // FFT: [L] twiddles exp(-2 pi i e / L)
    const uint32_t* pairs; // half: [L/2 + 1] digit-reversed positions of k (low 16 bits) and L - k
    const uint32_t* items; // half, fused last pass: [L/(2R) + 1] butterfly c (low 16 bits) and its partner c'
    const void* Hi;        // half, fused last pass: [n_bands][items][R] coefficients (alpha_k, alpha_{L-k}, beta_k)
    const void* twp;       // half: per-pass twiddles W_S^(j q), pass by pass, [q - 1][j] within a pass; may be null
    int half;              // 1: one whole block per CTA as L = N/2 complex points
    const void* band;      // direct: [n_bands][lambda+1]
    int L, logL, lam, V;
    FftPasses fp;
    const RhsState* state; // may be null: all right-hand sides active
    int tod_is_float;      // src TOD element type when from_tod (1: float, 0: double)
    const void* xmap;      // from_tod, float64 / double-float only: map x (V4<T>) whose P x is subtracted
                           // from the timeline, giving the residual P^T W (d - P x) = b - A x; may be null
};

// Template filter F = F_B W^-1 F_G W^-1 F_B (white W = w_b I per block):
// Legendre polynomials of each subscan and azimuth bins of each block.
struct TmplArgs {
    const int64_t* block_off;  // [n_blocks + 1]
    int n_blocks;
    int64_t max_block;         // longest block (shared memory size)
    const double* w_block;     // [n_blocks] white weight of each block
    const int64_t* sub_off;    // [n_sub + 1] subscans, each inside one block
    const int32_t* blk_sub;    // [n_blocks + 1] first subscan of each block
    const double* ginv;        // [n_sub][4][4] inverse Gram matrix of the subscan's Legendre columns
    int order;                 // polynomial order K (-1: no polynomial filter)
    const int32_t* az;         // [N] azimuth bin of each sample (-1: none); null: no ground filter
    int n_bins;
    int stokes;                // 0: rows (1, cos 2psi, sin 2psi); 1: (0, cos, sin), d^-; 2: (1, 0, 0), d^+
};
// prec: 0 float32, 1 float64, 2 double-float
void launch_filter_tmpl(const FilterArgs& a, const TmplArgs& t, int nrhs, int prec, bool from_tod, cudaStream_t s);
size_t tmpl_smem_bytes(int64_t max_block, int n_bins, bool f64);

// T = float or double; from_tod selects b = P^T W d (src is a TOD).
void launch_filter_fft_f32(const FilterArgs& a, bool from_tod, cudaStream_t s);
void launch_filter_fft_f64(const FilterArgs& a, bool from_tod, cudaStream_t s);
void launch_filter_direct_f32(const FilterArgs& a, bool from_tod, cudaStream_t s);
void launch_filter_direct_f64(const FilterArgs& a, bool from_tod, cudaStream_t s);
// Double-float (float32 pairs) variants: maps V4<df> in, float64 accumulators out.
void launch_filter_fft_df(const FilterArgs& a, bool from_tod, cudaStream_t s);
void launch_filter_direct_df(const FilterArgs& a, bool from_tod, cudaStream_t s);
void launch_weights_df(const double2* cs, float4* out, int64_t n, cudaStream_t s);
void launch_map_to_df(const V4<double>* src, void* dst, int64_t n, cudaStream_t s);
size_t fft_smem_bytes(int L, bool f64);
size_t direct_smem_bytes(int V, int lam, bool f64);
// H = DIF(h) for each band in float64 through global scratch; h [n_bands][L].
void launch_fft_spectrum(const double* h, double* H_out, double2* work, const double2* tw,
                         int n_bands, const FftPasses& fp, cudaStream_t s);
void launch_weights64(const float* psi, double2* cs, int64_t n, cudaStream_t s);

// ---------------- vectors, preconditioners, reductions ----------------
void launch_map_in(const double* src3, V4<double>* dst4, int64_t n_vec, cudaStream_t s);
void launch_map_out(const V4<double>* src4, double* dst3, int64_t n_vec, cudaStream_t s);
void launch_to_f32(const V4<double>* src, V4<float>* dst, int64_t n, cudaStream_t s);
void launch_from_f32(const V4<float>* src, V4<double>* dst, int64_t n, cudaStream_t s);
void launch_zero(void* p, size_t bytes, cudaStream_t s);

// M_BD build: 6 sums + hits per pixel; then flagging and inversion.
void launch_bd_accumulate(const int32_t* pix, const float* psi, const int64_t* block_off,
                          const int32_t* block_band, const double* band, int lam1, int n_blocks,
                          int64_t t_cap_per_det, int64_t n_t, const int64_t* rhs_len, int nrhs,
                          double* sums /*[nrhs][n_pix][7]*/, int n_pix, cudaStream_t s);
void launch_bd_invert(const double* sums, double* bd /*[nrhs][n_pix][6]*/, uint8_t* good,
                      int* n_dropped, int n_pix, int nrhs, double rcond_min, int set_good,
                      cudaStream_t s, int stokes = 0);
void launch_flag_samples(int32_t* pix, const uint8_t* good, int64_t n, cudaStream_t s);
void launch_bd_apply(const double* bd, int bd_per_rhs, const V4<double>* x, V4<double>* y,
                     int n_pix, int nrhs, cudaStream_t s);

// PCG building blocks (all nrhs at once; grid.y = rhs).
struct PcgArgs {
    int n_pix, nrhs;
    RhsState* st;
    V4<double>* x; V4<double>* r; V4<double>* z; V4<double>* p;
    const V4<double>* q64;   // A p in float64 (FP64 operator)
    const V4<float>* q32;    // A p in float32 (FP32 operator)
    void* src;               // gather source for the next product (V4<T>)
    int src_f32;             // operator input: 0 float64, 1 float32, 2 double-float
    void* qacc;              // accumulator to clear (V4<T>)
    const double* bd; int bd_per_rhs;
    // two-level
    int k;
    const V4<double>* Z; const V4<double>* AZ; const double* Einv;
    // float32 copies of Z and AZ (mixed precision, one coarse space for all right-hand sides):
    // the coarse sums of M_2l in float32 arithmetic; null: float64
    const V4<float>* Z32; const V4<float>* AZ32;
    double* u;               // [nrhs][k]
    double* partial;         // reduction scratch
    unsigned* counter;       // [nrhs]
    double* hist;            // [nrhs][hist_stride]
    int hist_stride;
    int grid_x;
    // per right-hand-side coarse operators (0 strides: shared)
    int64_t az_stride;       // in V4<double> units
    int einv_stride;         // in doubles
    // Lanczos harvest from an M_BD run (null when off)
    double* ahist;           // [nrhs][hist_stride] alpha_j
    double* bhist;           // [nrhs][hist_stride] beta_j
    V4<double>* harvest;     // [harvest_m][n_pix] z_j / sqrt(r_j^T z_j) of right-hand side 0
    int harvest_m;
};
void launch_pcg_init(const PcgArgs& a, const V4<double>* b, cudaStream_t s);
void launch_pcg_src(const PcgArgs& a, int first, cudaStream_t s);
void launch_pcg_pq(const PcgArgs& a, cudaStream_t s);
void launch_pcg_update(const PcgArgs& a, int two_level, cudaStream_t s);
void launch_precond_bd_dot(const PcgArgs& a, int finalize_beta, cudaStream_t s);
void launch_m2l_ztr(const PcgArgs& a, const V4<double>* v, cudaStream_t s);
void launch_m2l_apply(const PcgArgs& a, const V4<double>* v, V4<double>* out, int finalize_beta,
                      cudaStream_t s);
void launch_harvest(const PcgArgs& a, cudaStream_t s);
// M_2l on the tensor cores (tcgen05) for 8 <= nrhs <= 128 right-hand sides, k <= 64, a shared coarse space
bool m2l_tc_eligible(const PcgArgs& a);
bool m2l_tc_pays(const PcgArgs& a);
size_t m2l_tc_scratch_doubles(int n_pix, int nrhs, int k);
void launch_m2l_tc(const PcgArgs& a, const V4<double>* v, V4<double>* out, int finalize_beta, double* scratch,
                   cudaStream_t s);
cudaError_t m2l_tc_fault_take(cudaStream_t s, int* fault);

// Tall-skinny float64 products over vectors of n doubles (n = 4 n_pix).
// h[i] = sum_n X[i][n] v[n] for i < m  (deterministic two-phase reduction)
void launch_multidot(const double* X, int64_t ldx, int m, const double* v, int64_t n,
                     double* h, double* partial, unsigned* counter, int grid_x, cudaStream_t s);
// v[n] -= sum_i X[i][n] h[i]
void launch_sub_combo(const double* X, int64_t ldx, int m, const double* h, double* v, int64_t n,
                      cudaStream_t s);
// Y[c][n] = sum_i X[i][n] C[i*kc + c] for c < kc
void launch_combo(const double* X, int64_t ldx, int m, const double* C, int kc, double* Y,
                  int64_t ldy, int64_t n, cudaStream_t s);
// G[j*mx + i] = sum_n X[i][n] Y[j][n]
void launch_gram(const double* X, int mx, const double* Y, int my, int64_t ld, int64_t n, double* G,
                 double* partial, unsigned* counter, int grid_x, cudaStream_t s);
void launch_scale_host(double* v, int64_t n, double factor, cudaStream_t s);
void launch_residual(const V4<double>* b, const V4<double>* q, V4<double>* r_out, double* norms, int n_pix,
                     int nrhs, double* partial, unsigned* counter, int grid_x, cudaStream_t s);
void launch_axpy_masked(double* y, const double* x, int64_t n_per, int nrhs, const int32_t* mask,
                        cudaStream_t s);

// Read-only view of a context's preconditioner state (defined with the context).
struct CoarseView {
    int device;
    cudaStream_t stream;
    int n_pix, k, grid_x;
    bool have_bd;
    const double* bd;
    const V4<double>* Z;
    const V4<double>* AZ;
    const double* Einv;
};

// ---------------- host linear algebra ----------------
// Eigenvalues of a real upper Hessenberg m x m matrix (row-major) by
// double-shift QR; near-real values come back real.  False on failure.
bool host_hess_eigvals(const std::vector<double>& H, int m, std::vector<double>& wr, std::vector<double>& wi);
// Right eigenvector (unit norm, largest component real positive) of the
// Hessenberg H for the eigenvalue wr + i wi, by inverse iteration; hnorm =
// max |H_ij| when the caller has it (negative: computed here).
bool host_hess_eigvec(const std::vector<double>& H, int m, double wr, double wi, std::vector<double>& vr,
                      std::vector<double>& vi, double hnorm = -1.0);
// Eigenvalues (ascending order not guaranteed) of the symmetric tridiagonal
// matrix with diagonal d[n] and off-diagonal e[n-1]; false on failure.
bool host_tridiag_eigvals(const std::vector<double>& d, const std::vector<double>& e, int n,
                          std::vector<double>& w);
// Unit eigenvector (largest component positive) of that matrix for the eigenvalue lam.
bool host_tridiag_eigvec(const std::vector<double>& d, const std::vector<double>& e, int n, double lam,
                         std::vector<double>& v);
// Ritz selection (Appendix A, Eq. ritz) from the Arnoldi H_m or the
// symmetric tridiagonal Lanczos T_m: the k smallest Ritz pairs by real part
// (k <= 0: those below eps_lambda, at most kmax), complex pairs as real and imaginary
// parts, null values (|theta| <= 1e-10 max |theta|) skipped.  C [m][ksel]
// row-major holds the Ritz vectors in the Krylov basis, vals their values.
// Returns 0, 1 if an eigen-solve failed, 2 if nothing was selected.
int host_ritz_hess(const std::vector<double>& H, int m, int k, int kmax, double eps_lambda, std::vector<double>& C,
                   std::vector<double>& vals);
int host_ritz_tridiag(const std::vector<double>& d, const std::vector<double>& e, int m, int k, int kmax,
                      double eps_lambda, std::vector<double>& C, std::vector<double>& vals);
// The Lanczos matrix T_m of a PCG run with M_BD from its coefficients
// alpha_j, beta_j (j < m): diagonal d[m], off-diagonal e[m-1].
void host_lanczos_tridiag(const std::vector<double>& alpha, const std::vector<double>& beta, int m,
                          std::vector<double>& d, std::vector<double>& e);
// Layout of the polynomial templates (Sect. 4.1): checks that subscan
// offsets so[0..ns] increase, that every subscan lies inside one block and
// that block boundaries are subscan boundaries; blk_sub[b] = first subscan of
// block b (blk_sub[n_blocks] = ns); ginv[s][4][4] = (B^T B)^-1 of subscan s's
// Legendre columns P_0..P_min(K, m-1) (poly_order K < 0: zeros).  False with
// err set on a bad layout.
bool host_template_layout(const std::vector<int64_t>& block_off, const std::vector<int64_t>& so, int poly_order,
                          std::vector<int32_t>& blk_sub, std::vector<double>& ginv, std::string& err);
// Lower Cholesky factor in place (row-major n x n); false if not SPD.
bool host_cholesky(std::vector<double>& A, int n);
// Inverse of an SPD matrix from its Cholesky factor.
void host_spd_inverse_from_chol(const std::vector<double>& L, int n, std::vector<double>& inv);
int host_pivoted_spd_inverse(const std::vector<double>& E, int n, double rel_tol, std::vector<double>& inv);
// Inverse of an upper-triangular matrix R (row-major).
void host_upper_inverse(const std::vector<double>& R, int n, std::vector<double>& Rinv);

}  // namespace mm
