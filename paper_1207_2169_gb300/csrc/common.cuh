// Shared helpers of the CUDA library: error plumbing, the handle layout and launch prototypes.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gwas.h"

namespace gw {

// Thread-local message behind gwas_last_error().
void set_error(const char* fmt, ...);

struct Fail {
  gwas_status st;
};

#define GW_CUDA(call)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      ::gw::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,     \
                      __LINE__);                                                           \
      throw ::gw::Fail{e_ == cudaErrorMemoryAllocation ? GWAS_ERR_OOM : GWAS_ERR_CUDA};    \
    }                                                                                      \
  } while (0)

#define GW_CHECK_LAUNCH() GW_CUDA(cudaGetLastError())

#define GW_REQUIRE(cond, status, ...)                                                      \
  do {                                                                                     \
    if (!(cond)) {                                                                         \
      ::gw::set_error(__VA_ARGS__);                                                        \
      throw ::gw::Fail{status};                                                            \
    }                                                                                      \
  } while (0)

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }
inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// Per-stage device time of a handle's scans (gwas_stage_timing): CUDA events recorded on the
// launching stream around each stage's kernels, read back by gwas_stage_times.
struct StageTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;        // created on first use, reused after each read
  std::vector<int> stage;               // stage of each recorded (start, end) pair
  size_t used = 0;                      // events in use: 2 per recorded pair
  cudaEvent_t begin(cudaStream_t s, int st) {
    if (!on) return nullptr;
    while (pool.size() < used + 2) {
      cudaEvent_t e;
      GW_CUDA(cudaEventCreate(&e));
      pool.push_back(e);
    }
    GW_CUDA(cudaEventRecord(pool[used], s));
    stage.push_back(st);
    used += 2;
    return pool[used - 1];
  }
  void end(cudaStream_t s, cudaEvent_t e) {
    if (e) GW_CUDA(cudaEventRecord(e, s));
  }
  void destroy() {
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
    stage.clear();
    used = 0;
  }
};

// Stages a timer tells apart (the GWAS_STAGE_* values of gwas.h).
enum { STAGE_PACK = 0, STAGE_CENTRES = 1, STAGE_CHOL = 2, STAGE_ROT = 3, STAGE_SQ = 4,
       STAGE_AC = 5, STAGE_SIMT = 6, STAGE_COUNT = 8 };

// Device flags word layout (int32 array in the handle).
enum { FLAG_GENOTYPE = 0, FLAG_SINGULAR = 1, FLAG_NOT_SPD = 2, FLAG_ROTATIONS = 3,
       FLAG_TIMEOUT = 4, FLAG_STL_SINGULAR = 5, FLAG_COUNT = 8 };

// ------------------------------------------------------------------------------------------
// Setup kernels (FP64), setup_f64.cu
// ------------------------------------------------------------------------------------------
// C = alpha * op(A) * op(B) + beta * C with arbitrary element strides:
//   A(i,k) = A[i*sai + k*sak], B(k,j) = B[k*sbk + j*sbj], C(i,j) = C[i*sci + j*scj].
// lower_only: skip 64x64 tiles of C that lie strictly above the diagonal.
// b_tri: B is upper triangular (> 0: B(k,j) = 0 for k > j) or lower triangular (< 0: B(k,j) = 0
// for k < j), and only the k range that can be non-zero is summed; 0 for a full B.
void gemm_f64(cudaStream_t s, int M, int N, int K, double alpha, const double* A, int64_t sai,
              int64_t sak, const double* B, int64_t sbk, int64_t sbj, double beta, double* C,
              int64_t sci, int64_t scj, bool lower_only = false, int b_tri = 0);
// A (n x n, column-major, lower) := M = s2 (h2 Phi + (1-h2) I).
void form_M(cudaStream_t s, int n, const double* Phi, double h2, double s2, double* A);
// In-place lower Cholesky of A (column-major, ld n); upper part zeroed.  Sets flags[NOT_SPD].
void cholesky(cudaStream_t s, int n, double* A, int* flags);
// Linv (row-major, n x n, zeros above the diagonal) := L^-1 for lower L (column-major).
void tri_inverse(cudaStream_t s, int n, const double* L, double* Linv, double* work);
// One-sided Jacobi eigendecomposition of SPD Phi: Zt (row r = eigenvector r), w.  Returns
// sweeps used, or -1 when not converged within max_sweeps.
int jacobi_eig(cudaStream_t s, int n, const double* Phi, double* Zt, double* w, double* U,
               int* flags, int max_sweeps);
// The setup's eigensolver (eigh_f64.cu): Householder tridiagonalisation, multisection, inverse
// iteration, Cholesky QR and back-transformation (Zt row r = eigenvector r, w eigenvalues);
// falls back to jacobi_eig if the orthonormalisation fails.  Returns >= 0 on success, -1 if
// neither converged.  eigh_tridiag alone returns 0, or -1 without a result.
int eigh_tridiag(cudaStream_t s, int n, const double* Phi, double* Zt, double* w);
int eigh_f64(cudaStream_t s, int n, const double* Phi, double* Zt, double* w, double* U,
             int* flags);

// 1 / e in FP64 for 1e-30 <= |e| <= 1e30: an FP32 reciprocal as the seed (relative error
// ~2^-22), then two Newton-Raphson steps x <- x (2 - e x), each squaring the relative error
// (2^-44, then below FP64 rounding).  Four FMAs instead of an FP64 division, whose throughput
// on this GPU's FP64 units would dominate the loops that use it.
__device__ __forceinline__ double recip_f64(double e) {
  double x = (double)__frcp_rn((float)e);
  x = fma(x, fma(-e, x, 1.0), x);
  x = fma(x, fma(-e, x, 1.0), x);
  return x;
}

// Step 1 (estimate.cu): per trait j, the (h2, s2) maximising the ML (method 0) or REML (1)
// criterion of the reduced model, from the eigenvalues w of Phi and the rotated covariates
// XLt (q x n, row k = Z^T X_L[:, k]) and traits Yt (t x n, row j = Z^T y_j).  Writes h2, s2
// and the criterion (t each, device).  tables: device scratch of estimate_table_doubles(n)
// doubles.  Sets flags[FLAG_STL_SINGULAR] if X_L^T H^-1 X_L is singular.
void estimate_traits(cudaStream_t s, int n, int q, int t, int method, const double* w,
                     const double* XLt, const double* Yt, double* tables, double* h2, double* s2,
                     double* crit, int* flags);
size_t estimate_table_doubles(int n);

// Per-trait null-model precompute shared by both algorithms (bordered-system top block).
//   XLw (q x n, row k = k-th whitened covariate), yw (n) for each trait, weights d (n; all
//   ones for CHOL, D_j for EIG).  Produces P = S_TL^-1 (q x q), b0 = P X_L^T D y, and the
//   weighted residual rw = D (y - X_L b0) scaled for the scan (see trait_pack in setup_f64.cu).
struct TraitPackArgs {
  int n, q, t;
  const double* XLw;   // q x n (shared by all traits; EIG: Z^T X_L; CHOL: per trait)
  int64_t xlw_trait_stride;
  const double* yw;    // t x n (EIG: Z^T Y; CHOL: L_j^-1 y_j)
  const double* d;     // t x n weights or NULL (all ones)
  double* P;           // t x q x q
  double* b0;          // t x q
  double* rw;          // t x n: weighted residual d * (yw - XLw^T b0)
  int* flags;
};
void trait_pack(cudaStream_t s, const TraitPackArgs& a);
// EIG weights d_j[r] = 1 / (s2_j (h2_j w_r + 1 - h2_j)), t x n.
void eig_weights(cudaStream_t s, int n, int t, const double* w, const double* h2,
                 const double* s2, double* d, int* flags);
// EIG B-operand planes, K-major: planes[(j*(q+2)+c)*ldp + r] = d_j[r]*XLt[c][r] (c<q),
// rw_j[r] (c=q; already weighted), d_j[r] (c=q+1).  Zero for r >= n.
void eig_planes_f64(cudaStream_t s, int n, int q, int t, int ldp, const double* XLt,
                    const double* d, const double* rw, double* planes);

// lam_max(M) / lam_min(M) of SPD M = L L^T, each extreme eigenvalue by `iters` power
// iterations (M v = L L^T v; M^-1 v = L^-T L^-1 v) from a start with every component, so an
// estimate from below of each (and of the ratio).  L: column-major lower Cholesky factor, Linv:
// row-major lower inverse, both n x n.  work: 3 n + 1 doubles.  Synchronises s.
double condition_estimate(cudaStream_t s, int n, const double* L, const double* Linv,
                          double* work, int iters);

// Conversions.
void convert_f64_to_f32(cudaStream_t s, const double* x, float* y, int64_t count);
// hi = bf16(x), lo = bf16(x - hi) and, when lo2 is not NULL, lo2 = bf16(x - hi - lo), for a
// rows x cols row-major matrix with leading dims.
void split_bf16(cudaStream_t s, const double* x, int rows, int cols, int64_t ldx,
                __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ldo, __nv_bfloat16* lo2 = nullptr);
// As split_bf16, with output row r taken from input row (r / gout) * gin + r % gout + off
// (selects `gout` of every `gin` input rows, starting at `off`).
void split_bf16_rows(cudaStream_t s, const double* x, int rows, int cols, int64_t ldx, int gin,
                     int gout, int off, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ldo,
                     __nv_bfloat16* lo2 = nullptr);

// The FP16 hi + E4M3 lo split (SPLIT_FP8) of the rows of a rows x cols row-major matrix: row r
// is scaled by rscale[r] (a power of two, device array), hi = fp16(v), lo = e4m3(v - hi) with v
// the scaled value; both store their columns in e4m3_k_slot order within each aligned group of
// 16 (the order the tensor-core converters produce genotypes in).  Columns cols .. ldo-1 are
// zero.
// rowmax_abs writes max |x[r][c]| of each row into out[r].  e4m3_row_sums writes, per row r of
// the lo matrix, the sum of its values over all ldo columns into out[r] (FP32).
void rowmax_abs(cudaStream_t s, const double* x, int rows, int cols, int64_t ldx, double* out);
void split_f16_e4m3(cudaStream_t s, const double* x, int rows, int cols, int64_t ldx,
                    const double* rscale, __half* hi, uint8_t* lo, int64_t ldo);
void e4m3_row_sums(cudaStream_t s, const uint8_t* lo, int rows, int64_t ldo, float* out);
// w[c] = sum over r < rows of ls[r] (hi[r][c] + lo[r][c]) for the natural columns c < cols of the
// split (hi and lo in their stored order), in FP64.
void e4m3_weighted_col_sums(cudaStream_t s, const __half* hi, const uint8_t* lo, int rows,
                            int64_t ldo, int cols, const float* ls, double* w);

// ------------------------------------------------------------------------------------------
// Genetic models: the block X_R,i a SNP contributes to X_i = [X_L | X_R,i] has pr columns
// (1 or 2).  The kernels build the block in a working basis, column k taking the value
// code[k][x] for the hard call x = 0, 1, 2, and report the model's own coefficients
// b_model = tm b_work (tm: pr x pr, identity unless the model's columns are a different basis
// of the same span).  The fit, b_L and the joint Wald statistic do not depend on the basis.
// ------------------------------------------------------------------------------------------
struct GeneticModel {
  int pr = 1;
  int8_t code[2][3] = {{0, 1, 2}, {0, 0, 0}};
  float tm[2][2] = {{1.f, 0.f}, {0.f, 1.f}};
  // column k's coding as bytes cd(0) | cd(1) << 8 | cd(2) << 16 (the tensor-core converters' form)
  uint32_t code_word(int k) const {
    return (uint32_t)(uint8_t)code[k][0] | (uint32_t)(uint8_t)code[k][1] << 8 |
           (uint32_t)(uint8_t)code[k][2] << 16;
  }
};
// GWAS_MODEL_* -> its columns (throws Fail{GWAS_ERR_ARG} for an unknown model).
GeneticModel genetic_model(int model);

// ------------------------------------------------------------------------------------------
// Scan kernels, scan_simt.cu (plain FP64 / FP32 CUDA-core forms)
// ------------------------------------------------------------------------------------------
template <typename T>
struct CholScanArgs {
  int n, q, t, j;            // sizes, trait index j of this pass
  const T* Linv;             // n x n row-major lower (L_j^-1)
  const T* XLw;              // q x n whitened covariates
  const T* rw;               // n whitened null residual
  const T* P;                // q x q = S_TL^-1
  const T* b0;               // q null-model coefficients
  const int8_t* XR;          // m x n
  int64_t m;
  int64_t out_offset;        // first SNP's index in the output arrays
  void* B;                   // float or double, (m_total x t x p)
  void* wald;                // may be NULL
  bool out_f64;
  T sing_tol;
  int* flags;
  int out_snp = 0;           // B holds (b_R, standard errors) per pair instead of all p values
  int out_var = 0;           // B holds the p values, then the p(p+1)/2 of Var(b) (packed upper)
  GeneticModel gm;           // the SNP's columns (p = q + gm.pr)
};
template <typename T> void chol_scan_simt(cudaStream_t s, const CholScanArgs<T>& a);

template <typename T>
struct EigScanArgs {
  int n, q, t;
  const T* Zt;               // n x n, row r = eigenvector r
  const T* planes;           // t x (q+2) x ldp
  int ldp;
  const T* P;                // t x q x q
  const T* b0;               // t x q
  const int8_t* XR;
  int64_t m;
  int64_t out_offset;
  void* B;
  void* wald;
  bool out_f64;
  T sing_tol;
  T* xt;                     // scratch: (m pr) x ldp rotated genetic columns
  int* flags;
  int out_snp = 0;           // as CholScanArgs
  int out_var = 0;
  GeneticModel gm;
};
template <typename T> void eig_scan_simt(cudaStream_t s, const EigScanArgs<T>& a);

// Launches one thread that waits, bounded by limit_ms, on a barrier nothing completes
// (selftest.cu).  GWAS_ERR_TIMEOUT when the wait gave up as designed.
gwas_status selftest_wait_timeout(int limit_ms);

// Genotype check: flags[GENOTYPE] = 1 if any value is outside {0,1,2}.
void validate_genotypes(cudaStream_t s, const int8_t* XR, int64_t count, int* flags);

// ------------------------------------------------------------------------------------------
// Genotype formats, genotypes.cu (2-bit packed rows of packed_row_bytes(n) bytes)
// ------------------------------------------------------------------------------------------
int packed_row_bytes(int n);
// int8 m x n -> packed m x row_bytes (values outside {0,1,2} become code 3); with validate,
// flags[GENOTYPE] = 1 for such values.
void pack_genotypes(cudaStream_t s, const int8_t* x, int64_t m, int n, uint8_t* out, int* flags,
                    bool validate);
void unpack_genotypes(cudaStream_t s, const uint8_t* in, int64_t m, int n, int8_t* out);
void validate_packed(cudaStream_t s, const uint8_t* in, int64_t m, int n, int* flags);
// mu[i pr + k] = centre of SNP i's genetic column k (coding code[k]): the multiple of 1/64 nearest
// the column's mean over the n individuals, clamped to [0, 2].
void snp_centres_packed(cudaStream_t s, const uint8_t* in, int64_t m, int n, float* mu, int pr,
                        const uint32_t* code);
// pv[e] = erfc(sqrt(w[e] / 2)) (chi-square(1) upper tail); NaN stays NaN; in place allowed.
void wald_pvalues(cudaStream_t s, const float* w, int64_t count, int dof, float* pv);

}  // namespace gw
