/*
 * gwas.h -- C ABI of the GB300 library for the 2-D grid of generalized least-squares (GLS)
 * problems of mixed-model GWAS (CLAK-Chol / CLAK-Eig, arXiv 1207.2169).
 *
 * The operation (Supplementary Note Section 1, Eq. "probDef"): for every SNP i and trait j
 *
 *     b_ij  = (X_i^T M_j^-1 X_i)^-1 X_i^T M_j^-1 y_j ,   X_i = [X_L | X_R,i],
 *     M_j   = s2_j (h2_j Phi + (1 - h2_j) I),
 *     Var_ij = (X_i^T M_j^-1 X_i)^-1 ,   wald_ij = b_R^T Var_RR^-1 b_R,
 *
 * with n individuals, X_L = [1 | covariates] (q columns, shared by all problems), X_R,i the
 * p_R columns the i-th SNP's genotypes (hard calls 0/1/2) give under the genetic model (p_R = 1
 * for the default additive model: X_R,i = x_i), y_j the j-th trait, p = q + p_R, and b_R, Var_RR
 * the genetic block of b and Var (wald is chi-square with p_R degrees of freedom; for p_R = 1,
 * b_snp^2 / Var_snp,snp).  The output is the m x t x p object B of Fig. 1 plus the m x t Wald
 * statistics.
 *
 * Two algorithms, both exact rearrangements of the definition:
 *   CHOL (Algorithm 3): M = L L^T once per trait; each SNP block is whitened by L^-1
 *         (the aggregated triangular solve of "Sequences of GLS'") and reduced to a bordered
 *         p x p system solved by its Schur complement.
 *   EIG  (Algorithm 4): Phi = Z W Z^T once; each SNP block is rotated (Z^T X_R) and every
 *         (SNP, trait) pair is reduced by trait-weighted inner products to the same bordered
 *         system.
 *
 * Conventions for every call:
 *   - Matrices are column-major unless stated.  Inputs are borrowed: setup copies what it needs
 *     to the device; scan reads its genotype block during the call (or, for device pointers,
 *     until the stream reaches the end of the call's work).
 *   - Outputs are owned by the caller; the library never allocates them.
 *   - Every call returns a gwas_status and never aborts the process; gwas_last_error() gives a
 *     message for the last failure on the calling thread.
 *   - A handle is used by one host thread at a time.  It owns all device state.
 *   - A GLS whose Schur complement sigma = x^T M^-1 x - a^T S_TL^-1 a is not positive beyond
 *     rounding (sigma <= tol * x^T M^-1 x; tol = 1e-12 in FP64, 1e-5 otherwise), e.g. a
 *     monomorphic SNP, gets NaN in all p coefficients and the Wald value; it is not an error and
 *     is counted (gwas_singular_count).
 */
#ifndef GWAS_GB300_H
#define GWAS_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gwas_handle_s* gwas_handle;

typedef enum {
  GWAS_OK = 0,
  GWAS_ERR_ARG = -1,           /* bad pointer, size or option                              */
  GWAS_ERR_NOT_SPD = -2,       /* M_j (CHOL) or Phi (EIG) is not positive definite          */
  GWAS_ERR_CUDA = -3,          /* a CUDA runtime call failed                                */
  GWAS_ERR_OOM = -4,           /* device or pinned-host allocation failed                   */
  GWAS_ERR_UNSUPPORTED = -5,   /* option combination or size the build does not cover       */
  GWAS_ERR_GENOTYPE = -6,      /* validate_genotypes found a value outside {0, 1, 2}        */
  GWAS_ERR_TIMEOUT = -7,       /* a bounded wait gave up                                    */
  GWAS_ERR_SINGULAR = -8,      /* S_TL = X_L^T M^-1 X_L is singular (collinear covariates)  */
  GWAS_ERR_NOT_CONVERGED = -9  /* the eigensolver did not converge                          */
} gwas_status;

enum { GWAS_ALGO_AUTO = 0, GWAS_ALGO_CHOL = 1, GWAS_ALGO_EIG = 2 };

/* Arithmetic of the per-SNP scan (setup is always FP64):
 *   FP64        plain FP64 CUDA-core kernels;
 *   FP32        plain FP32 CUDA-core kernels;
 *   SPLIT_BF16  tensor-core kernels (tcgen05, sm_103a): the non-integer operand of each
 *               contraction is split into hi + lo BF16 pieces (a third for a badly conditioned
 *               M_j, see gwas_split_pieces), genotypes are exact in BF16, accumulation is FP32;
 *               the p x p Schur solve runs in FP64 (CHOL) or FP32 (EIG);
 *   SPLIT_FP8   as SPLIT_BF16, except that CHOL splits the augmented L_j^-1 into an FP16 hi piece
 *               and an E4M3 lo piece (each row group scaled by a power of two into FP16 range):
 *               the hi product takes the centred genotypes in FP16 and the lo product the
 *               uncentred ones in E4M3 (both exact), at the FP8 tensor rate, about 15 significant
 *               bits in all (BF16 x 2: 16); the epilogue subtracts the centring term the lo
 *               product misses.  A badly conditioned M_j takes three BF16 pieces as under
 *               SPLIT_BF16, and EIG scans run exactly as under SPLIT_BF16.                     */
enum { GWAS_PREC_FP64 = 0, GWAS_PREC_FP32 = 1, GWAS_PREC_SPLIT_BF16 = 2, GWAS_PREC_SPLIT_FP8 = 3 };

/* What a scan writes per (SNP, trait) pair into B (wald is the same in all modes):
 *   FULL  all p coefficients: B is m x t x p;
 *   SNP   the SNP effect and its standard error, sqrt(Var(b)[p-1][p-1]) = 1 / sqrt(sigma):
 *         B is m x t x 2 (GWAS summary statistics; with gwas_wald_pvalues, the p-values);
 *   VAR   the p coefficients, then the whole Var(b) = (X_i^T M_j^-1 X_i)^-1 of Eq. "probDef"
 *         as its upper triangle row by row, (0,0), (0,1), .., (0,p-1), (1,1), .., (p-1,p-1):
 *         B is m x t x (p + p(p+1)/2).  A singular pair has NaN in all of them. */
enum { GWAS_OUT_FULL = 0, GWAS_OUT_SNP = 1, GWAS_OUT_VAR = 2 };

/* Genetic models (Table 1: p is set by the covariates and "the genetic model assumed"): the
 * columns X_R,i of a SNP with hard calls x, placed after X_L's q columns in b and Var.
 *   ADDITIVE   x                  (p_R = 1; the default)
 *   DOMINANT   [x >= 1]           (p_R = 1)
 *   RECESSIVE  [x == 2]           (p_R = 1)
 *   ADD_DOM    x, [x == 1]        (p_R = 2: allele count and heterozygosity; wald is their joint
 *                                 2-d.o.f. test)
 * With GWAS_OUT_SNP, B holds per pair the p_R genetic coefficients, then their p_R standard
 * errors sqrt(Var_RR[k][k]) (2 p_R values).  ADD_DOM is solved in the basis of the genotype
 * indicators [x == 1], [x == 2] (the same columns, well conditioned when one homozygote class is
 * rare) and reported for (x, [x == 1]); the Wald statistic does not depend on the basis.  Every
 * precision takes every model, except that the tensor-core scans (SPLIT_BF16, SPLIT_FP8) of
 * ADD_DOM need column 0 of X_L to be the intercept (all ones), the paper's X = [1 | L | g];
 * without it gwas_setup returns GWAS_ERR_UNSUPPORTED (use FP64 or FP32). */
enum { GWAS_MODEL_ADDITIVE = 0, GWAS_MODEL_DOMINANT = 1, GWAS_MODEL_RECESSIVE = 2,
       GWAS_MODEL_ADD_DOM = 3 };

typedef struct {
  int algo;               /* GWAS_ALGO_*; AUTO = CHOL when t == 1, else EIG                   */
  int precision;          /* GWAS_PREC_*                                                      */
  int block_snps;         /* SNPs per device block when streaming host input; 0 = chosen by
                             timing on the first streamed call (gwas_stream_info)             */
  int validate_genotypes; /* nonzero: scan checks every genotype is 0, 1 or 2                 */
  int device;             /* CUDA device ordinal                                              */
  int out_mode;           /* GWAS_OUT_*                                                       */
  int genetic_model;      /* GWAS_MODEL_*                                                     */
} gwas_options;

/* Fills *opt with AUTO, SPLIT_BF16, block_snps 0, validation off, device 0, FULL outputs,
 * the additive genetic model. */
void gwas_default_options(gwas_options* opt);

/*
 * gwas_setup -- the per-cohort precomputation, in FP64 on the GPU: for Algorithm 3, M_j, its
 * Cholesky factor and inverse, the whitened covariates and trait, S_TL and b_T; for Algorithm 4,
 * the eigendecomposition of Phi, the rotated covariates and traits, and per trait D_j, S_TL, b_T.
 *   Phi  n x n kinship, symmetric; only the lower triangle is read.        (host pointer)
 *   XL   n x q covariates, column 0 is normally the intercept (all ones).   (host pointer)
 *   Y    n x t traits.                                                      (host pointer)
 *   h2   t heritabilities, each in [0, 1).  s2: t total variances, each > 0. (host pointers)
 *   opt  options (NULL = defaults).  out: receives the handle (set to NULL on failure).
 * Limits: 1 <= n <= 16384, 1 <= q <= 7, 1 <= t; CHOL additionally needs t * n^2 * 8 bytes.
 * Returns GWAS_ERR_NOT_SPD if M_j or Phi is not positive definite, GWAS_ERR_SINGULAR if X_L
 * is rank deficient in the M_j^-1 inner product.  Synchronous.
 */
gwas_status gwas_setup(const double* Phi, int n, const double* XL, int q, const double* Y, int t,
                       const double* h2, const double* s2, const gwas_options* opt,
                       gwas_handle* out);

/*
 * gwas_scan -- the GLS sequence over one block of m SNPs, every trait: the whitening of the
 * block and the per-SNP bordered solve of Algorithm 3, or the rotation of the block and the
 * per-pair bordered solve of Algorithm 4.
 *   XR    m x n genotypes, int8 hard calls, SNP-major (SNP i's n calls at XR + i*n).
 *   B     m x t x p results, B[(i*t + j)*p + k]; k < q follow XL, k = q .. p-1 are the genetic
 *         columns (k = p-1 is the SNP effect of the additive model).
 *   wald  m x t Wald statistics, wald[i*t + j].  May be NULL (not written).
 *   xr_on_device / out_on_device: nonzero when the pointer is device memory.
 *   stream: cudaStream_t (NULL = legacy default stream).
 * When XR and all outputs are on the device the call is asynchronous on `stream`.  Otherwise
 * XR is streamed through the handle's device ring in blocks of block_snps SNPs (host memory
 * pinned by the caller makes the copies asynchronous and overlapped; CHOL blocks alternate
 * between `stream` and a second stream of the handle) and the call returns when the outputs
 * are complete.
 */
gwas_status gwas_scan(gwas_handle h, const int8_t* XR, int64_t m, int xr_on_device, float* B,
                      float* wald, int out_on_device, void* stream);

/* gwas_scan_f64 -- as gwas_scan with FP64 outputs (meaningful for GWAS_PREC_FP64). */
gwas_status gwas_scan_f64(gwas_handle h, const int8_t* XR, int64_t m, int xr_on_device,
                          double* B, double* wald, int out_on_device, void* stream);

/*
 * gwas_wald_pvalues -- p-values of Wald statistics, the chi-square (1 degree of freedom) upper
 * tail erfc(sqrt(wald / 2)) (Section "Mixed Models for GWAS": the test of each SNP effect).  NaN
 * stays NaN.  on_device = 0: host arrays, synchronous; otherwise device arrays, asynchronous on
 * `stream`.  wald and pval may be the same array.
 */
gwas_status gwas_wald_pvalues(const float* wald, int64_t count, float* pval, int on_device,
                              void* stream);

/*
 * gwas_wald_pvalues_dof -- as gwas_wald_pvalues for the joint test of a p_R-column genetic model
 * (Eq. "probDef" with a block X_R; gwas_genetic_columns): the chi-square upper tail with `dof`
 * degrees of freedom, dof = 1 (erfc(sqrt(wald / 2))) or dof = 2 (exp(-wald / 2), exact for two
 * degrees of freedom).  Any other dof returns GWAS_ERR_ARG.
 */
gwas_status gwas_wald_pvalues_dof(const float* wald, int64_t count, int dof, float* pval,
                                  int on_device, void* stream);

/* Criteria of gwas_estimate. */
enum { GWAS_EST_ML = 0, GWAS_EST_REML = 1 };

/*
 * gwas_estimate -- step 1 of the two-step method (Supplementary Note Section 1, "Mixed Models
 * for GWAS"; "Time complexity"): per trait, the variance components of the reduced model
 * y_j = X_L beta + R, R ~ N(0, s2 (h2 Phi + (1 - h2) I)), that maximise its likelihood
 * (GWAS_EST_ML) or restricted likelihood (GWAS_EST_REML), for gwas_setup's h2 and s2.
 *   Phi, XL, Y, n, q, t: as in gwas_setup (host pointers, copied).  device: CUDA ordinal.
 *   h2, s2: t outputs (host).  crit: t outputs or NULL, the maximised log-likelihood
 *   (ML: -1/2 [n log(2 pi s2) + log|H| + n]; REML, the log-density of the error contrasts:
 *   -1/2 [(n - q) log(2 pi s2) + log|H| + log|X_L^T H^-1 X_L| - log|X_L^T X_L| + (n - q)],
 *   H = h2 Phi + (1 - h2) I).  ms: 2 outputs or NULL, device milliseconds of the
 *   eigendecomposition of Phi with the rotation of X_L and Y, and of the search.
 * Method (FP64 on the GPU): Phi = Z W Z^T; per trait the criterion, a weighted sum over the
 * eigen-coordinates, on the grid h2 = (g / 100) 0.999, g = 0..100, then a golden-section search
 * between the best grid point's neighbours.  h2 lies in [0, 0.999].  A trait that X_L fits
 * exactly (r^T H^-1 r at most 1e-12 of y^T H^-1 y) gets h2 = NaN, s2 = 0, crit = NaN.  Returns GWAS_ERR_NOT_SPD if h Phi + (1 - h) I is
 * not positive definite for some h in [0, 0.999], GWAS_ERR_SINGULAR for collinear covariates,
 * GWAS_ERR_NOT_CONVERGED if the eigensolver fails.  Synchronous; allocates device memory for
 * the duration of the call.
 */
gwas_status gwas_estimate(const double* Phi, int n, const double* XL, int q, const double* Y,
                          int t, int method, int device, double* h2, double* s2, double* crit,
                          double* ms);

/*
 * Packed genotype format (a storage format for the same genotype matrix X_R of "Sequences of
 * GLS'", hard calls of m SNPs for n individuals): SNP i occupies gwas_packed_row_bytes(n) =
 * ceil(n / 64) * 16 bytes starting at G + i * gwas_packed_row_bytes(n); the genotype of
 * individual k sits in byte k / 4 at bits 2 (k % 4) and 2 (k % 4) + 1 and holds the allele
 * count 0, 1 or 2.  Code 3 is invalid and every code past the n-th of a row is 0.  Four genotypes per byte: a quarter of the
 * int8 bytes to stream from host memory and HBM, and the tensor-core kernels read these rows
 * directly (int8 input is packed on the device first).
 */
int gwas_packed_row_bytes(int n); /* 0 for n < 1 */

/*
 * gwas_shard -- the SNP range [*start, *start + *count) that rank `rank` of `world` processes
 * when a genome of m_total SNPs is split across processes (one per GPU).  Every (SNP, trait)
 * pair of the grid of Eq. "probDef" is independent of the others given the setup state
 * (Algorithms 3 and 4 loop over SNPs with nothing carried between iterations), so ranks need
 * no exchange on the data path: each sets up its own handle and scans its own range.  The
 * ranges are contiguous, disjoint, ordered by rank and cover [0, m_total); each holds a whole
 * number of `align`-SNP units except where m_total ends, and the unit counts of two ranks differ
 * by at most one.  Host only, no GPU needed.  GWAS_ERR_ARG if m_total < 0, world < 1,
 * rank outside [0, world), align < 1 or an output pointer is NULL.
 */
gwas_status gwas_shard(int64_t m_total, int rank, int world, int64_t align, int64_t* start,
                       int64_t* count);

/*
 * gwas_pack_genotypes -- int8 m x n hard calls X -> packed rows G (m * gwas_packed_row_bytes(n)
 * bytes, caller-owned).  on_device = 0: both host pointers, synchronous; a value outside
 * {0,1,2} is written as code 3 and the call returns GWAS_ERR_GENOTYPE after packing every row.
 * on_device != 0: both device pointers on the current device, asynchronous on `stream`
 * (cudaStream_t); values outside {0,1,2} become code 3, which a scan with validate_genotypes
 * reports.
 */
gwas_status gwas_pack_genotypes(const int8_t* X, int64_t m, int n, uint8_t* G, int on_device,
                                void* stream);

/*
 * gwas_scan_packed -- gwas_scan on packed genotype rows G (m rows; device pointers must be
 * 16-byte aligned, else GWAS_ERR_ARG).  Every other argument, the streaming of host input
 * (now gwas_packed_row_bytes(n) bytes per SNP) and the synchronisation rules are gwas_scan's.
 * With validate_genotypes, a code 3 or a nonzero code past the n-th is GWAS_ERR_GENOTYPE.
 */
gwas_status gwas_scan_packed(gwas_handle h, const uint8_t* G, int64_t m, int g_on_device,
                             float* B, float* wald, int out_on_device, void* stream);

/*
 * Batched cohorts.  Several independent cohorts -- each its own kinship, covariates (q may
 * differ), traits and sizes -- share one batch.  gwas_scan_batch scans one block of packed
 * genotypes per cohort on the tensor cores as one CUDA graph: small cohorts cannot fill the GPU
 * alone, so their persistent kernels share the SMs.  The launch plan (all cohorts one after
 * another; all at once with SM shares proportional to their work; all at once with every SM; two
 * lanes of half the SMs) is chosen by timing each candidate on the first call for a given set
 * of block sizes.
 */
typedef struct gwas_batch_s* gwas_batch;

typedef struct {          /* one cohort: the inputs of gwas_setup (host pointers, copied)    */
  const double* Phi;
  int n;
  const double* XL;
  int q;
  const double* Y;
  int t;
  const double* h2;
  const double* s2;
} gwas_cohort;

typedef struct {          /* one cohort's block: device pointers                              */
  const uint8_t* G;       /* m packed genotype rows (gwas_packed_row_bytes(n) each), 16-byte
                             aligned                                                         */
  int64_t m;              /* SNPs of the block (0: this cohort is skipped)                   */
  float* B;               /* m x t x p, as gwas_scan                                         */
  float* wald;            /* m x t or NULL                                                   */
} gwas_cohort_block;

/* gwas_setup for every cohort (opt applies to all; precision SPLIT_BF16 or SPLIT_FP8).  Fails
 * with the first failing cohort's status (message names the cohort) and creates nothing then. */
gwas_status gwas_setup_batch(int n_cohorts, const gwas_cohort* cohorts, const gwas_options* opt,
                             gwas_batch* out);

/* Scans blocks[i] of every cohort i, asynchronously on `stream` (cudaStream_t).  The first call
 * for a given set of block sizes times the launch plans (it synchronises the stream) and keeps
 * the fastest; later calls with the same sizes replay that plan's graph on the new buffers.
 * Genotypes are not validated; use gwas_scan_packed with validate_genotypes for that. */
gwas_status gwas_scan_batch(gwas_batch b, const gwas_cohort_block* blocks, void* stream);

/* The chosen plan (0-3, -1 before the first scan) and the time of each plan (ms, 4 values) with
 * the chosen EIG chunk. */
gwas_status gwas_batch_plan(gwas_batch b, int* plan, double* plan_ms);

/* The whole tuning of the last new block shape: the chosen plan, the chosen EIG chunk divisor d
 * (each EIG cohort's scan takes its SNPs in chunks of its scratch capacity / 2^d, d = 0, 1, 2;
 * gwas_eig_chunk gives the SNPs), and the time (ms) of every (d, plan) candidate in
 * ms[d * 4 + plan] (12 values).  The autotuner of the batched launch (no counterpart in the
 * paper, which runs one cohort at a time). */
gwas_status gwas_batch_tuning(gwas_batch b, int* plan, int* chunk_div, double* ms);

/* The handle of cohort i (for gwas_info, gwas_singular_count; owned by the batch), or NULL. */
gwas_handle gwas_batch_handle(gwas_batch b, int i);

/* Frees the batch and every cohort's handle.  NULL is ignored. */
void gwas_destroy_batch(gwas_batch b);

/*
 * gwas_scan_static -- a scan that allocates no device memory.  (Not from the paper, which has
 * no counterpart: this is a deployment variant of gwas_scan.)
 *
 * Some callers cannot let a library call cudaMalloc during a scan: latency-critical loops,
 * where cudaMalloc's implicit device synchronisation would stall work the caller has queued on
 * other streams, and applications whose device memory is owned entirely by their own allocator
 * or memory budget (a serving process that reserves HBM up front), where an allocation behind
 * the allocator's back can fail or push another component out of memory.
 * gwas_scan may allocate on its first call (the EIG CUDA-core path's scratch for the rotated
 * genotypes Z^T X_R, and the host-streaming ring); this entry point never does.  It runs the
 * EIG CUDA-core scan (handles set up with algo EIG and precision FP64 or FP32) with that
 * scratch in one fixed 16 MiB device array that the library holds on every GPU that loads it,
 * from load until process exit.
 *   XR, B, wald: device pointers, as in gwas_scan (wald may be NULL); stream: cudaStream_t.
 *   Limit: m * ldp * e <= 16 MiB, where ldp = n rounded up to 64 and e = 8 (FP64) or 4 (FP32)
 *   bytes; larger m returns GWAS_ERR_ARG (scan such genotypes in several calls).  Other
 *   handles return GWAS_ERR_UNSUPPORTED.
 * Asynchronous on `stream`, except on a handle set up with validate_genotypes: then every
 * genotype is checked first (a value outside {0, 1, 2} returns GWAS_ERR_GENOTYPE, and that
 * call's outputs are not meaningful) and the call returns when the scan is complete.
 * The first call on a device looks up the array's device address
 * (once per device; a cudaGetSymbolAddress, not an allocation): make that first call before
 * any stream capture.  Every call shares the one array and finds it holding the previous
 * call's data (the scan overwrites everything it reads), so calls whose work overlaps on the
 * GPU -- other streams, other threads, other handles -- race on it and must be serialised
 * by the caller (e.g. one stream).
 */
gwas_status gwas_scan_static(gwas_handle h, const int8_t* XR, int64_t m, float* B, float* wald,
                             void* stream);

/* Milliseconds the FP64 setup took on the device (CUDA events around it). */
gwas_status gwas_setup_timing(gwas_handle h, double* ms_setup);

/* Sizes and resolved options of a handle (any pointer may be NULL). */
gwas_status gwas_info(gwas_handle h, int* n, int* q, int* t, int* algo, int* precision);

/*
 * gwas_stream_info -- how a handle streams host input or output (not from the paper: the
 * pipeline of "Sequences of GLS'" on this GPU).  Any pointer may be NULL.
 *   block_snps      SNPs per streamed block now in use;
 *   tuned           1 once the block size was chosen by timing: with block_snps = 0 at setup,
 *                   the first streamed call times, on its own first SNPs, the H2D copy, the scan
 *                   and the D2H copy of a block at sizes 8 Ki .. 256 Ki SNPs (within the output
 *                   ring's 2 GB) and keeps the size minimising that call's modelled pipeline
 *                   time (the fill plus, per further block, its slowest stage);
 *   graph_launches  full blocks whose device work ran as a replayed CUDA graph (one graph per
 *                   ring slot, captured on first use);
 *   ncand, cand_snps (8), cand_ms (8 x 3)  the timed candidates: size, and ms of H2D copy,
 *                   scan and D2H copy (0 for a copy the call did not need).
 */
gwas_status gwas_stream_info(gwas_handle h, int* block_snps, int* tuned, int64_t* graph_launches,
                             int* ncand, int64_t* cand_snps, double* cand_ms);

/* p_R, the genetic columns per SNP of the handle's model (p = q + p_R), or -1 for NULL. */
int gwas_genetic_columns(gwas_handle h);

/* BF16 pieces of the tensor-core scans' split operands: 2, or 3 when setup found some
 * M_j = s2 (h2 Phi + (1 - h2) I) with lam_max / lam_min above 100 (h2 near 1 on a kinship with
 * many eigenvalues at its ridge), where two pieces (~16 significant bits) would not hold the
 * 1e-4 bound.  CHOL chooses per trait (3 pieces of its augmented L_j^-1: one product in two
 * more); EIG per handle (3 pieces of every U_j = M_j^-1 [X_L | r_j]: the a/c kernel one product
 * in two more).  0 for CUDA-core handles, -1 for NULL.  Past lam_max / lam_min = 500 the EIG
 * contraction's FP32 accumulation, not its pieces, would bound the error near 1e-4: EIG handles
 * scan those traits with the CHOL kernel as well (gwas_chol_routed_traits). */
int gwas_split_pieces(gwas_handle h);

/* Number of traits whose CHOL scan runs the FP16 hi + E4M3 lo split (precision SPLIT_FP8: every
 * trait whose M_j is not badly conditioned; the others take three BF16 pieces); 0 for other
 * precisions and for EIG; -1 for a NULL handle. */
int gwas_fp8_traits(gwas_handle h);

/* EIG tensor-core handles: the number of traits whose M_j is conditioned past the point where
 * the EIG contraction's FP32 accumulation keeps 1e-4 (lam_max / lam_min of M_j above 500, e.g.
 * h^2 near 1 on a kinship with many eigenvalues at its ridge).  Setup also factors those traits'
 * M_j (Algorithm 3's setup), and every scan runs the CHOL kernel on them after the EIG kernels,
 * overwriting their outputs; 0 for other handles, -1 for a NULL handle.  A routed trait costs
 * what a CHOL trait costs: setup holds its L_j^-1 in FP64 (8 n^2 bytes per routed trait, all at
 * once) and keeps three BF16 pieces of it (6 n^2 bytes), and each scan adds one CHOL pass over
 * the block's SNPs per routed trait (about n^2 / 2 multiply-adds per SNP and piece), so a cohort whose
 * traits are mostly routed is better set up with GWAS_ALGO_CHOL. */
int gwas_chol_routed_traits(gwas_handle h);

/* EIG tensor-core handles: SNPs per internal chunk of a scan (one launch of each EIG kernel per
 * chunk; set by setup, or by the batch tuner for a batch's cohorts); 0 for other handles; -1 for
 * a NULL handle. */
int64_t gwas_eig_chunk(gwas_handle h);

/* Number of singular pairs (written as NaN) seen by completed scans of this handle, or -1. */
int64_t gwas_singular_count(gwas_handle h);

/*
 * gwas_sync -- waits for all work on the handle's device, then reports GWAS_ERR_TIMEOUT if a
 * tensor-core kernel of this handle gave up one of its bounded waits since the last report
 * (that call's outputs are incomplete; the flag is cleared and the handle stays usable).
 * Synchronous scans (host buffers, or validate_genotypes) report it themselves.
 */
gwas_status gwas_sync(gwas_handle h);

/*
 * gwas_selftest_timeout -- checks the bounded-wait mechanism of the tensor-core kernels on
 * `device` (not from the paper: a failure-detection self-test).  One GPU thread waits on a
 * barrier phase that nothing completes; after limit_ms (1..10000) it must give up and record
 * the timeout, and the GPU context stays usable.  Returns GWAS_ERR_TIMEOUT when that happened
 * as designed, GWAS_ERR_CUDA otherwise.
 */
gwas_status gwas_selftest_timeout(int device, int limit_ms);

/*
 * Per-stage device time of a handle's scans (not from the paper: instrumentation for the
 * roofline of each kernel).  While enabled, every stage launch of a gwas_scan /
 * gwas_scan_packed on this handle is bracketed by two CUDA events on the stream it runs on;
 * gwas_stage_times waits for the recorded events, writes per stage the summed milliseconds
 * (ms[GWAS_NSTAGES]) and the number of timed launches (launches[GWAS_NSTAGES], may be NULL),
 * and starts a new tally.  A "launch" is one stage call for one chunk of SNPs (CHOL: one per
 * trait).  gwas_stage_timing(h, 0 or 1) switches it off or on (waiting for the device first)
 * and clears the tally.  Events are created on first use and kept by the handle.
 */
enum { GWAS_STAGE_PACK = 0,    /* int8 -> packed rows (tensor cores) or back (CUDA cores)      */
       GWAS_STAGE_CENTRES = 1, /* per-SNP centres of the EIG tensor-core path                  */
       GWAS_STAGE_CHOL = 2,    /* CHOL tensor-core whiten + reduce + Schur                      */
       GWAS_STAGE_ROT = 3,     /* EIG rotation (Z^T X_R)^2                                      */
       GWAS_STAGE_SQ = 4,      /* EIG s_ij                                                      */
       GWAS_STAGE_AC = 5,      /* EIG a_ij, c_ij + Schur                                        */
       GWAS_STAGE_SIMT = 6,    /* a whole CUDA-core (FP64 / FP32) scan of a block              */
       GWAS_NSTAGES = 8 };
gwas_status gwas_stage_timing(gwas_handle h, int enable);
gwas_status gwas_stage_times(gwas_handle h, double* ms, int64_t* launches);

/* Message of the last failure on the calling thread ("" if none).  Never NULL. */
const char* gwas_last_error(void);

/* Frees every resource of the handle.  NULL is ignored. */
void gwas_destroy(gwas_handle h);

#ifdef __cplusplus
}
#endif
#endif /* GWAS_GB300_H */
