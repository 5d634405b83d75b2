// Tensor-core (tcgen05, sm_103a) split-BF16 scan path: state and entry points.
#pragma once

#include <vector>

#include "common.cuh"

namespace gw {

struct TcState;

// Pieces of the BF16 split of the M_j^-1-weighted operand (CHOL: the augmented L_j^-1; EIG:
// U_j = M_j^-1 [X_L | r_j]): two (~16 significant bits) unless the conditioning of M_j,
// kappa = lam_max / lam_min, exceeds this, then three (~24 bits).  The two-piece error grows with
// kappa when Phi has many eigenvalues at its ridge (a kinship from fewer SNPs than individuals):
// ~3e-5 at kappa = 100, past 1e-4 near kappa = 600-1000, while three pieces stay near 2e-6.
constexpr double KAPPA_THIRD_PIECE = 100.0;
// Past this conditioning even three pieces leave the EIG contraction at its FP32 accumulation
// floor (the error of a and c, amplified by the cancellation in sigma = s - a^T P a, passes 1e-4
// near kappa = 1000-1500), while the CHOL kernel, which sums its blocks in FP64, stays well within
// it: an EIG handle scans such traits with the CHOL kernel (three BF16 pieces of their own L_j^-1)
// after the EIG kernels, overwriting their outputs.
constexpr double KAPPA_CHOL_ROUTE = 500.0;

struct TcSetupArgs {
  int algo, n, q, t;
  const double* Linv;    // CHOL: t x n x n row-major lower (FP64)
  const double* XLw;     // CHOL: t x q x n
  const double* rw;      // t x n: CHOL whitened null residual / EIG weighted residual
  const double* Zt;      // EIG: n x n, row r = eigenvector r
  const double* planes;  // EIG: t x (q+2) x ldp FP64 planes
  int ldp;
  const double* P;       // t x q x q
  const double* b0;      // t x q
  int block_snps;        // EIG: SNPs per internal chunk (sizes the per-chunk scratch)
  int intercept;         // column 0 of X_L is all ones: SNPs are centred (CHOL, EIG)
  int out_snp;           // B holds (b_snp, standard error) per pair instead of all p values
  int out_var;           // B holds the p values, then the p(p+1)/2 of Var(b) (packed upper)
  GeneticModel gm;       // the SNP's genetic columns (p = q + gm.pr)
  const int* pieces;     // CHOL: split pieces (2 or 3) per trait; EIG: pieces[0] for every U_j
  int fp8_lo;            // CHOL: a two-piece trait is split FP16 hi + E4M3 lo (SPLIT_FP8)
};

struct TcScanArgs {
  const uint8_t* G;  // m rows of packed_row_bytes(n) bytes, 2-bit genotype codes; device,
                     // 16-byte aligned
  int64_t m;
  float* B;          // m x t x p (or x 2 with out_snp) device
  float* wald;       // m x t device or NULL
  int* flags;
  int max_ctas;      // CTAs per kernel at most (0: one per SM); lets scans share the GPU
  StageTimer* timer; // per-stage events (NULL or off: none)
};

// Throws Fail{GWAS_ERR_UNSUPPORTED} for sizes the tensor-core kernels do not cover.
void tc_check_supported(int algo, int n, int q, int t);
TcState* tc_setup(cudaStream_t s, const TcSetupArgs& a);
void tc_scan(cudaStream_t s, TcState* st, const TcScanArgs& a);
void tc_destroy(TcState* st);
// Rough tensor-core work of scanning m SNPs (FLOPs issued), for planning concurrent scans.
double tc_scan_work(const TcState* st, int64_t m);
// Largest number of split pieces the state's kernels use (2 or 3).
int tc_split_pieces(const TcState* st);
// Number of CHOL traits whose split is FP16 hi + E4M3 lo (SPLIT_FP8).
int tc_fp8_traits(const TcState* st);
// EIG: the traits `route` (a CHOL state over those traits only, set up from their own L_j^-1)
// scans after the EIG kernels; route's local trait k writes global trait jmap[k] of t_global.
// The EIG a/c kernel leaves those traits out of its singular count (their P_j is set to NaN in
// its constants; the CHOL pass counts them).  st takes ownership of route.
void tc_attach_chol_route(cudaStream_t s, TcState* st, TcState* route, const std::vector<int>& jmap);
int tc_chol_routed_traits(const TcState* st);
// EIG: SNPs per internal chunk of a tensor-core scan (the ROT, SQ, AC launches cover one chunk
// each), the most the per-chunk scratch holds, and a new chunk (clamped to [128, capacity],
// rounded up to 128).  CHOL: 0 / no effect.
int64_t tc_eig_chunk(const TcState* st);
int64_t tc_eig_chunk_capacity(const TcState* st);
void tc_set_eig_chunk(TcState* st, int64_t snps);

}  // namespace gw
