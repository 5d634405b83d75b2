// Launchers and parameter blocks of the tcgen05 kernels (internal to the library).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace gw {

// ------------------------------------------------------------------------------------------
// CHOL fused whiten-and-reduce (tc_chol.cu)
// ------------------------------------------------------------------------------------------
struct CholTcParams {
  int64_t m;          // SNPs of this launch (genotypes come through the mapG tensor map)
  int n, q, t, j;     // sizes; j = trait of this launch
  int kpad;           // n rounded up to 64: K extent of the split rows
  int rpad;           // n + q + 1 rounded up to 256: rows of each piece of the split matrix
                      // [L^-1; (M^-1 X_L)^T; (M^-1 r)^T] of trait j
  const double* P;    // q x q  (X_L^T M^-1 X_L)^-1
  const double* b0;   // q      null-model coefficients
  int centre;         // nonzero: centre each SNP by the multiple of 1/64 nearest its mean
  const uint8_t* G;   // the launch's packed genotype rows (also read through mapG)
  int row_bytes;      // packed_row_bytes(n)
  int out_snp;        // B holds (b_R, standard errors) per pair instead of all p values
  int out_var;        // B holds the p values, then the p(p+1)/2 of Var(b) (packed upper)
  float* B;           // m x t x p (p = q + gp)
  float* W;           // m x t or NULL
  int* flags;
  int gp;             // genetic columns per SNP (1 or 2); a tile holds CHOL_TC_BM / gp SNPs
  uint32_t code[2];   // coding of each genetic column: values of genotypes 0, 1, 2 in bytes 0-2
  float tm[4];        // gp = 2: reported coefficients = tm (row-major 2 x 2) x working ones
  int pieces;         // BF16 pieces of trait j's split matrix (2 or 3), rpad rows each
  int fp8;            // nonzero: trait j's split is FP16 hi (lmaps.m) + E4M3 lo (lmaps.m8)
  // fp8: the matrix has one more augmented row, w (row n + q + 1, below); row group g is held
  // scaled by 2^e_g (g = 0: the rows of L^-1; g = 1 + k: augmented row n + k, k = 0 .. q + 1);
  // unscale[g] = 2^-e_g.  lsa[k] = the sum of augmented row n + k's E4M3 lo piece (scaled), and
  // k2 = sum over the rows r < n of lsum_r^2, lsum_r the sum of row r's lo piece (scaled).
  // With the lo product taking uncentred codes, accumulator row r holds x'_r + mu lsum_r; the
  // epilogue corrects s with w . (x - mu) = sum_r lsum_r x'_r (row n + q + 1 of the product):
  // s = sum_r acc_r^2 - 2 mu (w . (x - mu)) - mu^2 k2, and a_k, c by -mu lsa[k].
  float unscale[10];
  float lsa[9];
  double k2;
  int naug;           // augmented rows below L^-1: q + 1, or q + 2 with fp8
};
constexpr int CHOL_TC_BM = 128;  // rows (SNP columns) per tile
// Tensor maps of one trait's split augmented L^-1: rows = 2 * rpad (hi piece then lo piece),
// cols = kpad, BF16, 128-byte swizzle, 64-column boxes of 256 - 64 j rows (m[j]: the rows
// 64 j .. 255 of a block, which a K step on the block's diagonal meets).
// With SPLIT_FP8, m[] covers the FP16 hi piece (rpad rows; the same boxes) and m8[] the E4M3 lo
// piece: uint8 [rpad][kpad], 64-byte boxes of 256 - 64 j rows, 64-byte swizzle, its columns in
// e4m3_k_slot order within each aligned group of 16.
struct CholMaps {
  CUtensorMap m[4];
  CUtensorMap m8[4];
};
// mapG: the 2-bit packed genotypes of the launch, uint8 [m][packed_row_bytes(n)], boxes of
// 16 bytes x (128 / gp) rows, no swizzle.
void chol_tc_launch(cudaStream_t s, const CholMaps& lmaps, const CUtensorMap& mapG,
                    const CholTcParams& p, int num_sms);
// uint8 map over packed genotype rows (boxes 16 bytes x box_rows rows).
CUtensorMap make_map_packed(const void* base, int64_t rows, int row_bytes, int box_rows = 128);
// uint8 map over [rows][cols] bytes (cols a multiple of 16, base 16-byte aligned), boxes of 64
// bytes x box_rows rows, 64-byte swizzle; out-of-range reads are zero.
CUtensorMap make_map_u8_sw64(const void* base, int64_t rows, int64_t cols, int box_rows);
void chol_tc_prepare();
// CTAs of the CHOL kernel that fit on the device at once (after chol_tc_prepare).
int chol_tc_resident_ctas(int q);

// ------------------------------------------------------------------------------------------
// EIG stages (tc_eig.cu): 0 = ROT (Xsq = (Z^T X_R)^2 split), 1 = SQ (s_ij), 2 = AC (a, c, Schur)
// ------------------------------------------------------------------------------------------
struct EigTcParams {
  int64_t m;               // SNPs of this launch (ROT, AC: genotypes through mapG)
  int n, q, t, kpad;
  int nblk;                // 256-column blocks of the accumulator
  int b_piece_rows;        // row of the lo piece in the B tensor map
  int b_rows_per_blk;      // B rows per column block
  int a_piece_rows;        // Xsq capacity: row of the lo piece (SQ map, ROT output)
  int traits_per_blk;      // AC: traits per column block
  __nv_bfloat16* xsq;      // ROT output: hi rows [0, cap), lo rows [cap, 2 cap), ld kpad
  float* sbuf;             // SQ output / AC input: s_ij at sbuf[j * lds + i]
  int64_t lds;
  int64_t xplane;          // gp = 2: row stride of the three squared planes (x0 x0, x0 x1, x1 x1)
                           // in xsq and of the three s planes in sbuf
  const float* P;          // AC: t x q x q
  const float* b0;         // AC: t x q
  const float* mu;         // ROT, AC: per-SNP centring (multiples of 1/64) or NULL
  float* B;                // AC: m x t x p (or x 2 with out_snp)
  int out_snp;             // AC: B holds (b_snp, standard error) per pair
  int out_var;             // AC: B holds the p values, then the p(p+1)/2 of Var(b)
  float* W;                // AC: m x t or NULL
  int* flags;
  int gp;                  // genetic columns per SNP
  uint32_t code[2];        // coding of each genetic column (bytes: values of genotypes 0, 1, 2)
  float tm[4];             // gp = 2: reported coefficients = tm (row-major 2 x 2) x working ones
  int pieces;              // ROT, AC: BF16 pieces of the B operand (b_piece_rows rows each)
};
// Traits per AC column block: T (q+1) accumulator columns, with the last trait's load of
// QP = (q+1 rounded up to 4 or 8) columns still inside the 256-column block.
__host__ __device__ constexpr int eig_ac_traits(int q) {
  return 256 / (q + 1) < (256 - (q + 1 <= 4 ? 4 : 8)) / (q + 1) + 1
             ? 256 / (q + 1)
             : (256 - (q + 1 <= 4 ? 4 : 8)) / (q + 1) + 1;
}
// mapA: the Xsq planes (SQ only; ignored otherwise).  mapB: Z^T split (ROT), d split (SQ),
// U split (AC).  All BF16, 64-column boxes, 128-byte swizzle; mapA has 128-row boxes and mapB
// 256-row boxes.  mapG: packed genotypes as for CHOL (ROT, AC; ignored by SQ).
void eig_tc_launch(cudaStream_t s, int stage, const CUtensorMap& mapA, const CUtensorMap& mapB,
                   const CUtensorMap& mapG, const EigTcParams& p, int num_sms);
// Kernel attributes of every EIG stage (once per process; before any launch or graph capture).
void eig_tc_prepare();

}  // namespace gw
