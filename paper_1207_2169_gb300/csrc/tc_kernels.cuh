// Launchers and parameter blocks of the tcgen05 kernels (internal to the library).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace gw {

// ------------------------------------------------------------------------------------------
// CHOL fused whiten-and-reduce (tc_chol.cu)
// ------------------------------------------------------------------------------------------
struct CholTcParams {
  const int8_t* XR;   // m x n genotypes (device)
  int64_t m;
  int n, q, t, j;     // sizes; j = trait of this launch
  int kpad;           // n rounded up to 64: K extent of the split L^-1 rows
  int rpad;           // n rounded up to 256: rows of each piece of the split L^-1
  const float* XLw;   // q x n  whitened covariates L^-1 X_L of trait j
  const float* rw;    // n      whitened null residual of trait j
  const double* P;    // q x q  (X_L^T M^-1 X_L)^-1
  const double* b0;   // q      null-model coefficients
  float* B;           // m x t x p
  float* W;           // m x t or NULL
  int* flags;
};
constexpr int CHOL_TC_BM = 128;  // SNPs per tile
// Tensor maps: rows = 2 * rpad (hi piece then lo piece), cols = kpad, BF16, 128-byte swizzle;
// map256 has 64 x 256 boxes, map128 64 x 128 boxes.
void chol_tc_launch(cudaStream_t s, const CUtensorMap& map256, const CUtensorMap& map128,
                    const CholTcParams& p, int num_sms);
void chol_tc_prepare();

}  // namespace gw
