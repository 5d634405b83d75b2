// FP64 setup kernels: the once-per-cohort and once-per-trait work of Algorithms 3 and 4.
//
//   form_M       Supplementary Note Section 1 / Algorithm 3: M = s2 (h2 Phi + (1-h2) I)
//   cholesky     Algorithm 3: L L^T = M (blocked right-looking, 32-wide panels)
//   tri_inverse  L^-1, so that the per-block whitening of Algorithm 3 is one product
//   jacobi_eig   Algorithm 4: Phi = Z W Z^T (one-sided Jacobi, FP64)
//   trait_pack   Algorithms 3 and 4, per trait: S_TL, b_T, P = S_TL^-1,
//                b0 = P b_T and the weighted null residual used by the bordered solve
//
// All of it runs on CUDA cores in FP64; none of it is on the per-SNP path.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <vector>

#include <cuda_fp8.h>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace gw {

// ------------------------------------------------------------------------------------------
// Generic strided FP64 GEMM (64 x 64 tiles, 256 threads, 4 x 4 per thread)
// ------------------------------------------------------------------------------------------
namespace {
constexpr int GT = 64, GK = 16;

__global__ void __launch_bounds__(256) gemm_f64_kernel(int M, int N, int K, double alpha,
                                                       const double* __restrict__ A, int64_t sai,
                                                       int64_t sak, const double* __restrict__ B,
                                                       int64_t sbk, int64_t sbj, double beta,
                                                       double* __restrict__ C, int64_t sci,
                                                       int64_t scj, int lower_only, int b_tri,
                                                       int64_t bsa, int64_t bsb, int64_t bsc,
                                                       int M_last, int K_last) {
  const int bi = blockIdx.y, bj = blockIdx.x, z = blockIdx.z;
  if (lower_only && bj * GT > bi * GT + GT - 1) return;
  // batch member z: operands offset by z times their batch strides; the last member may have
  // fewer rows and a shorter inner dimension
  if (z == (int)gridDim.z - 1) {
    M = M_last;
    K = K_last;
  }
  if (bi * GT >= M) return;
  A += z * bsa;
  B += z * bsb;
  C += z * bsc;
  // a triangular B has zeros outside k <= j (b_tri > 0) or k >= j (b_tri < 0): the tile's
  // columns j0 .. j0 + GT - 1 need only the k range that can be non-zero
  const int kbeg = b_tri < 0 ? min(bj * GT, K) : 0;
  const int kend = b_tri > 0 ? min(bj * GT + GT, K) : K;
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int i0 = bi * GT, j0 = bj * GT;
  double acc[4][4] = {};
  for (int k0 = kbeg; k0 < kend; k0 += GK) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = tid + 256 * l;
      int i, k;
      if (sai == 1) { i = e % GT; k = e / GT; } else { k = e % GK; i = e / GK; }
      const int gi = i0 + i, gk = k0 + k;
      As[k][i] = (gi < M && gk < K) ? A[gi * sai + gk * sak] : 0.0;
      int j;
      if (sbj == 1) { j = e % GT; k = e / GT; } else { k = e % GK; j = e / GK; }
      const int gj = j0 + j, gk2 = k0 + k;
      Bs[k][j] = (gj < N && gk2 < K) ? B[gk2 * sbk + gj * sbj] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < GK; ++k) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = As[k][ty + 16 * u]; b[u] = Bs[k][tx + 16 * u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int gi = i0 + ty + 16 * u, gj = j0 + tx + 16 * v;
      if (gi < M && gj < N) {
        double* c = C + gi * sci + gj * scj;
        *c = alpha * acc[u][v] + (beta == 0.0 ? 0.0 : beta * *c);
      }
    }
}
}  // namespace

void gemm_f64(cudaStream_t s, int M, int N, int K, double alpha, const double* A, int64_t sai,
              int64_t sak, const double* B, int64_t sbk, int64_t sbj, double beta, double* C,
              int64_t sci, int64_t scj, bool lower_only, int b_tri) {
  if (M <= 0 || N <= 0) return;
  dim3 grid(ceil_div(N, GT), ceil_div(M, GT));
  gemm_f64_kernel<<<grid, 256, 0, s>>>(M, N, K, alpha, A, sai, sak, B, sbk, sbj, beta, C, sci,
                                       scj, lower_only ? 1 : 0, b_tri, 0, 0, 0, M, K);
  GW_CHECK_LAUNCH();
}

// batch GEMMs in one launch: member z (0 <= z < batch) is the product above with A, B and C
// offset by z * bsa, z * bsb, z * bsc elements; the last member has M_last rows and inner
// dimension K_last (<= M, K), every other member M rows and K.
static void gemm_f64_batched(cudaStream_t s, int batch, int M, int N, int K, double alpha,
                             const double* A, int64_t sai, int64_t sak, int64_t bsa,
                             const double* B, int64_t sbk, int64_t sbj, int64_t bsb, double beta,
                             double* C, int64_t sci, int64_t scj, int64_t bsc, int M_last,
                             int K_last, int b_tri) {
  if (batch <= 0 || M <= 0 || N <= 0) return;
  dim3 grid(ceil_div(N, GT), ceil_div(M, GT), batch);
  gemm_f64_kernel<<<grid, 256, 0, s>>>(M, N, K, alpha, A, sai, sak, B, sbk, sbj, beta, C, sci,
                                       scj, 0, b_tri, bsa, bsb, bsc, M_last, K_last);
  GW_CHECK_LAUNCH();
}

// ------------------------------------------------------------------------------------------
// M and its Cholesky factor
// ------------------------------------------------------------------------------------------
namespace {
__global__ void form_M_kernel(int n, const double* __restrict__ Phi, double h2, double s2,
                              double* __restrict__ A) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), c = (int)(e / n);  // column-major (i, c)
  // only the lower triangle of Phi is read; M is stored symmetric-lower
  const double phi = (i >= c) ? Phi[e] : Phi[c + (int64_t)i * n];
  A[e] = s2 * (h2 * phi + (i == c ? 1.0 - h2 : 0.0));
}

constexpr int NB = 32;

__global__ void potrf_diag_kernel(int n, double* A, int j0, int jb, int* flags) {
  __shared__ double a[NB][NB + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;  // (col, row)
  if (ty < jb && tx < jb) a[ty][tx] = A[(j0 + ty) + (int64_t)(j0 + tx) * n];
  for (int k = 0; k < jb; ++k) {
    __syncthreads();
    if (tx == 0 && ty == 0) {
      double d = a[k][k];
      if (!(d > 0.0) || !isfinite(d)) {
        atomicExch(&flags[FLAG_NOT_SPD], 1);
        d = 1.0;
      }
      a[k][k] = sqrt(d);
    }
    __syncthreads();
    if (tx == 0 && ty > k && ty < jb) a[ty][k] /= a[k][k];
    __syncthreads();
    if (ty > k && ty < jb && tx > k && tx <= ty) a[ty][tx] -= a[ty][k] * a[tx][k];
  }
  __syncthreads();
  if (ty < jb && tx < jb && tx <= ty) A[(j0 + ty) + (int64_t)(j0 + tx) * n] = a[ty][tx];
}

// Rows below the diagonal block: x L_jj^T = a, one thread per row.
__global__ void trsm_panel_kernel(int n, double* A, int j0, int jb) {
  __shared__ double L[NB][NB + 1];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    L[r][c] = (r < jb && c < jb) ? A[(j0 + r) + (int64_t)(j0 + c) * n] : 0.0;
  }
  __syncthreads();
  const int i = j0 + jb + blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    if (k < jb) {
      double v = A[i + (int64_t)(j0 + k) * n];
#pragma unroll
      for (int l = 0; l < k; ++l) v -= x[l] * L[k][l];
      x[k] = v / L[k][k];
      A[i + (int64_t)(j0 + k) * n] = x[k];
    } else {
      x[k] = 0.0;
    }
  }
}

__global__ void zero_upper_kernel(int n, double* A) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), c = (int)(e / n);
  if (c > i) A[e] = 0.0;
}
}  // namespace

void form_M(cudaStream_t s, int n, const double* Phi, double h2, double s2, double* A) {
  const int64_t nn = (int64_t)n * n;
  form_M_kernel<<<ceil_div(nn, 256), 256, 0, s>>>(n, Phi, h2, s2, A);
  GW_CHECK_LAUNCH();
}

void cholesky(cudaStream_t s, int n, double* A, int* flags) {
  for (int j0 = 0; j0 < n; j0 += NB) {
    const int jb = n - j0 < NB ? n - j0 : NB;
    potrf_diag_kernel<<<1, dim3(NB, NB), 0, s>>>(n, A, j0, jb, flags);
    GW_CHECK_LAUNCH();
    const int rest = n - j0 - jb;
    if (rest > 0) {
      trsm_panel_kernel<<<ceil_div(rest, 128), 128, 0, s>>>(n, A, j0, jb);
      GW_CHECK_LAUNCH();
      double* P = A + (j0 + jb) + (int64_t)j0 * n;
      gemm_f64(s, rest, rest, jb, -1.0, P, 1, n, P, n, 1, 1.0,
               A + (j0 + jb) + (int64_t)(j0 + jb) * n, 1, n, /*lower_only=*/true);
    }
  }
  const int64_t nn = (int64_t)n * n;
  zero_upper_kernel<<<ceil_div(nn, 256), 256, 0, s>>>(n, A);
  GW_CHECK_LAUNCH();
}

// ------------------------------------------------------------------------------------------
// L^-1 (row-major output)
// ------------------------------------------------------------------------------------------
namespace {
// Inverse of each 32 x 32 diagonal block; thread c computes column c by forward substitution.
__global__ void diag_inv_kernel(int n, const double* __restrict__ L, double* __restrict__ Linv) {
  __shared__ double Lb[NB][NB + 1];
  __shared__ double X[NB][NB + 1];
  const int j0 = blockIdx.x * NB;
  const int jb = n - j0 < NB ? n - j0 : NB;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    Lb[r][c] = (r < jb && c < jb) ? L[(j0 + r) + (int64_t)(j0 + c) * n] : 0.0;
    X[r][c] = 0.0;
  }
  __syncthreads();
  const int c = threadIdx.x;
  if (c < jb) {
    X[c][c] = 1.0 / Lb[c][c];
    for (int r = c + 1; r < jb; ++r) {
      double v = 0.0;
      for (int k = c; k < r; ++k) v += Lb[r][k] * X[k][c];
      X[r][c] = -v / Lb[r][r];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    const int r = e / jb, cc = e % jb;
    Linv[(int64_t)(j0 + r) * n + j0 + cc] = X[r][cc];
  }
}
}  // namespace

// Recursive doubling: with the inverses of the diagonal blocks [o, o + b) and [o + b, o + b + b2)
// known, the inverse of [[L11, 0], [L21, L22]] has the lower-left block -L22^-1 L21 L11^-1.  Level
// b = 32, 64, ... joins every aligned pair of b-blocks at once (one batched launch per product),
// so each level's products run side by side instead of one 32-row panel at a time.  work (n x n)
// holds T = L21 L11^-1 at the position of the block it becomes.
void tri_inverse(cudaStream_t s, int n, const double* L, double* Linv, double* work) {
  GW_CUDA(cudaMemsetAsync(Linv, 0, sizeof(double) * (size_t)n * n, s));
  const int nblk = ceil_div(n, NB);
  diag_inv_kernel<<<nblk, NB, 0, s>>>(n, L, Linv);
  GW_CHECK_LAUNCH();
  for (int b = NB; b < n; b *= 2) {
    const int pairs = ceil_div(n - b, 2 * b);  // pairs at o = 2 b p with o + b < n
    const int o_last = 2 * b * (pairs - 1);
    const int b2_last = n - o_last - b < b ? n - o_last - b : b;
    const int64_t bs = 2 * (int64_t)b * (n + 1);  // from one pair's blocks to the next
    // T (b2 x b, row-major in work) = L21 (column-major in L) * L11^-1 (lower triangular)
    gemm_f64_batched(s, pairs, b, b, b, 1.0, L + b, 1, n, bs, Linv, n, 1, bs, 0.0,
                     work + (int64_t)b * n, n, 1, bs, b2_last, b, /*b_tri=*/-1);
    // Linv21 (b2 x b) = -L22^-1 (b2 x b2) * T
    gemm_f64_batched(s, pairs, b, b, b, -1.0, Linv + (int64_t)b * n + b, n, 1, bs,
                     work + (int64_t)b * n, n, 1, bs, 0.0, Linv + (int64_t)b * n, n, 1, bs,
                     b2_last, b2_last, 0);
  }
}

// ------------------------------------------------------------------------------------------
// One-sided Jacobi eigendecomposition (Hestenes).  U starts as Phi, V as I; every round of a
// sweep orthogonalises n/2 disjoint column pairs (round-robin order), until no pair's cosine
// exceeds tol.  Then U = Phi V has orthogonal columns, so V diagonalises Phi^2 and, for SPD Phi,
// Phi; its columns are the eigenvectors.
// ------------------------------------------------------------------------------------------
namespace {
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32, nw = blockDim.x / 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < nw; ++i) t += red[i];
  return t;
}

__global__ void jacobi_init_kernel(int n, const double* __restrict__ Phi, double* U, double* V) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), c = (int)(e / n);
  U[e] = (i >= c) ? Phi[e] : Phi[c + (int64_t)i * n];
  V[e] = (i == c) ? 1.0 : 0.0;
}

__global__ void __launch_bounds__(256) jacobi_round_kernel(int n, int N, int round, double* U,
                                                           double* V, int* flags, double tol) {
  __shared__ double red[8];
  const int k = blockIdx.x;
  auto idx = [&](int x) { return (x + round) % (N - 1) + 1; };
  int a, b;
  if (k == 0) { a = 0; b = idx(0); } else { a = idx(k); b = idx(N - 1 - k); }
  if (a >= n || b >= n) return;  // the dummy player of an odd n
  double* ua = U + (int64_t)a * n;
  double* ub = U + (int64_t)b * n;
  double al = 0.0, be = 0.0, ga = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = ua[i], y = ub[i];
    al = fma(x, x, al);
    be = fma(y, y, be);
    ga = fma(x, y, ga);
  }
  al = block_sum(al, red);
  be = block_sum(be, red);
  ga = block_sum(ga, red);
  if (!(fabs(ga) > tol * sqrt(al * be))) return;
  if (threadIdx.x == 0) atomicAdd(&flags[FLAG_ROTATIONS], 1);
  const double zeta = (be - al) / (2.0 * ga);
  const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + tt * tt), sn = c * tt;
  double* va = V + (int64_t)a * n;
  double* vb = V + (int64_t)b * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double x = ua[i], y = ub[i];
    ua[i] = c * x - sn * y;
    ub[i] = sn * x + c * y;
    const double xv = va[i], yv = vb[i];
    va[i] = c * xv - sn * yv;
    vb[i] = sn * xv + c * yv;
  }
}

// Eigenvalue r as the Rayleigh quotient v_r^T Phi v_r = v_r^T u_r (keeps the sign, so an
// indefinite Phi is detected downstream).
__global__ void rayleigh_kernel(int n, const double* __restrict__ U, const double* __restrict__ V,
                                double* w) {
  __shared__ double red[8];
  const double* u = U + (int64_t)blockIdx.x * n;
  const double* v = V + (int64_t)blockIdx.x * n;
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a = fma(u[i], v[i], a);
  a = block_sum(a, red);
  if (threadIdx.x == 0) w[blockIdx.x] = a;
}
}  // namespace

int jacobi_eig(cudaStream_t s, int n, const double* Phi, double* Zt, double* w, double* U,
               int* flags, int max_sweeps) {
  const int64_t nn = (int64_t)n * n;
  jacobi_init_kernel<<<ceil_div(nn, 256), 256, 0, s>>>(n, Phi, U, Zt);
  GW_CHECK_LAUNCH();
  if (n == 1) {
    rayleigh_kernel<<<1, 256, 0, s>>>(n, U, Zt, w);
    GW_CHECK_LAUNCH();
    return 0;
  }
  const int N = n + (n & 1);
  const double tol = fmax(1e-15, 2.0 * n * 2.220446049250313e-16);
  // One sweep = N-1 rounds, captured once as a CUDA graph and replayed.
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  cudaStream_t cap;
  GW_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  GW_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  for (int r = 0; r < N - 1; ++r)
    jacobi_round_kernel<<<N / 2, 256, 0, cap>>>(n, N, r, U, Zt, flags, tol);
  cudaError_t le = cudaGetLastError();
  GW_CUDA(cudaStreamEndCapture(cap, &graph));
  GW_CUDA(le);
  GW_CUDA(cudaGraphInstantiate(&exec, graph, 0));
  int sweeps = -1;
  int* h_rot = nullptr;
  GW_CUDA(cudaMallocHost(&h_rot, sizeof(int)));
  for (int sw = 1; sw <= max_sweeps; ++sw) {
    GW_CUDA(cudaMemsetAsync(flags + FLAG_ROTATIONS, 0, sizeof(int), s));
    GW_CUDA(cudaGraphLaunch(exec, s));
    GW_CUDA(cudaMemcpyAsync(h_rot, flags + FLAG_ROTATIONS, sizeof(int), cudaMemcpyDeviceToHost, s));
    GW_CUDA(cudaStreamSynchronize(s));
    if (*h_rot == 0) { sweeps = sw; break; }
  }
  cudaFreeHost(h_rot);
  cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  rayleigh_kernel<<<n, 256, 0, s>>>(n, U, Zt, w);
  GW_CHECK_LAUNCH();
  return sweeps;
}

// ------------------------------------------------------------------------------------------
// Per-trait null-model block of the bordered system
// ------------------------------------------------------------------------------------------
namespace {
constexpr int QMAX = 7;
constexpr int NRED = QMAX * (QMAX + 1) / 2 + QMAX;

__global__ void __launch_bounds__(256) trait_pack_kernel(TraitPackArgs a) {
  __shared__ double red[NRED][8];
  __shared__ double sb0[QMAX];
  const int j = blockIdx.x, q = a.q, n = a.n;
  const double* xl = a.XLw + j * a.xlw_trait_stride;
  const double* y = a.yw + (int64_t)j * n;
  const double* d = a.d ? a.d + (int64_t)j * n : nullptr;
  double acc[NRED];
#pragma unroll
  for (int u = 0; u < NRED; ++u) acc[u] = 0.0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double dr = d ? d[r] : 1.0;
    double x[QMAX];
#pragma unroll
    for (int k = 0; k < QMAX; ++k) x[k] = k < q ? xl[(int64_t)k * n + r] : 0.0;
    int u = 0;
#pragma unroll
    for (int k = 0; k < QMAX; ++k)
#pragma unroll
      for (int l = 0; l <= k; ++l) acc[u++] += dr * x[k] * x[l];
#pragma unroll
    for (int k = 0; k < QMAX; ++k) acc[u++] += dr * x[k] * y[r];
  }
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
#pragma unroll
  for (int u = 0; u < NRED; ++u) {
    double v = acc[u];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (l == 0) red[u][w] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot[NRED];
    for (int u = 0; u < NRED; ++u) {
      double v = 0.0;
      for (int i = 0; i < (int)(blockDim.x / 32); ++i) v += red[u][i];
      tot[u] = v;
    }
    double S[QMAX][QMAX], bT[QMAX];
    int u = 0;
    for (int k = 0; k < QMAX; ++k)
      for (int l2 = 0; l2 <= k; ++l2) { S[k][l2] = tot[u]; S[l2][k] = tot[u]; ++u; }
    for (int k = 0; k < QMAX; ++k) bT[k] = tot[u++];
    // S = C C^T, then P = C^-T C^-1
    double C[QMAX][QMAX] = {}, Ci[QMAX][QMAX] = {};
    bool ok = true;
    for (int k = 0; k < q; ++k) {
      double dd = S[k][k];
      for (int m = 0; m < k; ++m) dd -= C[k][m] * C[k][m];
      if (!(dd > 1e-13 * S[k][k])) { ok = false; dd = 1.0; }
      C[k][k] = sqrt(dd);
      for (int i = k + 1; i < q; ++i) {
        double v = S[i][k];
        for (int m = 0; m < k; ++m) v -= C[i][m] * C[k][m];
        C[i][k] = v / C[k][k];
      }
    }
    if (!ok) atomicExch(&a.flags[FLAG_STL_SINGULAR], 1);
    for (int i = 0; i < q; ++i) {
      Ci[i][i] = 1.0 / C[i][i];
      for (int c = 0; c < i; ++c) {
        double v = 0.0;
        for (int m = c; m < i; ++m) v += C[i][m] * Ci[m][c];
        Ci[i][c] = -v / C[i][i];
      }
    }
    double* P = a.P + (int64_t)j * q * q;
    for (int i = 0; i < q; ++i)
      for (int c = 0; c < q; ++c) {
        double v = 0.0;
        for (int m = (i > c ? i : c); m < q; ++m) v += Ci[m][i] * Ci[m][c];
        P[i * q + c] = v;
      }
    for (int i = 0; i < q; ++i) {
      double v = 0.0;
      for (int c = 0; c < q; ++c) v += P[i * q + c] * bT[c];
      sb0[i] = v;
      a.b0[(int64_t)j * q + i] = v;
    }
  }
  __syncthreads();
  double* rw = a.rw + (int64_t)j * n;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    double v = y[r];
    for (int k = 0; k < q; ++k) v -= xl[(int64_t)k * n + r] * sb0[k];
    rw[r] = (d ? d[r] : 1.0) * v;
  }
}

__global__ void eig_weights_kernel(int n, int t, const double* __restrict__ w,
                                   const double* __restrict__ h2, const double* __restrict__ s2,
                                   double* __restrict__ d, int* flags) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * t) return;
  const int j = (int)(e / n), r = (int)(e % n);
  const double v = s2[j] * (h2[j] * w[r] + (1.0 - h2[j]));
  if (!(v > 0.0)) atomicExch(&flags[FLAG_NOT_SPD], 1);  // M_j = Z diag(v) Z^T not SPD
  d[e] = v > 0.0 ? 1.0 / v : 0.0;
}

__global__ void eig_planes_kernel(int n, int q, int t, int ldp, const double* __restrict__ XLt,
                                  const double* __restrict__ d, const double* __restrict__ rw,
                                  double* __restrict__ planes) {
  const int64_t total = (int64_t)t * (q + 2) * ldp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e % ldp);
    const int64_t row = e / ldp;
    const int c = (int)(row % (q + 2));
    const int j = (int)(row / (q + 2));
    double v = 0.0;
    if (r < n) {
      const double dr = d[(int64_t)j * n + r];
      if (c < q) v = dr * XLt[(int64_t)c * n + r];
      else if (c == q) v = rw[(int64_t)j * n + r];
      else v = dr;
    }
    planes[e] = v;
  }
}

__global__ void f64_to_f32_kernel(const double* __restrict__ x, float* __restrict__ y,
                                  int64_t count) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    y[e] = (float)x[e];
}

// x = hi + lo (+ lo2): each piece the BF16 rounding of what the previous pieces leave; lo2 may
// be NULL (two pieces, ~16 significant bits; three carry ~24).
__device__ __forceinline__ void split_store(double v, int64_t e, __nv_bfloat16* hi,
                                            __nv_bfloat16* lo, __nv_bfloat16* lo2) {
  const __nv_bfloat16 h = __double2bfloat16(v);
  const double r1 = v - (double)__bfloat162float(h);
  const __nv_bfloat16 l = __double2bfloat16(r1);
  hi[e] = h;
  lo[e] = l;
  if (lo2) lo2[e] = __double2bfloat16(r1 - (double)__bfloat162float(l));
}

__global__ void split_bf16_kernel(const double* __restrict__ x, int rows, int cols, int64_t ldx,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo,
                                  __nv_bfloat16* __restrict__ lo2, int64_t ldo) {
  const int64_t total = (int64_t)rows * ldo;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / ldo), c = (int)(e % ldo);
    const double v = c < cols ? x[(int64_t)r * ldx + c] : 0.0;
    split_store(v, e, hi, lo, lo2);
  }
}

__global__ void split_bf16_rows_kernel(const double* __restrict__ x, int rows, int cols,
                                       int64_t ldx, int gin, int gout, int off,
                                       __nv_bfloat16* __restrict__ hi,
                                       __nv_bfloat16* __restrict__ lo,
                                       __nv_bfloat16* __restrict__ lo2, int64_t ldo) {
  const int64_t total = (int64_t)rows * ldo;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ldo;
    const int c = (int)(e % ldo);
    const int64_t src = (r / gout) * gin + r % gout + off;
    const double v = c < cols ? x[src * ldx + c] : 0.0;
    split_store(v, e, hi, lo, lo2);
  }
}
}  // namespace

void split_bf16_rows(cudaStream_t s, const double* x, int rows, int cols, int64_t ldx, int gin,
                     int gout, int off, __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ldo,
                     __nv_bfloat16* lo2) {
  split_bf16_rows_kernel<<<1184, 256, 0, s>>>(x, rows, cols, ldx, gin, gout, off, hi, lo, lo2,
                                              ldo);
  GW_CHECK_LAUNCH();
}

void trait_pack(cudaStream_t s, const TraitPackArgs& a) {
  GW_REQUIRE(a.q >= 1 && a.q <= QMAX, GWAS_ERR_ARG, "q=%d outside [1,%d]", a.q, QMAX);
  trait_pack_kernel<<<a.t, 256, 0, s>>>(a);
  GW_CHECK_LAUNCH();
}

void eig_weights(cudaStream_t s, int n, int t, const double* w, const double* h2,
                 const double* s2, double* d, int* flags) {
  const int64_t tot = (int64_t)n * t;
  eig_weights_kernel<<<ceil_div(tot, 256), 256, 0, s>>>(n, t, w, h2, s2, d, flags);
  GW_CHECK_LAUNCH();
}

void eig_planes_f64(cudaStream_t s, int n, int q, int t, int ldp, const double* XLt,
                    const double* d, const double* rw, double* planes) {
  eig_planes_kernel<<<1184, 256, 0, s>>>(n, q, t, ldp, XLt, d, rw, planes);
  GW_CHECK_LAUNCH();
}

void convert_f64_to_f32(cudaStream_t s, const double* x, float* y, int64_t count) {
  if (count <= 0) return;
  f64_to_f32_kernel<<<1184, 256, 0, s>>>(x, y, count);
  GW_CHECK_LAUNCH();
}

namespace {

// One power-iteration step: rq[0] = v . y (the Rayleigh quotient of unit v), then v = y / |y|.
__global__ void power_step_kernel(int n, double* __restrict__ v, const double* __restrict__ y,
                                  double* __restrict__ rq) {
  __shared__ double red[2][32];
  double vy = 0.0, yy = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    vy += v[i] * y[i];
    yy += y[i] * y[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    vy += __shfl_xor_sync(0xffffffffu, vy, o);
    yy += __shfl_xor_sync(0xffffffffu, yy, o);
  }
  if (threadIdx.x % 32 == 0) {
    red[0][threadIdx.x / 32] = vy;
    red[1][threadIdx.x / 32] = yy;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    vy = threadIdx.x < blockDim.x / 32 ? red[0][threadIdx.x] : 0.0;
    yy = threadIdx.x < blockDim.x / 32 ? red[1][threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      vy += __shfl_xor_sync(0xffffffffu, vy, o);
      yy += __shfl_xor_sync(0xffffffffu, yy, o);
    }
    if (threadIdx.x == 0) {
      red[0][0] = vy;
      red[1][0] = yy > 0.0 ? rsqrt(yy) : 0.0;
    }
  }
  __syncthreads();
  const double inv = red[1][0];
  if (threadIdx.x == 0) rq[0] = red[0][0];
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = y[i] * inv;
}

// y = A x for an n x n matrix whose rows are contiguous (A(i, k) = A[i * n + k]): one warp per
// output, coalesced along the row.
__global__ void gemv_rows_kernel(int n, const double* __restrict__ A, const double* __restrict__ x,
                                 double* __restrict__ y) {
  const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
  if (i >= n) return;  // warp-uniform
  const double* row = A + (int64_t)i * n;
  double acc = 0.0;
  for (int k = lane; k < n; k += 32) acc += row[k] * x[k];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) y[i] = acc;
}

// y = A x for an n x n matrix whose columns are contiguous (A(i, k) = A[i + k * n]): one thread
// per output, consecutive threads reading consecutive elements of each column.
__global__ void gemv_cols_kernel(int n, const double* __restrict__ A, const double* __restrict__ x,
                                 double* __restrict__ y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = 0.0;
  for (int k = 0; k < n; ++k) acc += A[i + (int64_t)k * n] * x[k];
  y[i] = acc;
}

__global__ void power_start_kernel(int n, double* __restrict__ v) {
  const double inv = rsqrt((double)n);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    v[i] = inv * (1.0 + 0.25 * (double)((i * 7919) % 13) / 13.0);  // a start with every component
}

}  // namespace

double condition_estimate(cudaStream_t s, int n, const double* L, const double* Linv,
                          double* work, int iters) {
  double* v = work;
  double* y = work + n;
  double* z = work + 2 * n;
  double* rq = work + 3 * n;
  double lam[2] = {0.0, 0.0};
  for (int which = 0; which < 2; ++which) {
    power_start_kernel<<<ceil_div(n, 256), 256, 0, s>>>(n, v);
    GW_CHECK_LAUNCH();
    for (int it = 0; it < iters; ++it) {
      const unsigned gw = (unsigned)ceil_div(n, 8), gt = (unsigned)ceil_div(n, 256);
      if (which == 0) {  // M v = L (L^T v); L column-major: L^T has contiguous rows
        gemv_rows_kernel<<<gw, 256, 0, s>>>(n, L, v, y);
        gemv_cols_kernel<<<gt, 256, 0, s>>>(n, L, y, z);
      } else {  // M^-1 v = L^-T (L^-1 v); L^-1 row-major: L^-T has contiguous columns
        gemv_rows_kernel<<<gw, 256, 0, s>>>(n, Linv, v, y);
        gemv_cols_kernel<<<gt, 256, 0, s>>>(n, Linv, y, z);
      }
      GW_CHECK_LAUNCH();
      power_step_kernel<<<1, 1024, 0, s>>>(n, v, z, rq);
      GW_CHECK_LAUNCH();
    }
    GW_CUDA(cudaMemcpyAsync(&lam[which], rq, sizeof(double), cudaMemcpyDeviceToHost, s));
    GW_CUDA(cudaStreamSynchronize(s));
  }
  return lam[0] * lam[1];  // lam_max(M) lam_max(M^-1) = lam_max(M) / lam_min(M)
}

void split_bf16(cudaStream_t s, const double* x, int rows, int cols, int64_t ldx,
                __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t ldo, __nv_bfloat16* lo2) {
  split_bf16_kernel<<<1184, 256, 0, s>>>(x, rows, cols, ldx, hi, lo, lo2, ldo);
  GW_CHECK_LAUNCH();
}

namespace {

__global__ void rowmax_abs_kernel(const double* __restrict__ x, int cols, int64_t ldx,
                                  double* __restrict__ out) {
  __shared__ double red[32];
  const double* row = x + (int64_t)blockIdx.x * ldx;
  double v = 0.0;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) v = fmax(v, fabs(row[c]));
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) out[blockIdx.x] = v;
  }
}

// the position of column c in the lo matrix: e4m3_k_slot order within its group of 16
__device__ __forceinline__ int64_t e4m3_col(int c) { return (c & ~15) | tc::e4m3_k_slot(c & 15); }

__global__ void split_f16_e4m3_kernel(const double* __restrict__ x, int rows, int cols,
                                      int64_t ldx, const double* __restrict__ rscale,
                                      __half* __restrict__ hi, uint8_t* __restrict__ lo,
                                      int64_t ldo) {
  const int64_t total = (int64_t)rows * ldo;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / ldo;
    const int c = (int)(e % ldo);
    const double v = c < cols ? x[r * ldx + c] * rscale[r] : 0.0;
    const __half h = __double2half(v);
    const double rem = v - (double)__half2float(h);
    hi[r * ldo + e4m3_col(c)] = h;
    lo[r * ldo + e4m3_col(c)] = (uint8_t)__nv_cvt_double_to_fp8(rem, __NV_SATFINITE, __NV_E4M3);
  }
}

__device__ __forceinline__ double e4m3_value(uint8_t b) {
  const __half_raw hr = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)b, __NV_E4M3);
  return (double)__half2float(__half(hr));
}

__global__ void e4m3_weighted_col_sums_kernel(const __half* __restrict__ hi,
                                              const uint8_t* __restrict__ lo, int rows,
                                              int64_t ldo, int cols, const float* __restrict__ ls,
                                              double* __restrict__ w) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < cols; c += gridDim.x * blockDim.x) {
    const int64_t pos = e4m3_col(c);
    double acc = 0.0;
    for (int r = 0; r < rows; ++r)
      acc += (double)ls[r] * ((double)__half2float(hi[r * ldo + pos]) + e4m3_value(lo[r * ldo + pos]));
    w[c] = acc;
  }
}

__global__ void e4m3_row_sums_kernel(const uint8_t* __restrict__ lo, int64_t ldo,
                                     float* __restrict__ out) {
  __shared__ double red[32];
  const uint8_t* row = lo + (int64_t)blockIdx.x * ldo;
  double v = 0.0;
  for (int64_t c = threadIdx.x; c < ldo; c += blockDim.x) v += e4m3_value(row[c]);
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) out[blockIdx.x] = (float)v;
  }
}

}  // namespace

void rowmax_abs(cudaStream_t s, const double* x, int rows, int cols, int64_t ldx, double* out) {
  if (rows <= 0) return;
  rowmax_abs_kernel<<<rows, 256, 0, s>>>(x, cols, ldx, out);
  GW_CHECK_LAUNCH();
}

void split_f16_e4m3(cudaStream_t s, const double* x, int rows, int cols, int64_t ldx,
                    const double* rscale, __half* hi, uint8_t* lo, int64_t ldo) {
  GW_REQUIRE(ldo % 16 == 0 && cols <= ldo, GWAS_ERR_ARG, "FP8 split: bad leading dimension");
  split_f16_e4m3_kernel<<<1184, 256, 0, s>>>(x, rows, cols, ldx, rscale, hi, lo, ldo);
  GW_CHECK_LAUNCH();
}

void e4m3_weighted_col_sums(cudaStream_t s, const __half* hi, const uint8_t* lo, int rows,
                            int64_t ldo, int cols, const float* ls, double* w) {
  if (cols <= 0) return;
  e4m3_weighted_col_sums_kernel<<<ceil_div(cols, 128), 128, 0, s>>>(hi, lo, rows, ldo, cols, ls, w);
  GW_CHECK_LAUNCH();
}

void e4m3_row_sums(cudaStream_t s, const uint8_t* lo, int rows, int64_t ldo, float* out) {
  if (rows <= 0) return;
  e4m3_row_sums_kernel<<<rows, 256, 0, s>>>(lo, ldo, out);
  GW_CHECK_LAUNCH();
}

}  // namespace gw
