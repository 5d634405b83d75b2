// Plain CUDA-core forms (FP64 and FP32) of the per-SNP scan.
//
// CHOL (Algorithm 3, per SNP block): for a block of SNPs, X' = L^-1 X_R is formed tile by
// tile (lower-triangular tiles of L^-1 only) and immediately reduced to the bordered-system
// entries a = X_L'^T x', c = r'^T x', s = x'^T x' of each SNP; X' never reaches memory.
//
// EIG (Algorithm 4, per SNP block): X~ = Z^T X_R is written to scratch, then every
// (SNP, trait) pair reduces X~ against the trait planes E_k = d_j o X~_L[:,k], F = d_j o r~_j,
// Dm = d_j:  a_k = <x~, E_k>, c = <x~, F>, s = <x~ o x~, Dm>.
//
// Both end in the same Schur-complement solve of the bordered p x p system
//   [[S_TL, a], [a^T, s]] [b_L; b_s] = [b_T; x^T M^-1 y]:
//   v = P a (P = S_TL^-1), sigma = s - a^T v, b_s = c / sigma, b_L = b0 - v b_s,
//   wald = b_s^2 sigma  (= b_s^2 / Var(b_s) with Var(b_s) = 1 / sigma),
// where c uses the null residual r = y - X_L b0, so that c = x^T M^-1 y - a^T b0 without the
// cancellation of forming the two terms separately.
#include "common.cuh"

namespace gw {
namespace {

constexpr int QMAX = 7;
constexpr int TS = 64;  // SNPs per tile
constexpr int TR = 64;  // rows (individuals) per tile
constexpr int TK = 16;  // reduction chunk

template <typename T>
__device__ __forceinline__ void schur_store(int q, const T* __restrict__ P, const T* __restrict__ b0,
                                            const T* a, T c, T s, T tol, int64_t i, int j, int t,
                                            void* B, void* wald, bool out_f64, int* flags,
                                            int out_snp, int out_var) {
  const int p = q + 1;
  T v[QMAX];
  T aPa = 0;
#pragma unroll
  for (int k = 0; k < QMAX; ++k) {
    T acc = 0;
    if (k < q) {
#pragma unroll
      for (int l = 0; l < QMAX; ++l)
        if (l < q) acc += P[k * q + l] * a[l];
      aPa += a[k] * acc;
    }
    v[k] = acc;
  }
  const T sigma = s - aPa;
  T out[QMAX + 1];
  T w;
  if (sigma > tol * s) {
    const T bs = c / sigma;
#pragma unroll
    for (int k = 0; k < QMAX; ++k)
      if (k < q) out[k] = b0[k] - v[k] * bs;
    out[q] = bs;
    w = bs * c;
  } else {
    const T nanv = (T)NAN;
#pragma unroll
    for (int k = 0; k <= QMAX; ++k) out[k] = nanv;
    w = nanv;
    atomicAdd(&flags[FLAG_SINGULAR], 1);
  }
  if (out_snp) {  // (b_snp, standard error 1 / sqrt(sigma)) per pair
    const T se = sigma > tol * s ? (T)1 / sqrt(sigma) : (T)NAN;
    out[0] = out[q];
    out[1] = se;
  }
  const int pw = out_snp ? 2 : out_var ? p + p * (p + 1) / 2 : p;
  const int64_t o = (i * t + j) * pw;
  if (out_f64) {
    double* Bd = (double*)B;
#pragma unroll
    for (int k = 0; k <= QMAX; ++k)
      if (k < (out_snp ? 2 : p)) Bd[o + k] = (double)out[k];
    if (wald) ((double*)wald)[i * t + j] = (double)w;
  } else {
    float* Bf = (float*)B;
#pragma unroll
    for (int k = 0; k <= QMAX; ++k)
      if (k < (out_snp ? 2 : p)) Bf[o + k] = (float)out[k];
    if (wald) ((float*)wald)[i * t + j] = (float)w;
  }
  if (out_var) {
    // Var(b) = S^-1 of the bordered S = [[S_TL, a], [a^T, s]]: [[P + v v^T / sigma, -v / sigma],
    // [-v^T / sigma, 1 / sigma]], packed upper triangle row by row after the p coefficients
    // (constant loop bounds keep v[] in registers)
    const bool ok = sigma > tol * s;
    const T inv = ok ? (T)1 / sigma : (T)NAN;
#pragma unroll
    for (int r = 0; r <= QMAX; ++r)
#pragma unroll
      for (int cc = r; cc <= QMAX; ++cc) {
        if (r >= p || cc >= p) continue;
        const int e = p + r * p - r * (r - 1) / 2 + (cc - r);
        const T vr = v[r < QMAX ? r : QMAX - 1], vcc = v[cc < QMAX ? cc : QMAX - 1];
        T vrc;
        if (cc < q)
          vrc = P[r * q + cc] + vr * vcc * inv;
        else if (r < q)
          vrc = -vr * inv;
        else
          vrc = inv;
        if (!ok) vrc = (T)NAN;
        if (out_f64)
          ((double*)B)[o + e] = (double)vrc;
        else
          ((float*)B)[o + e] = (float)vrc;
      }
  }
}

// ------------------------------------------------------------------------------------------
// CHOL: fused whiten-and-reduce, one CTA per 64 SNPs
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) chol_scan_kernel(CholScanArgs<T> a) {
  __shared__ T Ls[TK][TR + 1];
  __shared__ T Xs[TK][TS + 1];
  __shared__ T Rs[QMAX + 1][TR];
  __shared__ T red[16][TS + 1];
  __shared__ T res[QMAX + 2][TS];
  const int n = a.n, q = a.q;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t s0 = (int64_t)blockIdx.x * TS;
  T ps[4] = {}, pc[4] = {}, pa[4][QMAX] = {};
  for (int r0 = 0; r0 < n; r0 += TR) {
    const int kend = min(n, r0 + TR);
    T acc[4][4] = {};
    for (int k0 = 0; k0 < kend; k0 += TK) {
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int e = tid + 256 * l, k = e % TK, i = e / TK;
        const int gr = r0 + i, gk = k0 + k;
        Ls[k][i] = (gr < n && gk < n) ? a.Linv[(int64_t)gr * n + gk] : T(0);
        const int64_t gs = s0 + i;
        Xs[k][i] = (gs < a.m && gk < n) ? (T)a.XR[gs * n + gk] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < TK; ++k) {
        T lv[4], xv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { lv[u] = Ls[k][ty + 16 * u]; xv[u] = Xs[k][tx + 16 * u]; }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] += lv[u] * xv[v];
      }
      __syncthreads();
    }
    // per-row data of this row tile: whitened covariates and null residual
    for (int e = tid; e < (q + 1) * TR; e += 256) {
      const int c = e / TR, i = e % TR, gr = r0 + i;
      Rs[c][i] = gr < n ? (c < q ? a.XLw[(int64_t)c * n + gr] : a.rw[gr]) : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = ty + 16 * u;
      const T rr = Rs[q][i];
      T xl[QMAX];
#pragma unroll
      for (int k = 0; k < QMAX; ++k) xl[k] = k < q ? Rs[k][i] : T(0);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const T x = acc[u][v];
        ps[v] += x * x;
        pc[v] += rr * x;
#pragma unroll
        for (int k = 0; k < QMAX; ++k) pa[v][k] += xl[k] * x;
      }
    }
    __syncthreads();
  }
  // reduce the 16 row-groups of each SNP
  for (int slot = 0; slot < q + 2; ++slot) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T val;
      if (slot < q) {
        val = T(0);
#pragma unroll
        for (int k = 0; k < QMAX; ++k)
          if (k == slot) val = pa[v][k];
      } else {
        val = slot == q ? pc[v] : ps[v];
      }
      red[ty][tx + 16 * v] = val;
    }
    __syncthreads();
    if (tid < TS) {
      T sum = 0;
      for (int g = 0; g < 16; ++g) sum += red[g][tid];
      res[slot][tid] = sum;
    }
    __syncthreads();
  }
  if (tid < TS && s0 + tid < a.m) {
    T av[QMAX];
#pragma unroll
    for (int k = 0; k < QMAX; ++k) av[k] = k < q ? res[k][tid] : T(0);
    schur_store<T>(q, a.P, a.b0, av, res[q][tid], res[q + 1][tid], a.sing_tol,
                   a.out_offset + s0 + tid, a.j, a.t, a.B, a.wald, a.out_f64, a.flags, a.out_snp,
                   a.out_var);
  }
}

// ------------------------------------------------------------------------------------------
// EIG stage 1: X~ = Z^T X_R into scratch (SNP-major, leading dimension ldp)
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) eig_rotate_kernel(int n, int ldp, const T* __restrict__ Zt,
                                                         const int8_t* __restrict__ XR, int64_t m,
                                                         T* __restrict__ xt) {
  __shared__ T Zs[TK][TR + 1];
  __shared__ T Xs[TK][TS + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int r0 = blockIdx.x * TR;
  const int64_t s0 = (int64_t)blockIdx.y * TS;
  T acc[4][4] = {};  // [snp u][row v]
  for (int k0 = 0; k0 < n; k0 += TK) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = tid + 256 * l, k = e % TK, i = e / TK;
      const int gr = r0 + i, gk = k0 + k;
      Zs[k][i] = (gr < n && gk < n) ? Zt[(int64_t)gr * n + gk] : T(0);
      const int64_t gs = s0 + i;
      Xs[k][i] = (gs < m && gk < n) ? (T)XR[gs * n + gk] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < TK; ++k) {
      T xv[4], zv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { xv[u] = Xs[k][ty + 16 * u]; zv[u] = Zs[k][tx + 16 * u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += xv[u] * zv[v];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t gs = s0 + ty + 16 * u;
    if (gs >= m) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int gr = r0 + tx + 16 * v;
      if (gr < ldp) xt[gs * ldp + gr] = gr < n ? acc[u][v] : T(0);
    }
  }
}

// ------------------------------------------------------------------------------------------
// EIG stage 2: trait-batched reduction + Schur, one CTA per 64 SNPs x 16 traits
// ------------------------------------------------------------------------------------------
constexpr int TT = 16;

template <typename T>
__global__ void __launch_bounds__(256) eig_reduce_kernel(EigScanArgs<T> a) {
  __shared__ T Xs[TK][TS + 1];
  __shared__ T Ps[TK][TT * (QMAX + 2) + 1];
  const int n = a.n, q = a.q, qc = q + 2, t = a.t;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t s0 = (int64_t)blockIdx.x * TS;
  const int j0 = blockIdx.y * TT;
  const int j = j0 + ty;
  T acc[4][QMAX + 2] = {};
  for (int k0 = 0; k0 < n; k0 += TK) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = tid + 256 * l, k = e % TK, i = e / TK;
      const int64_t gs = s0 + i;
      Xs[k][i] = (gs < a.m && k0 + k < n) ? a.xt[gs * a.ldp + k0 + k] : T(0);
    }
    for (int e = tid; e < TK * TT * qc; e += 256) {
      const int k = e % TK, row = e / TK;
      const int jj = j0 + row / qc;
      Ps[k][row] = (jj < t && k0 + k < n) ? a.planes[((int64_t)j0 * qc + row) * a.ldp + k0 + k] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < TK; ++k) {
      T xv[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) xv[u] = Xs[k][tx + 16 * u];
      const T* pr = &Ps[k][ty * qc];
#pragma unroll
      for (int c = 0; c < QMAX + 1; ++c) {
        if (c < q + 1) {
          const T pv = pr[c];
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u][c] += xv[u] * pv;
        }
      }
      const T dm = pr[q + 1];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u][QMAX + 1] += xv[u] * xv[u] * dm;
    }
    __syncthreads();
  }
  if (j >= t) return;
  const T* P = a.P + (int64_t)j * q * q;
  const T* b0 = a.b0 + (int64_t)j * q;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int64_t gs = s0 + tx + 16 * u;
    if (gs >= a.m) continue;
    T av[QMAX];
#pragma unroll
    for (int k = 0; k < QMAX; ++k) av[k] = k < q ? acc[u][k] : T(0);
    T c = 0;
#pragma unroll
    for (int k = 0; k < QMAX + 1; ++k)
      if (k == q) c = acc[u][k];
    schur_store<T>(q, P, b0, av, c, acc[u][QMAX + 1], a.sing_tol, a.out_offset + gs, j, t, a.B,
                   a.wald, a.out_f64, a.flags, a.out_snp, a.out_var);
  }
}

__global__ void validate_kernel(const int8_t* __restrict__ XR, int64_t count, int* flags) {
  bool bad = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x)
    bad |= (uint8_t)XR[e] > 2;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(&flags[FLAG_GENOTYPE], 1);
}

}  // namespace

template <typename T>
void chol_scan_simt(cudaStream_t s, const CholScanArgs<T>& a) {
  if (a.m <= 0) return;
  GW_REQUIRE(a.q >= 1 && a.q <= QMAX, GWAS_ERR_ARG, "q=%d outside [1,%d]", a.q, QMAX);
  chol_scan_kernel<T><<<ceil_div(a.m, TS), 256, 0, s>>>(a);
  GW_CHECK_LAUNCH();
}

template <typename T>
void eig_scan_simt(cudaStream_t s, const EigScanArgs<T>& a) {
  if (a.m <= 0) return;
  GW_REQUIRE(a.q >= 1 && a.q <= QMAX, GWAS_ERR_ARG, "q=%d outside [1,%d]", a.q, QMAX);
  GW_REQUIRE(a.m <= (int64_t)65535 * TS, GWAS_ERR_ARG, "block of %lld SNPs too large", (long long)a.m);
  dim3 g1(ceil_div(a.ldp, TR), ceil_div(a.m, TS));
  eig_rotate_kernel<T><<<g1, 256, 0, s>>>(a.n, a.ldp, a.Zt, a.XR, a.m, a.xt);
  GW_CHECK_LAUNCH();
  GW_REQUIRE(ceil_div(a.t, TT) <= 65535, GWAS_ERR_ARG, "t=%d too large", a.t);
  dim3 g2(ceil_div(a.m, TS), ceil_div(a.t, TT));
  eig_reduce_kernel<T><<<g2, 256, 0, s>>>(a);
  GW_CHECK_LAUNCH();
}

template void chol_scan_simt<double>(cudaStream_t, const CholScanArgs<double>&);
template void chol_scan_simt<float>(cudaStream_t, const CholScanArgs<float>&);
template void eig_scan_simt<double>(cudaStream_t, const EigScanArgs<double>&);
template void eig_scan_simt<float>(cudaStream_t, const EigScanArgs<float>&);

void validate_genotypes(cudaStream_t s, const int8_t* XR, int64_t count, int* flags) {
  if (count <= 0) return;
  validate_kernel<<<1184, 256, 0, s>>>(XR, count, flags);
  GW_CHECK_LAUNCH();
}

}  // namespace gw
