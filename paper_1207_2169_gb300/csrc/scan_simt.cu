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
// cancellation of forming the two terms separately.  A genetic model of two columns per SNP
// (X_R,i = [x, x == 1], say) makes a, c and s a q x 2 block, a 2-vector and a 2 x 2 block, and
// the solve a 2 x 2 Schur complement (schur_store).
#include "common.cuh"

namespace gw {
namespace {

constexpr int QMAX = 7;
constexpr int TS = 64;  // SNPs per tile
constexpr int TR = 64;  // rows (individuals) per tile
constexpr int TK = 16;  // reduction chunk

// The bordered solve of one pair for a genetic block of pr <= 2 columns (in the model's working
// basis, see GeneticModel):
//   a[r][k] = X_R,r^T M^-1 X_L[:,k],  c[r] = X_R,r^T M^-1 r0,  S[0..2] = (S_00, S_01, S_11) of
//   S_RR = X_R^T M^-1 X_R (S[1], S[2] unused when pr = 1);
//   V = P A (q x pr), Sigma = S_RR - A^T V, b_w = Sigma^-1 c, b_L = b0 - V b_w,
//   wald = c^T Sigma^-1 c = b_w . c (pr d.o.f.),  Var(b) = [[P + V Sigma^-1 V^T, -V Sigma^-1],
//   [-Sigma^-1 V^T, Sigma^-1]];
// the genetic coefficients and their rows and columns of Var are reported as b_R = tm b_w,
// Var_RR = tm Sigma^-1 tm^T, Var_LR = -V Sigma^-1 tm^T.
// Singular (NaN outputs, counted) when a pivot of Sigma's Cholesky falls to <= tol times the
// matching diagonal entry of S_RR -- the pivots of the full p x p Cholesky for the last rows.
template <typename T>
__device__ __forceinline__ void schur_store(int q, const GeneticModel& gm, const T* __restrict__ P,
                                            const T* __restrict__ b0, const T (*a)[QMAX],
                                            const T* c, const T* S, T tol, int64_t i, int j, int t,
                                            void* B, void* wald, bool out_f64, int* flags,
                                            int out_snp, int out_var) {
  const int pr = gm.pr;
  const int p = q + pr;
  T v[2][QMAX];
  T sg[2][2];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
#pragma unroll
    for (int k = 0; k < QMAX; ++k) {
      T acc = 0;
      if (k < q && r < pr) {
#pragma unroll
        for (int l = 0; l < QMAX; ++l)
          if (l < q) acc += P[k * q + l] * a[r][l];
      }
      v[r][k] = acc;
    }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      T acc = 0;
#pragma unroll
      for (int k = 0; k < QMAX; ++k)
        if (k < q) acc += a[r][k] * v[u][k];
      sg[r][u] = (r == 0 ? (u == 0 ? S[0] : S[1]) : (u == 0 ? S[1] : S[2])) - acc;
    }
  // Sigma^-1 (pr = 1: 1 / sigma; pr = 2: the 2 x 2 inverse) after the pivot test
  T si[2][2] = {{0, 0}, {0, 0}};
  bool ok;
  if (pr == 1) {
    ok = sg[0][0] > tol * S[0];
    si[0][0] = (T)1 / sg[0][0];
  } else {
    const T piv1 = sg[1][1] - sg[0][1] * sg[0][1] / sg[0][0];
    ok = sg[0][0] > tol * S[0] && piv1 > tol * S[2];
    const T det = sg[0][0] * piv1;  // = sigma00 sigma11 - sigma01^2
    si[0][0] = sg[1][1] / det;
    si[1][1] = sg[0][0] / det;
    si[0][1] = si[1][0] = -sg[0][1] / det;
  }
  // the map to the reported basis (identity for one column)
  const T tm[2][2] = {{(T)gm.tm[0][0], (T)gm.tm[0][1]}, {(T)gm.tm[1][0], (T)gm.tm[1][1]}};
  T out[QMAX + 4];
  T w;
  T bw[2] = {0, 0};
  if (ok) {
#pragma unroll
    for (int r = 0; r < 2; ++r)
      if (r < pr) bw[r] = si[r][0] * c[0] + (pr > 1 ? si[r][1] * c[1] : (T)0);
#pragma unroll
    for (int k = 0; k < QMAX; ++k)
      if (k < q) out[k] = b0[k] - v[0][k] * bw[0] - (pr > 1 ? v[1][k] * bw[1] : (T)0);
    if (pr == 1) {
      out[q] = bw[0];
    } else {
      out[q] = tm[0][0] * bw[0] + tm[0][1] * bw[1];
      out[q + 1] = tm[1][0] * bw[0] + tm[1][1] * bw[1];
    }
    w = bw[0] * c[0] + (pr > 1 ? bw[1] * c[1] : (T)0);
  } else {
    const T nanv = (T)NAN;
#pragma unroll
    for (int k = 0; k < QMAX + 4; ++k) out[k] = nanv;
    w = nanv;
    atomicAdd(&flags[FLAG_SINGULAR], 1);
  }
  // Var_RR in the reported basis: vr[g][h] = (tm Sigma^-1 tm^T)[g][h]
  T vr[2][2];
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      T acc = 0;
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int z = 0; z < 2; ++z)
          if (u < pr && z < pr) acc += (pr == 1 ? (T)1 : tm[g][u]) * si[u][z] * (pr == 1 ? (T)1 : tm[hh][z]);
      vr[g][hh] = acc;
    }
  if (out_snp) {  // (b_R, standard errors sqrt(diag Var_RR)) per pair
    const T b0v = out[q], b1v = out[q + 1 < QMAX + 4 ? q + 1 : 0];
    out[0] = b0v;
    if (pr > 1) out[1] = b1v;
    out[pr] = ok ? sqrt(vr[0][0]) : (T)NAN;
    if (pr > 1) out[pr + 1] = ok ? sqrt(vr[1][1]) : (T)NAN;
  }
  const int nb = out_snp ? 2 * pr : p;
  const int pw = out_snp ? 2 * pr : out_var ? p + p * (p + 1) / 2 : p;
  const int64_t o = (i * t + j) * pw;
  if (out_f64) {
    double* Bd = (double*)B;
#pragma unroll
    for (int k = 0; k < QMAX + 2; ++k)
      if (k < nb) Bd[o + k] = (double)out[k];
    if (wald) ((double*)wald)[i * t + j] = (double)w;
  } else {
    float* Bf = (float*)B;
#pragma unroll
    for (int k = 0; k < QMAX + 2; ++k)
      if (k < nb) Bf[o + k] = (float)out[k];
    if (wald) ((float*)wald)[i * t + j] = (float)w;
  }
  if (out_var) {
    // packed upper triangle row by row after the p coefficients; rows/cols < q are X_L's,
    // q + g the reported genetic column g (constant loop bounds keep v[] in registers)
#pragma unroll
    for (int r = 0; r < QMAX + 2; ++r)
#pragma unroll
      for (int cc = r; cc < QMAX + 2; ++cc) {
        if (r >= p || cc >= p) continue;
        const int e = p + r * p - r * (r - 1) / 2 + (cc - r);
        T x;
        if (cc < q) {  // both covariates: P + V Sigma^-1 V^T
          const int rr = r < QMAX ? r : 0, c2 = cc < QMAX ? cc : 0;
          x = P[rr * q + c2];
#pragma unroll
          for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int z = 0; z < 2; ++z)
              if (u < pr && z < pr) x += v[u][rr] * si[u][z] * v[z][c2];
        } else if (r < q) {  // covariate r, genetic g: -(V Sigma^-1 tm^T)[r][g]
          const int g = (cc - q) < 2 ? cc - q : 0, rr = r < QMAX ? r : 0;
          x = 0;
#pragma unroll
          for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int z = 0; z < 2; ++z)
              if (u < pr && z < pr) x -= v[z][rr] * si[z][u] * (pr == 1 ? (T)1 : tm[g][u]);
        } else {  // both genetic
          x = vr[(r - q) < 2 ? r - q : 0][(cc - q) < 2 ? cc - q : 0];
        }
        if (!ok) x = (T)NAN;
        if (out_f64)
          ((double*)B)[o + e] = (double)x;
        else
          ((float*)B)[o + e] = (float)x;
      }
  }
}

// Virtual columns of a tile of 64: with pr = 1 column i is SNP i; with pr = 2 the SNPs' two
// genetic columns sit 16 apart (column i: SNP (i / 32) 16 + i % 16, genetic column (i / 16) % 2),
// so that a thread holding columns tx + 16 u holds both columns of SNPs tx and 16 + tx.
__device__ __forceinline__ int vcol_snp(int i, int pr) { return pr == 1 ? i : (i >> 5) * 16 + (i & 15); }
__device__ __forceinline__ int vcol_k(int i, int pr) { return pr == 1 ? 0 : (i >> 4) & 1; }

// Coded value of hard call x for genetic column k (0 outside {0, 1, 2}: validation reports it).
__device__ __forceinline__ int code_of(const GeneticModel& gm, int k, int8_t x) {
  return (uint8_t)x <= 2 ? gm.code[k][x] : 0;
}

// ------------------------------------------------------------------------------------------
// CHOL: fused whiten-and-reduce, one CTA per 64 genetic columns (64 SNPs, or 32 with pr = 2)
// ------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) chol_scan_kernel(CholScanArgs<T> a) {
  __shared__ T Ls[TK][TR + 1];
  __shared__ T Xs[TK][TS + 1];
  __shared__ T Rs[QMAX + 1][TR];
  __shared__ T red[16][TS + 1];
  __shared__ T res[QMAX + 3][TS];
  const int n = a.n, q = a.q, pr = a.gm.pr;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t s0 = (int64_t)blockIdx.x * (TS / pr);  // first SNP of the tile
  T ps[4] = {}, pc[4] = {}, pa[4][QMAX] = {}, px[2] = {};
  for (int r0 = 0; r0 < n; r0 += TR) {
    const int kend = min(n, r0 + TR);
    T acc[4][4] = {};
    for (int k0 = 0; k0 < kend; k0 += TK) {
#pragma unroll
      for (int l = 0; l < 4; ++l) {
        const int e = tid + 256 * l, k = e % TK, i = e / TK;
        const int gr = r0 + i, gk = k0 + k;
        Ls[k][i] = (gr < n && gk < n) ? a.Linv[(int64_t)gr * n + gk] : T(0);
        const int64_t gs = s0 + vcol_snp(i, pr);
        Xs[k][i] = (gs < a.m && gk < n) ? (T)code_of(a.gm, vcol_k(i, pr), a.XR[gs * n + gk]) : T(0);
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
      // the cross product of a SNP's two genetic columns (columns tx and tx + 16 of this thread)
      px[0] += acc[u][0] * acc[u][1];
      px[1] += acc[u][2] * acc[u][3];
    }
    __syncthreads();
  }
  // reduce the 16 row-groups of each column: a (q), c, s, and with pr = 2 the cross product
  // (held at the SNP's first column)
  const int nslot = q + 2 + (pr > 1);
  for (int slot = 0; slot < nslot; ++slot) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T val;
      if (slot < q) {
        val = T(0);
#pragma unroll
        for (int k = 0; k < QMAX; ++k)
          if (k == slot) val = pa[v][k];
      } else if (slot == q) {
        val = pc[v];
      } else if (slot == q + 1) {
        val = ps[v];
      } else {
        val = (v & 1) ? T(0) : px[v >> 1];
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
  // one thread per SNP: its first column (and, with pr = 2, the second 16 columns on)
  const int i0 = tid < TS / pr ? (pr == 1 ? tid : (tid / 16) * 32 + tid % 16) : 0;
  const int64_t snp = s0 + vcol_snp(i0, pr);
  if (tid < TS / pr && snp < a.m) {
    T av[2][QMAX], cv[2], S[3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int k = 0; k < QMAX; ++k) av[r][k] = (k < q && r < pr) ? res[k][i0 + 16 * r] : T(0);
    cv[0] = res[q][i0];
    cv[1] = pr > 1 ? res[q][i0 + 16] : T(0);
    S[0] = res[q + 1][i0];
    S[1] = pr > 1 ? res[q + 2][i0] : T(0);
    S[2] = pr > 1 ? res[q + 1][i0 + 16] : T(0);
    schur_store<T>(q, a.gm, a.P, a.b0, av, cv, S, a.sing_tol, a.out_offset + snp, a.j, a.t, a.B,
                   a.wald, a.out_f64, a.flags, a.out_snp, a.out_var);
  }
}

// ------------------------------------------------------------------------------------------
// EIG stage 1: X~ = Z^T X_R into scratch (SNP-major, leading dimension ldp)
// ------------------------------------------------------------------------------------------
// xt row v = snp * pr + k holds Z^T of genetic column k of the SNP (m pr rows).
template <typename T>
__global__ void __launch_bounds__(256) eig_rotate_kernel(int n, int ldp, const T* __restrict__ Zt,
                                                         const int8_t* __restrict__ XR, int64_t m,
                                                         T* __restrict__ xt, GeneticModel gm) {
  const int pr = gm.pr;
  const int64_t mv = m * pr;  // rows of xt
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
      const int64_t gv = s0 + i;
      Xs[k][i] = (gv < mv && gk < n) ? (T)code_of(gm, (int)(gv % pr), XR[(gv / pr) * n + gk]) : T(0);
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
    if (gs >= mv) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int gr = r0 + tx + 16 * v;
      if (gr < ldp) xt[gs * ldp + gr] = gr < n ? acc[u][v] : T(0);
    }
  }
}

// ------------------------------------------------------------------------------------------
// EIG stage 2: trait-batched reduction + Schur, one CTA per 64 genetic columns (64 SNPs, or
// 32 with pr = 2, in the column order of vcol_snp / vcol_k) x 16 traits
// ------------------------------------------------------------------------------------------
constexpr int TT = 16;

template <typename T>
__global__ void __launch_bounds__(256) eig_reduce_kernel(EigScanArgs<T> a) {
  __shared__ T Xs[TK][TS + 1];
  __shared__ T Ps[TK][TT * (QMAX + 2) + 1];
  const int n = a.n, q = a.q, qc = q + 2, t = a.t, pr = a.gm.pr;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const int64_t s0 = (int64_t)blockIdx.x * (TS / pr);  // first SNP of the tile
  const int j0 = blockIdx.y * TT;
  const int j = j0 + ty;
  T acc[4][QMAX + 2] = {};
  T ax[2] = {};  // cross products of a SNP's two genetic columns (columns u = 0, 1 and 2, 3)
  for (int k0 = 0; k0 < n; k0 += TK) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int e = tid + 256 * l, k = e % TK, i = e / TK;
      const int64_t gs = s0 + vcol_snp(i, pr);
      Xs[k][i] = (gs < a.m && k0 + k < n) ? a.xt[(gs * pr + vcol_k(i, pr)) * a.ldp + k0 + k] : T(0);
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
      const T* pl = &Ps[k][ty * qc];
#pragma unroll
      for (int c = 0; c < QMAX + 1; ++c) {
        if (c < q + 1) {
          const T pv = pl[c];
#pragma unroll
          for (int u = 0; u < 4; ++u) acc[u][c] += xv[u] * pv;
        }
      }
      const T dm = pl[q + 1];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u][QMAX + 1] += xv[u] * xv[u] * dm;
      ax[0] += xv[0] * xv[1] * dm;
      ax[1] += xv[2] * xv[3] * dm;
    }
    __syncthreads();
  }
  if (j >= t) return;
  const T* P = a.P + (int64_t)j * q * q;
  const T* b0 = a.b0 + (int64_t)j * q;
  // this thread's SNPs: u = 0..3 (pr = 1), or the pairs (0, 1) and (2, 3) (pr = 2)
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    if (pr > 1 && w >= 2) break;
    const int u0 = pr > 1 ? 2 * w : w;
    const int64_t gs = s0 + vcol_snp(tx + 16 * u0, pr);
    if (gs >= a.m) continue;
    T av[2][QMAX], cv[2] = {0, 0}, S[3] = {0, 0, 0};
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int k = 0; k < QMAX; ++k) av[r][k] = (k < q && r < pr) ? acc[u0 + r < 4 ? u0 + r : 0][k] : T(0);
#pragma unroll
    for (int k = 0; k < QMAX + 1; ++k)
      if (k == q) {
        cv[0] = acc[u0][k];
        if (pr > 1) cv[1] = acc[u0 + 1 < 4 ? u0 + 1 : 0][k];
      }
    S[0] = acc[u0][QMAX + 1];
    if (pr > 1) {
      S[1] = ax[w < 2 ? w : 0];
      S[2] = acc[u0 + 1 < 4 ? u0 + 1 : 0][QMAX + 1];
    }
    schur_store<T>(q, a.gm, P, b0, av, cv, S, a.sing_tol, a.out_offset + gs, j, t, a.B, a.wald,
                   a.out_f64, a.flags, a.out_snp, a.out_var);
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
  GW_REQUIRE(a.gm.pr == 1 || a.gm.pr == 2, GWAS_ERR_ARG, "pr=%d outside [1,2]", a.gm.pr);
  chol_scan_kernel<T><<<ceil_div(a.m, TS / a.gm.pr), 256, 0, s>>>(a);
  GW_CHECK_LAUNCH();
}

template <typename T>
void eig_scan_simt(cudaStream_t s, const EigScanArgs<T>& a) {
  if (a.m <= 0) return;
  GW_REQUIRE(a.q >= 1 && a.q <= QMAX, GWAS_ERR_ARG, "q=%d outside [1,%d]", a.q, QMAX);
  GW_REQUIRE(a.gm.pr == 1 || a.gm.pr == 2, GWAS_ERR_ARG, "pr=%d outside [1,2]", a.gm.pr);
  const int64_t mv = a.m * a.gm.pr;  // rotated genetic columns
  GW_REQUIRE(mv <= (int64_t)65535 * TS, GWAS_ERR_ARG, "block of %lld SNPs too large", (long long)a.m);
  dim3 g1(ceil_div(a.ldp, TR), ceil_div(mv, TS));
  eig_rotate_kernel<T><<<g1, 256, 0, s>>>(a.n, a.ldp, a.Zt, a.XR, a.m, a.xt, a.gm);
  GW_CHECK_LAUNCH();
  GW_REQUIRE(ceil_div(a.t, TT) <= 65535, GWAS_ERR_ARG, "t=%d too large", a.t);
  dim3 g2(ceil_div(a.m, TS / a.gm.pr), ceil_div(a.t, TT));
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
