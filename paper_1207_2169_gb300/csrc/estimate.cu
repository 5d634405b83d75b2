// Step 1 of the two-step method on the GPU (FP64): per trait, the variance components
// (h^2, sigma^2) that maximise the ML or REML criterion of the reduced model y = X_L beta + R,
// R ~ N(0, sigma^2 (h^2 Phi + (1 - h^2) I)) (Supplementary Note Section 1, "Mixed Models for
// GWAS"; "Time complexity": an eigendecomposition of Phi, then an iterative search per trait).
//
// With Phi = Z W Z^T and h standing for h^2, H(h) = h Phi + (1 - h) I = Z diag(h w + 1 - h) Z^T,
// so in the rotated coordinates X~ = Z^T X_L and y~ = Z^T y every term of the criterion is a
// weighted sum over the n eigen-coordinates with weights d_r = 1 / (h w_r + 1 - h):
//   X_L^T H^-1 X_L = X~^T D X~,  X_L^T H^-1 y = X~^T D y~,  y^T H^-1 y = y~^T D y~,
//   log|H| = sum_r log(h w_r + 1 - h),  Q = r^T H^-1 r = y~^T D y~ - b^T X~^T D y~,
// b the GLS coefficients.  ML: s2 = Q / n, l = -1/2 [n log(2 pi s2) + log|H| + n].  REML (the
// density of the error contrasts): s2 = Q / (n - q),
//   l = -1/2 [(n - q) log(2 pi s2) + log|H| + log|X~^T D X~| - log|X_L^T X_L| + (n - q)].
// One CTA per trait evaluates the criterion at every h of the search -- the grid
// h_g = (g / 100) 0.999, g = 0..100, then a golden-section search between the best grid point's
// neighbours -- and keeps the better of the grid's best and the refined point.  A trait that
// X_L fits exactly (Q <= 1e-12 y~^T D y~, far above the rounding of the subtraction that forms
// Q) gets NaN for h^2 and the criterion, 0 for sigma^2.
#include "common.cuh"

namespace gw {
namespace {

constexpr int THREADS = 256;
constexpr int GRID = 100;
constexpr double H2_MAX = 0.999;
constexpr double EXACT_FIT = 1e-12;  // Q / y~^T D y~ of a trait X_L fits exactly
constexpr int GOLDEN_ITERS = 64;  // the bracket (<= 0.02 wide) shrinks below 1e-15
constexpr double TWO_PI = 6.283185307179586;

constexpr int NA_MAX = 28;  // packed lower triangle of a 7 x 7 matrix

struct EstArgs {
  int n, q, t, method;
  const double* w;    // n eigenvalues of Phi
  const double* XLt;  // q x n: row k = Z^T X_L[:, k]
  const double* Yt;   // t x n: row j = Z^T y_j
  // trait-independent terms at the grid points h_g (grid_tables_kernel): the weights
  // d_gr = 1 / (h_g w_r + 1 - h_g) (GRID + 1 rows of n), X~^T D_g X~ (packed, NA_MAX per
  // point) and log|H(h_g)|
  const double *Dtab, *Atab, *ldtab;
  double *h2, *s2, *crit;
  int* flags;
};

template <int QM>
struct Acc {
  static constexpr int NA = QM * (QM + 1) / 2;  // X~^T D X~, packed lower triangle
  static constexpr int N = NA + QM + 2;         // then X~^T D y~, y~^T D y~, log|H|
};

// Thread 0: the criterion from the reduced sums.  A: X~^T D X~ (packed lower triangle), bx:
// X~^T D y~, yy: y~^T D y~, log_h: log|H|.  ld_xtx: log|X_L^T X_L| (REML); NaN on the first
// call, which is at h = 0 where it equals log|X~^T D X~|.
template <int QM>
__device__ void solve_criterion(const EstArgs& a, const double* A, const double* bx, double yy,
                                double log_h, double& ld_xtx, double* bc) {
  const int n = a.n, q = a.q;
  // X~^T D X~ = C C^T (Cholesky); b^T X~^T D y~ = z^T z with z = C^-1 X~^T D y~
  double C[QM][QM], z[QM];
  bool ok = true;
  double logdet_a = 0.0;
  for (int k = 0; k < q; ++k) {
    for (int i = k; i < q; ++i) {
      double v = A[i * (i + 1) / 2 + k];
      for (int m = 0; m < k; ++m) v -= C[i][m] * C[k][m];
      if (i == k) {
        if (!(v > 1e-13 * A[k * (k + 1) / 2 + k])) { ok = false; v = 1.0; }
        C[k][k] = sqrt(v);
        logdet_a += 2.0 * log(C[k][k]);
      } else {
        C[i][k] = v / C[k][k];
      }
    }
  }
  double zz = 0.0;
  for (int k = 0; k < q; ++k) {
    double v = bx[k];
    for (int m = 0; m < k; ++m) v -= C[k][m] * z[m];
    z[k] = v / C[k][k];
    zz += z[k] * z[k];
  }
  const double Q = yy - zz;
  if (ld_xtx != ld_xtx) ld_xtx = logdet_a;
  double crit, sig2;
  if (!ok) {
    atomicExch(&a.flags[FLAG_STL_SINGULAR], 1);
    crit = NAN;
    sig2 = 0.0;
  } else if (!(Q > EXACT_FIT * yy)) {
    crit = NAN;
    sig2 = 0.0;
  } else if (a.method == 0) {
    sig2 = Q / n;
    crit = -0.5 * (n * log(TWO_PI * sig2) + log_h + n);
  } else {
    const double dof = n - q;
    sig2 = Q / dof;
    crit = -0.5 * (dof * log(TWO_PI * sig2) + log_h + logdet_a - ld_xtx + dof);
  }
  bc[0] = crit;
  bc[1] = sig2;
  bc[2] = ld_xtx;
}

// Block-wide sums of v[0..N) (every thread's partials) into red; returns after a barrier.
template <int N>
__device__ __forceinline__ void block_sums(double (&v)[N], double (*red)[THREADS / 32]) {
  const int wp = threadIdx.x / 32, ln = threadIdx.x % 32;
#pragma unroll
  for (int u = 0; u < N; ++u) {
    double x = v[u];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (ln == 0) red[u][wp] = x;
  }
  __syncthreads();
}

__device__ __forceinline__ double red_total(const double (*red)[THREADS / 32], int u) {
  double v = 0.0;
  for (int i = 0; i < THREADS / 32; ++i) v += red[u][i];
  return v;
}

// Broadcasts thread 0's result to every thread; bc and red are free again on return.
__device__ __forceinline__ double broadcast(const double* bc, double& s2, double& ld_xtx) {
  __syncthreads();
  const double crit = bc[0];
  s2 = bc[1];
  ld_xtx = bc[2];
  __syncthreads();
  return crit;
}

// The criterion at any h for the CTA's trait (every thread calls it and gets the result; s2
// gets sigma^2).  Returns NaN for an exact fit.
template <int QM>
__device__ double criterion(const EstArgs& a, const double* __restrict__ y, double h,
                            double& ld_xtx, double& s2, double (*red)[THREADS / 32],
                            double* bc) {
  constexpr int N = Acc<QM>::N, NA = Acc<QM>::NA;
  const int n = a.n, q = a.q;
  double acc[N];
#pragma unroll
  for (int u = 0; u < N; ++u) acc[u] = 0.0;
  // log|H| as a sum of logs of products of 16 factors (each in [0.001, max w]: no overflow)
  double prod = 1.0;
  int nprod = 0;
  for (int r = threadIdx.x; r < n; r += THREADS) {
    const double e = fma(h, a.w[r] - 1.0, 1.0);  // h w_r + 1 - h
    const double d = recip_f64(e);
    prod *= e;
    if (++nprod == 16) {
      acc[NA + QM + 1] += log(prod);
      prod = 1.0;
      nprod = 0;
    }
    const double yr = y[r];
    double x[QM];
#pragma unroll
    for (int k = 0; k < QM; ++k) x[k] = k < q ? a.XLt[(int64_t)k * n + r] : 0.0;
    int u = 0;
#pragma unroll
    for (int k = 0; k < QM; ++k) {
      const double dx = d * x[k];
#pragma unroll
      for (int l = 0; l <= k; ++l, ++u) acc[u] = fma(dx, x[l], acc[u]);
    }
    const double dy = d * yr;
#pragma unroll
    for (int k = 0; k < QM; ++k) acc[NA + k] = fma(dy, x[k], acc[NA + k]);
    acc[NA + QM] = fma(dy, yr, acc[NA + QM]);
  }
  acc[NA + QM + 1] += log(prod);
  block_sums<N>(acc, red);
  if (threadIdx.x == 0) {
    double tot[N];
    for (int u = 0; u < N; ++u) tot[u] = red_total(red, u);
    solve_criterion<QM>(a, tot, tot + NA, tot[NA + QM], tot[NA + QM + 1], ld_xtx, bc);
  }
  return broadcast(bc, s2, ld_xtx);
}

// The criterion at grid point g: the trait-independent terms come from the tables, so each
// eigen-coordinate costs q + 1 multiply-adds.
template <int QM>
__device__ double criterion_grid(const EstArgs& a, const double* __restrict__ y, int g,
                                 double& ld_xtx, double& s2, double (*red)[THREADS / 32],
                                 double* bc) {
  const int n = a.n, q = a.q;
  const double* dg = a.Dtab + (int64_t)g * n;
  double acc[QM + 1];
#pragma unroll
  for (int u = 0; u <= QM; ++u) acc[u] = 0.0;
  for (int r = threadIdx.x; r < n; r += THREADS) {
    const double yr = y[r];
    const double dy = dg[r] * yr;
#pragma unroll
    for (int k = 0; k < QM; ++k)
      if (k < q) acc[k] = fma(dy, a.XLt[(int64_t)k * n + r], acc[k]);
    acc[QM] = fma(dy, yr, acc[QM]);
  }
  block_sums<QM + 1>(acc, red);
  if (threadIdx.x == 0) {
    double tot[QM + 1];
    for (int u = 0; u <= QM; ++u) tot[u] = red_total(red, u);
    solve_criterion<QM>(a, a.Atab + (int64_t)g * NA_MAX, tot, tot[QM], a.ldtab[g], ld_xtx, bc);
  }
  return broadcast(bc, s2, ld_xtx);
}

// One CTA per grid point: d_gr, X~^T D_g X~ and log|H(h_g)| for every trait to share.
__global__ void __launch_bounds__(THREADS) grid_tables_kernel(EstArgs a, double* Dtab,
                                                              double* Atab, double* ldtab) {
  __shared__ double red[NA_MAX + 1][THREADS / 32];
  const int g = blockIdx.x, n = a.n, q = a.q;
  const double h = (double)g / GRID * H2_MAX;
  double acc[NA_MAX + 1];
#pragma unroll
  for (int u = 0; u <= NA_MAX; ++u) acc[u] = 0.0;
  double prod = 1.0;
  int nprod = 0;
  for (int r = threadIdx.x; r < n; r += THREADS) {
    const double e = fma(h, a.w[r] - 1.0, 1.0);
    const double d = recip_f64(e);
    Dtab[(int64_t)g * n + r] = d;
    prod *= e;
    if (++nprod == 16) {
      acc[NA_MAX] += log(prod);
      prod = 1.0;
      nprod = 0;
    }
    double x[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) x[k] = k < q ? a.XLt[(int64_t)k * n + r] : 0.0;
    int u = 0;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      const double dx = d * x[k];
#pragma unroll
      for (int l = 0; l <= k; ++l, ++u) acc[u] = fma(dx, x[l], acc[u]);
    }
  }
  acc[NA_MAX] += log(prod);
  block_sums<NA_MAX + 1>(acc, red);
  if (threadIdx.x <= NA_MAX) {
    const double v = red_total(red, threadIdx.x);
    if (threadIdx.x < NA_MAX)
      Atab[(int64_t)g * NA_MAX + threadIdx.x] = v;
    else
      ldtab[g] = v;
  }
}

template <int QM>
__global__ void __launch_bounds__(THREADS) estimate_kernel(EstArgs a) {
  __shared__ double red[Acc<QM>::N][THREADS / 32];
  __shared__ double bc[3];
  const int j = blockIdx.x;
  const double* y = a.Yt + (int64_t)j * a.n;
  double ld_xtx = NAN, s2 = 0.0;
  // grid: the first point is h = 0, which also gives log|X_L^T X_L|
  double best = -INFINITY;
  int gbest = -1;
  for (int g = 0; g <= GRID; ++g) {
    const double c = criterion_grid<QM>(a, y, g, ld_xtx, s2, red, bc);
    if (c > best) {
      best = c;
      gbest = g;
    }
  }
  double h_est = NAN, c_est = NAN, s2_est = 0.0;
  if (gbest >= 0) {
    // golden-section search for the maximum between the neighbours of the best grid point
    const double gr = 0.6180339887498949;  // (sqrt(5) - 1) / 2
    double lo = (double)(gbest > 0 ? gbest - 1 : 0) / GRID * H2_MAX;
    double hi = (double)(gbest < GRID ? gbest + 1 : GRID) / GRID * H2_MAX;
    double xc = hi - gr * (hi - lo), xd = lo + gr * (hi - lo);
    double fc = criterion<QM>(a, y, xc, ld_xtx, s2, red, bc);
    double fd = criterion<QM>(a, y, xd, ld_xtx, s2, red, bc);
    for (int it = 0; it < GOLDEN_ITERS; ++it) {
      if (fc > fd) {
        hi = xd;
        xd = xc;
        fd = fc;
        xc = hi - gr * (hi - lo);
        fc = criterion<QM>(a, y, xc, ld_xtx, s2, red, bc);
      } else {
        lo = xc;
        xc = xd;
        fc = fd;
        xd = lo + gr * (hi - lo);
        fd = criterion<QM>(a, y, xd, ld_xtx, s2, red, bc);
      }
    }
    const double h_ref = fc > fd ? xc : xd, f_ref = fc > fd ? fc : fd;
    h_est = f_ref >= best ? h_ref : (double)gbest / GRID * H2_MAX;
    c_est = criterion<QM>(a, y, h_est, ld_xtx, s2_est, red, bc);
  }
  if (threadIdx.x == 0) {
    a.h2[j] = h_est;
    a.s2[j] = s2_est;
    a.crit[j] = c_est;
  }
}

}  // namespace

void estimate_traits(cudaStream_t s, int n, int q, int t, int method, const double* w,
                     const double* XLt, const double* Yt, double* tables, double* h2, double* s2,
                     double* crit, int* flags) {
  double* Dtab = tables;
  double* Atab = Dtab + (size_t)(GRID + 1) * n;
  double* ldtab = Atab + (size_t)(GRID + 1) * NA_MAX;
  EstArgs a{n, q, t, method, w, XLt, Yt, Dtab, Atab, ldtab, h2, s2, crit, flags};
  grid_tables_kernel<<<GRID + 1, THREADS, 0, s>>>(a, Dtab, Atab, ldtab);
  GW_CHECK_LAUNCH();
  if (q <= 3)
    estimate_kernel<3><<<t, THREADS, 0, s>>>(a);
  else
    estimate_kernel<7><<<t, THREADS, 0, s>>>(a);
  GW_CHECK_LAUNCH();
}

size_t estimate_table_doubles(int n) { return (size_t)(GRID + 1) * (n + NA_MAX + 1); }

}  // namespace gw
