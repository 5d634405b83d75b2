// Symmetric FP64 eigendecomposition for the setup, Phi = Z W Z^T (Algorithm 4), by the
// tridiagonal route the complexity count of the paper assumes (10/3 n^3):
//   1. Householder reduction Q^T Phi Q = T (T tridiagonal: diagonal d, off-diagonal e);
//   2. eigenvalues of T by multisection on Sturm counts, one warp per eigenvalue;
//   3. eigenvectors of T by inverse iteration, one thread per eigenvector (tridiagonal LU with
//      partial pivoting).  Eigenvalues closer than 1e-12 ||T|| form a cluster; all of a
//      cluster's members iterate with one shift placed just below the cluster (further than
//      its spread, nearer than the next eigenvalue), so that their random starts are amplified
//      alike and stay independent while the rest of the spectrum is damped;
//   4. the vectors orthonormalised by Cholesky QR, twice (FP64 Gram matrix, Cholesky, inverse);
//   5. Z = Q S by applying the reflectors to the eigenvectors of T.
// Returns -1 if step 4 meets a matrix that is not positive definite (the caller then uses the
// Jacobi solver).
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace gw {
namespace {

constexpr int ET = 256;  // threads per CTA

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum_all(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int i = 0; i < (int)(blockDim.x / 32); ++i) t += red[i];
  return t;
}

// A (column-major, n x n) := Phi with its lower triangle mirrored.
__global__ void symmetrize_kernel(int n, const double* __restrict__ Phi, double* __restrict__ A) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  const int i = (int)(e % n), c = (int)(e / n);
  A[e] = i >= c ? Phi[e] : Phi[c + (int64_t)i * n];
}

// Step k: the reflector H = I - tau v v^T that maps x = A(k+1:n, k) onto alpha e_1.  v is stored
// in A(k+1:n, k) and in vbuf; d[k] = A(k,k), e[k] = alpha.
__global__ void house_kernel(int n, int k, double* A, double* vbuf, double* tau, double* d,
                             double* e) {
  __shared__ double red[ET / 32];
  const int m = n - k - 1;
  double* x = A + (int64_t)k * n + k + 1;
  double ss = 0.0;
  for (int i = threadIdx.x; i < m; i += ET) ss = fma(x[i], x[i], ss);
  ss = block_sum_all(ss, red);
  const double x0 = x[0];
  double t = 0.0, alpha = x0, v0 = 0.0;
  if (ss > 0.0 && ss - x0 * x0 > 0.0) {
    alpha = -copysign(sqrt(ss), x0);
    v0 = x0 - alpha;
    t = 2.0 / (ss - x0 * x0 + v0 * v0);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += ET) {
    const double vi = t != 0.0 ? (i == 0 ? v0 : x[i]) : 0.0;
    vbuf[i] = vi;
    x[i] = vi;
  }
  if (threadIdx.x == 0) {
    tau[k] = t;
    d[k] = A[(int64_t)k * n + k];
    e[k] = alpha;
  }
}

// p_i = tau sum_j A(k+1+j, k+1+i) v_j (A symmetric: column k+1+i), one warp per i.
__global__ void house_matvec_kernel(int n, int k, const double* __restrict__ A,
                                    const double* __restrict__ v, const double* __restrict__ tau,
                                    double* __restrict__ p) {
  const int m = n - k - 1;
  const int i = blockIdx.x * (ET / 32) + threadIdx.x / 32, l = threadIdx.x % 32;
  if (i >= m) return;
  const double* col = A + (int64_t)(k + 1 + i) * n + k + 1;
  double acc = 0.0;
  for (int j = l; j < m; j += 32) acc = fma(col[j], v[j], acc);
  acc = warp_sum(acc);
  if (l == 0) p[i] = tau[k] * acc;
}

// w = p - (tau/2) (p^T v) v
__global__ void house_w_kernel(int n, int k, const double* __restrict__ v,
                               const double* __restrict__ tau, const double* __restrict__ p,
                               double* __restrict__ wv) {
  __shared__ double red[ET / 32];
  const int m = n - k - 1;
  double s = 0.0;
  for (int i = threadIdx.x; i < m; i += ET) s = fma(p[i], v[i], s);
  s = block_sum_all(s, red);
  const double K = 0.5 * tau[k] * s;
  for (int i = threadIdx.x; i < m; i += ET) wv[i] = p[i] - K * v[i];
}

// A(k+1:, k+1:) -= v w^T + w v^T; 32 x 32 tiles, 256 threads each updating four elements.
__global__ void house_update_kernel(int n, int k, double* A, const double* __restrict__ v,
                                    const double* __restrict__ wv) {
  const int m = n - k - 1;
  const int i = blockIdx.x * 32 + threadIdx.x % 32;
  const int j0 = blockIdx.y * 32 + threadIdx.x / 32;
  if (i >= m) return;
  const double vi = v[i], wi = wv[i];
  for (int j = j0; j < m && j < blockIdx.y * 32 + 32; j += ET / 32) {
    double* a = A + (int64_t)(k + 1 + j) * n + k + 1 + i;
    *a -= vi * wv[j] + wi * v[j];
  }
}

// Barrier of all CTAs of a cooperative launch (every CTA is resident): a counter and a generation
// word in global memory.  The wait is bounded (limit_ns); on expiry it sets *gflag and returns
// false, and so does every later barrier of the launch, so that the kernel unwinds.
__device__ bool grid_barrier(unsigned* count, volatile unsigned* gen, int* gflag,
                             uint64_t limit_ns) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = *(volatile int*)gflag == 0;
    const unsigned g = *gen;
    __threadfence();
    if (atomicAdd(count, 1u) == gridDim.x - 1) {
      *count = 0;
      __threadfence();
      atomicAdd((unsigned*)gen, 1u);
    } else if (ok) {
      uint64_t t0;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      while (*gen == g) {
        uint64_t t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        if (t1 - t0 > limit_ns || *(volatile int*)gflag) {
          atomicExch(gflag, 1);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// The whole Householder reduction in one cooperative launch: per column k, every CTA finds the
// reflector of A(k+1:n, k) itself (the arithmetic of house_kernel, so every CTA holds the same v
// and tau), the CTAs' warps share the rows of p = tau A v, then (after a barrier) every CTA forms
// w = p - (tau/2)(p.v) v and updates its share of the trailing columns,
// A(k+1:, k+1:) -= v w^T + w v^T, while CTA 0 stores v, tau, d, e; a second barrier ends the
// step.  Two barriers per column instead of four launches.
__global__ void __launch_bounds__(ET) house_coop_kernel(int n, double* A, double* pbuf,
                                                        double* tau, double* d, double* e,
                                                        unsigned* bar, int* gflag) {
  __shared__ double red[ET / 32];
  __shared__ double sh[3];  // v0, t, alpha
  const int warps = ET / 32, gw = blockIdx.x * warps + threadIdx.x / 32, l = threadIdx.x % 32;
  const int nw = gridDim.x * warps;
  const uint64_t LIMIT = 2000000000ull;
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    double* x = A + (int64_t)k * n + k + 1;
    // the reflector, in every CTA (as house_kernel)
    double ss = 0.0;
    for (int i = threadIdx.x; i < m; i += ET) ss = fma(x[i], x[i], ss);
    ss = block_sum_all(ss, red);
    if (threadIdx.x == 0) {
      const double x0 = x[0];
      double t = 0.0, alpha = x0, v0 = 0.0;
      if (ss > 0.0 && ss - x0 * x0 > 0.0) {
        alpha = -copysign(sqrt(ss), x0);
        v0 = x0 - alpha;
        t = 2.0 / (ss - x0 * x0 + v0 * v0);
      }
      sh[0] = v0;
      sh[1] = t;
      sh[2] = alpha;
    }
    __syncthreads();
    const double v0 = sh[0], t = sh[1];
    auto vat = [&](int j) -> double { return t != 0.0 ? (j == 0 ? v0 : x[j]) : 0.0; };
    // p = tau A(k+1:, k+1:) v, one warp per row (A symmetric: row i = column k+1+i)
    for (int i = gw; i < m; i += nw) {
      const double* col = A + (int64_t)(k + 1 + i) * n + k + 1;
      double acc = 0.0;
      for (int j = l; j < m; j += 32) acc = fma(col[j], vat(j), acc);
      acc = warp_sum(acc);
      if (l == 0) pbuf[i] = t * acc;
    }
    if (!grid_barrier(bar, bar + 1, gflag, LIMIT)) return;
    // w = p - (tau/2)(p.v) v, then the rank-2 update of this CTA's columns
    double pv = 0.0;
    for (int i = threadIdx.x; i < m; i += ET) pv = fma(pbuf[i], vat(i), pv);
    pv = block_sum_all(pv, red);
    const double K = 0.5 * t * pv;
    for (int jc = blockIdx.x; jc < m; jc += gridDim.x) {
      const double vj = vat(jc), wj = pbuf[jc] - K * vj;
      double* a = A + (int64_t)(k + 1 + jc) * n + k + 1;
      for (int i = threadIdx.x; i < m; i += ET) {
        const double vi = vat(i), wi = pbuf[i] - K * vi;
        a[i] -= vi * wj + wi * vj;
      }
    }
    if (blockIdx.x == 0) {
      // column k now takes the reflector (read by the back-transformation); no trailing
      // column reads it
      __syncthreads();  // every thread of this CTA is done reading x
      const double dk = A[(int64_t)k * n + k];
      for (int i = threadIdx.x; i < m; i += ET) x[i] = t != 0.0 ? (i == 0 ? v0 : x[i]) : 0.0;
      if (threadIdx.x == 0) {
        tau[k] = t;
        d[k] = dk;
        e[k] = sh[2];
      }
    }
    if (!grid_barrier(bar, bar + 1, gflag, LIMIT)) return;
  }
}

// The last 2 x 2 block: d[n-2], d[n-1], e[n-2] (n >= 2), or d[0] (n == 1).
__global__ void house_tail_kernel(int n, const double* A, double* d, double* e) {
  if (threadIdx.x != 0) return;
  if (n == 1) {
    d[0] = A[0];
    return;
  }
  d[n - 2] = A[(int64_t)(n - 2) * n + n - 2];
  d[n - 1] = A[(int64_t)(n - 1) * n + n - 1];
  e[n - 2] = A[(int64_t)(n - 2) * n + n - 1];
}

// Eigenvalue i (ascending) of T by multisection on the Sturm count (the number of eigenvalues
// below x is the number of negative pivots of T - x I): one warp per eigenvalue, its lanes
// counting at 31 interior points of the current interval, which then shrinks 32-fold per round
// (a Sturm count is a chain of n dependent steps, so fewer rounds, not more threads per round,
// shorten it).
__device__ __forceinline__ int sturm_count(int n, const double* __restrict__ d,
                                           const double* __restrict__ e2, double x,
                                           double pivmin) {
  // a pivot smaller than pivmin is replaced by -pivmin before it is counted, so that a shift
  // landing exactly on a pivot counts it the way the rest of the recurrence uses it
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int cnt = q < 0.0;
  for (int j = 1; j < n; ++j) {
    // correctly rounded division: with every step correctly rounded the count cannot fall as
    // x rises (the monotonicity the multisection's interval update relies on)
    q = d[j] - x - e2[j - 1] / q;
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0;
  }
  return cnt;
}

__global__ void bisect_kernel(int n, const double* __restrict__ d, const double* __restrict__ e2,
                              double gl, double gu, double pivmin, double* __restrict__ w) {
  const int i = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32, lane = threadIdx.x % 32;
  if (i >= n) return;  // warp-uniform
  double lo = gl, hi = gu;
  for (int it = 0; it < 64; ++it) {
    if (hi - lo <= 4.4e-16 * fmax(fabs(lo), fabs(hi)) + pivmin) break;  // warp-uniform
    // the points rise with the lane; a point rounded onto or past an end takes that end's vote,
    // so the votes stay monotone and the interval keeps eigenvalue i
    const double x = lo + (hi - lo) * (double)(lane + 1) * (1.0 / 32.0);
    bool above;
    if (lane == 31 || x >= hi) above = true;
    else if (x <= lo) above = false;
    else above = sturm_count(n, d, e2, x, pivmin) > i;
    // the first point with eigenvalue i below it bounds the interval from above
    const unsigned bal = __ballot_sync(0xffffffffu, above);
    const int f = __ffs(bal) - 1;  // 0..31 (lane 31 always votes)
    const double xf = __shfl_sync(0xffffffffu, x, f);
    const double xp = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
    const double nhi = f < 31 ? fmin(xf, hi) : hi;
    const double nlo = f > 0 ? fmax(xp, lo) : lo;
    if (!(nhi < hi || nlo > lo)) break;  // no progress left in floating point
    hi = nhi;
    lo = nlo;
  }
  if (lane == 0) w[i] = 0.5 * (lo + hi);
}

// Counter-based uniform in (-1, 1) for start vector i, component j (splitmix64 of (i, j)).
__device__ __forceinline__ double hash_uniform(uint64_t i, uint64_t j) {
  uint64_t x = (i * 0x9E3779B97F4A7C15ull) ^ (j * 0xBF58476D1CE4E5B9ull) ^ 0x94D049BB133111EBull;
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x ^= x >> 31;
  return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Eigenvector i of T by inverse iteration with shift sig[i]: ITERS solves of (T - sig I) z = b,
// each a tridiagonal LU with partial pivoting whose forward elimination runs on b as it
// factors.  Workspace rows are interleaved by thread (element j of thread i at j * n + i).
// The normalised vector is written to column i of S (column-major).
constexpr int INV_ITERS = 3;
__global__ void invit_kernel(int n, const double* __restrict__ d, const double* __restrict__ e,
                             const double* __restrict__ sig, double anorm, double* u1,
                             double* u2, double* u3, double* z, double* __restrict__ S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double s = sig[i], tiny = 2.220446049250313e-16 * anorm;
  auto at = [&](double* a, int j) -> double& { return a[(int64_t)j * n + i]; };
  for (int j = 0; j < n; ++j) at(z, j) = hash_uniform(i, j);
  double scale = 1.0;
  for (int it = 0; it < INV_ITERS; ++it) {
    // Factor T - s I with row interchanges while eliminating the right-hand side: the current
    // row k is (a, up) in columns k, k+1 with right-hand side bk; row k + 1 is (e_k, an, upn)
    // with right-hand side bn.  Stored: U's diagonal u1, first and second super-diagonals u2,
    // u3, and the eliminated right-hand side in z.
    double a = d[0] - s, up = n > 1 ? e[0] : 0.0, bk = at(z, 0) * scale;
    for (int k = 0; k < n - 1; ++k) {
      const double c = e[k];
      const double an = d[k + 1] - s;
      const double upn = k + 1 < n - 1 ? e[k + 1] : 0.0;
      const double bn = at(z, k + 1) * scale;
      if (fabs(a) >= fabs(c)) {
        if (a == 0.0) a = tiny;
        const double f = c / a;
        at(u1, k) = a;
        at(u2, k) = up;
        at(u3, k) = 0.0;
        at(z, k) = bk;
        a = an - f * up;
        up = upn;
        bk = bn - f * bk;
      } else {
        const double f = a / c;
        at(u1, k) = c;
        at(u2, k) = an;
        at(u3, k) = upn;
        at(z, k) = bn;
        a = up - f * an;
        up = -f * upn;
        bk = bk - f * bn;
      }
    }
    if (a == 0.0) a = tiny;
    at(u1, n - 1) = a;
    at(z, n - 1) = bk;
    // back substitution, keeping the largest magnitude to rescale the next right-hand side
    double x1 = bk / a, x2 = 0.0, mx = fabs(x1);
    at(z, n - 1) = x1;
    for (int k = n - 2; k >= 0; --k) {
      const double x = (at(z, k) - at(u2, k) * x1 - at(u3, k) * x2) / at(u1, k);
      at(z, k) = x;
      x2 = x1;
      x1 = x;
      mx = fmax(mx, fabs(x));
    }
    scale = mx > 0.0 ? 1.0 / mx : 1.0;
  }
  double nrm = 0.0;
  for (int j = 0; j < n; ++j) {
    const double x = at(z, j) * scale;
    nrm = fma(x, x, nrm);
  }
  nrm = scale / sqrt(nrm);
  for (int j = 0; j < n; ++j) S[(int64_t)i * n + j] = at(z, j) * nrm;
}

}  // namespace
}  // namespace gw

namespace gw {
namespace {

// Z(:, c) := H_0 H_1 ... H_{n-3} Z(:, c), one warp per column c with the column in shared memory:
// the columns are independent, so each warp walks every reflector (from the last to the first)
// with no step shared with other warps (no block or grid barrier between reflectors), reading the
// reflectors from L1 / L2.  Per reflector k: y = v_k . Z(k+1:, c) (a warp reduction), then
// Z(k+1:, c) -= tau_k y v_k.
constexpr int BT_WARPS = 4;  // columns (warps) per CTA at most
__global__ void __launch_bounds__(32 * BT_WARPS) bt_columns_kernel(int n,
                                                                   const double* __restrict__ A,
                                                                   const double* __restrict__ tau,
                                                                   double* Zt) {
  extern __shared__ double zs[];  // (blockDim.x / 32) x n
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  const int c = blockIdx.x * (blockDim.x / 32) + w;
  if (c >= n) return;  // warp-uniform; no block barrier follows
  double* z = zs + (int64_t)w * n;
  const double* zc = Zt + (int64_t)c * n;
  for (int r = l; r < n; r += 32) z[r] = zc[r];
  __syncwarp();
  for (int k = n - 3; k >= 0; --k) {
    const int m = n - k - 1;
    const double* v = A + (int64_t)k * n + k + 1;
    double* zk = z + k + 1;
    double dot = 0.0;
    for (int r = l; r < m; r += 32) dot = fma(v[r], zk[r], dot);
    const double y = tau[k] * warp_sum(dot);
    for (int r = l; r < m; r += 32) zk[r] -= y * v[r];
    __syncwarp();  // the next reflector's dot reads elements other lanes updated
  }
  double* zo = Zt + (int64_t)c * n;
  for (int r = l; r < n; r += 32) zo[r] = z[r];
}

// Device buffers of one call, freed on every exit.
struct DevBufs {
  std::vector<void*> p;
  double* get(size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, (count ? count : 1) * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc(%zu bytes) failed: %s", count * sizeof(double), cudaGetErrorString(e));
      throw Fail{GWAS_ERR_OOM};
    }
    p.push_back(q);
    return (double*)q;
  }
  ~DevBufs() {
    for (void* q : p) cudaFree(q);
  }
};

}  // namespace

int eigh_tridiag(cudaStream_t s, int n, const double* Phi, double* Zt, double* w) {
  const size_t nn = (size_t)n * n;
  DevBufs mem;
  double* A = mem.get(nn);
  double* S = mem.get(nn);
  double* G = mem.get(nn);
  double* Li = mem.get(nn);
  double* W2 = mem.get(nn);
  double* wk = mem.get(4 * nn);  // inverse-iteration workspace: u1, u2, u3, z
  double* vb = mem.get(n);
  double* pv = mem.get(n);
  double* wv = mem.get(n);
  double* tau = mem.get(n);
  double* d = mem.get(n);
  double* e = mem.get(n);
  double* e2 = mem.get(n);
  double* sg = mem.get(n);
  int* flags = (int*)mem.get(FLAG_COUNT);
  GW_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * FLAG_COUNT, s));
  GW_CUDA(cudaMemsetAsync(e, 0, sizeof(double) * n, s));
  symmetrize_kernel<<<ceil_div((int64_t)nn, 256), 256, 0, s>>>(n, Phi, A);
  GW_CHECK_LAUNCH();
  // 1. Householder reduction to tridiagonal form: one cooperative launch (every CTA resident,
  //    one per SM), or four launches per column where a cooperative launch is not available
  bool coop = false;
  if (n > 2) {
    int dev = 0, can = 0, per_sm = 0, sms = 0;
    GW_CUDA(cudaGetDevice(&dev));
    GW_CUDA(cudaDeviceGetAttribute(&can, cudaDevAttrCooperativeLaunch, dev));
    GW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, house_coop_kernel, ET, 0));
    if (can && per_sm >= 1) {
      unsigned* bar = (unsigned*)mem.get(1);  // count, generation
      GW_CUDA(cudaMemsetAsync(bar, 0, 8, s));
      int n_arg = n;
      int* tflag = flags + FLAG_TIMEOUT;
      void* args[] = {&n_arg, &A, &pv, &tau, &d, &e, &bar, &tflag};
      // one such launch at a time in the process (setups may run on several host threads): two
      // grids that each hold part of the SMs while waiting for the rest could only time out
      static std::mutex coop_mu;
      std::lock_guard<std::mutex> lock(coop_mu);
      const cudaError_t ce = cudaLaunchCooperativeKernel((const void*)house_coop_kernel,
                                                         dim3(sms), dim3(ET), args, 0, s);
      if (ce == cudaSuccess)
        coop = true;
      else
        cudaGetLastError();
      GW_CUDA(cudaStreamSynchronize(s));
    }
  }
  for (int k = 0; !coop && k + 2 < n; ++k) {
    const int m = n - k - 1;
    house_kernel<<<1, ET, 0, s>>>(n, k, A, vb, tau, d, e);
    house_matvec_kernel<<<ceil_div(m, ET / 32), ET, 0, s>>>(n, k, A, vb, tau, pv);
    house_w_kernel<<<1, ET, 0, s>>>(n, k, vb, tau, pv, wv);
    house_update_kernel<<<dim3(ceil_div(m, 32), ceil_div(m, 32)), ET, 0, s>>>(n, k, A, vb, wv);
  }
  house_tail_kernel<<<1, 32, 0, s>>>(n, A, d, e);
  GW_CHECK_LAUNCH();
  if (coop) {
    int hf[FLAG_COUNT];
    GW_CUDA(cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, s));
    GW_CUDA(cudaStreamSynchronize(s));
    GW_REQUIRE(!hf[FLAG_TIMEOUT], GWAS_ERR_TIMEOUT,
               "the Householder reduction gave up waiting at a grid barrier");
  }
  // 2. eigenvalues by multisection within the Gershgorin interval
  std::vector<double> hd(n), he(n), he2(n), hw(n), hs(n);
  GW_CUDA(cudaMemcpyAsync(hd.data(), d, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  GW_CUDA(cudaMemcpyAsync(he.data(), e, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  GW_CUDA(cudaStreamSynchronize(s));
  double gl = INFINITY, gu = -INFINITY, emax2 = 0.0;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? fabs(he[i - 1]) : 0.0) + (i + 1 < n ? fabs(he[i]) : 0.0);
    gl = fmin(gl, hd[i] - r);
    gu = fmax(gu, hd[i] + r);
    he2[i] = i + 1 < n ? he[i] * he[i] : 0.0;
    emax2 = fmax(emax2, he2[i]);
  }
  const double anorm = fmax(fabs(gl), fabs(gu));
  GW_REQUIRE(isfinite(anorm), GWAS_ERR_NOT_SPD, "the kinship matrix has non-finite entries");
  gl -= 2.3e-16 * anorm * n + 1e-300;
  gu += 2.3e-16 * anorm * n + 1e-300;
  const double pivmin = 2.3e-308 * fmax(1.0, emax2);
  GW_CUDA(cudaMemcpyAsync(e2, he2.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  // one warp per eigenvalue, four per CTA
  bisect_kernel<<<ceil_div(n, 4), 128, 0, s>>>(n, d, e2, gl, gu, pivmin, w);
  GW_CHECK_LAUNCH();
  GW_CUDA(cudaMemcpyAsync(hw.data(), w, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  GW_CUDA(cudaStreamSynchronize(s));
  // 3. shifts: an eigenvalue's own, or for a cluster (gaps <= 1e-12 ||T||) one shift below it
  for (int i = 0; i < n;) {
    int j = i;
    while (j + 1 < n && hw[j + 1] - hw[j] <= 1e-12 * anorm) ++j;
    if (j == i) {
      hs[i] = hw[i];
    } else {
      const double spread = hw[j] - hw[i];
      double out = INFINITY;
      if (i > 0) out = fmin(out, hw[i] - hw[i - 1]);
      if (j + 1 < n) out = fmin(out, hw[j + 1] - hw[j]);
      double delta = fmin(1e-8 * anorm, 0.1 * out);
      delta = fmax(delta, fmax(100.0 * spread, 1e-15 * anorm));
      for (int k = i; k <= j; ++k) hs[k] = hw[i] - delta;
    }
    i = j + 1;
  }
  GW_CUDA(cudaMemcpyAsync(sg, hs.data(), sizeof(double) * n, cudaMemcpyHostToDevice, s));
  invit_kernel<<<ceil_div(n, 32), 32, 0, s>>>(n, d, e, sg, anorm, wk, wk + nn, wk + 2 * nn,
                                               wk + 3 * nn, S);
  GW_CHECK_LAUNCH();
  // 4. Cholesky QR, twice: G = S^T S = L L^T, S := S L^-T (the Cholesky reads the lower triangle
  //    of G only; L^-T is upper triangular)
  double* Sc = S;
  double* So = wk;
  for (int pass = 0; pass < 2; ++pass) {
    gemm_f64(s, n, n, n, 1.0, Sc, n, 1, Sc, 1, n, 0.0, G, 1, n, /*lower_only=*/true);
    cholesky(s, n, G, flags);
    tri_inverse(s, n, G, Li, W2);
    gemm_f64(s, n, n, n, 1.0, Sc, 1, n, Li, 1, n, 0.0, So, 1, n, false, /*b_tri=*/1);
    std::swap(Sc, So);
  }
  int hflags[FLAG_COUNT];
  GW_CUDA(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
  GW_CUDA(cudaStreamSynchronize(s));
  if (hflags[FLAG_NOT_SPD]) return -1;
  // 5. Z = H_0 H_1 ... H_{n-3} S (column c of Z = row c of Zt)
  GW_CUDA(cudaMemcpyAsync(Zt, Sc, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s));
  if (n >= 3) {
    // one warp per column; as many columns per CTA (up to BT_WARPS) as n doubles each fit in
    // 200 KB of shared memory (n <= 16384: at least one)
    const int warps = (int)std::max<int64_t>(
        1, std::min<int64_t>(BT_WARPS, (int64_t)(200 * 1024) / ((int64_t)n * 8)));
    const size_t smem = (size_t)warps * n * 8;
    GW_CUDA(cudaFuncSetAttribute(bt_columns_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    bt_columns_kernel<<<ceil_div(n, warps), 32 * warps, smem, s>>>(n, A, tau, Zt);
    GW_CHECK_LAUNCH();
  }
  GW_CUDA(cudaStreamSynchronize(s));
  return 0;
}

int eigh_f64(cudaStream_t s, int n, const double* Phi, double* Zt, double* w, double* U,
             int* flags) {
  if (eigh_tridiag(s, n, Phi, Zt, w) == 0) return 0;
  return jacobi_eig(s, n, Phi, Zt, w, U, flags, 60);
}

}  // namespace gw
