// The C ABI (include/gwas.h): handle, FP64 setup on the device and the streamed scan.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

#define GW_API extern "C" __attribute__((visibility("default")))

namespace gw {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}

}  // namespace gw

using namespace gw;

struct gwas_handle_s {
  // prec: the scan's path (SPLIT_FP8 runs the tensor-core path of SPLIT_BF16, so prec holds
  // SPLIT_BF16 then and fp8 is set); prec_opt: the precision the caller asked for
  int dev = 0, n = 0, q = 0, p = 0, t = 0, algo = 0, prec = 0, prec_opt = 0, validate = 0;
  bool fp8 = false;
  int model = GWAS_MODEL_ADDITIVE;  // genetic model: the SNP's pr columns, p = q + pr
  GeneticModel gm;
  int out_snp = 0;  // GWAS_OUT_SNP: B holds (b_R, se_R) per pair
  int out_var = 0;  // GWAS_OUT_VAR: B holds b, then Var(b) packed (p(p+1)/2) per pair
  int pw = 0;       // values per pair in B: p, 2 pr with out_snp, p + p(p+1)/2 with out_var
  int block_snps = 0;
  // block_snps = 0 at setup: the streaming block is chosen by timing on the first streamed call
  bool block_auto = false, block_tuned = false;
  int ntune = 0;
  int64_t tune_b[8] = {};
  double tune_ms[8][3] = {};  // per candidate: H2D copy, scan, D2H copy (ms)
  int ldp = 0;  // n rounded up to 64: leading dimension of padded per-individual operands
  double setup_ms = 0.0;
  // st: setup and flag reads; st_lane: second compute stream of streamed scans; st_h2d /
  // st_d2h: copies of streamed scans
  cudaStream_t st = nullptr, st_lane = nullptr, st_h2d = nullptr, st_d2h = nullptr;
  static constexpr int NRING = 4;  // streaming buffers at most (2, or 4 with two lanes)
  cudaEvent_t ev_loaded[NRING] = {}, ev_computed[NRING] = {}, ev_drained[NRING] = {};
  cudaEvent_t ev_begin = nullptr, ev_lane_done = nullptr;
  int* flags = nullptr;
  int* h_flags = nullptr;
  // per-trait null-model block (both algorithms)
  double *P = nullptr, *b0 = nullptr, *rw = nullptr;
  float *P32 = nullptr, *b032 = nullptr, *rw32 = nullptr;
  // CHOL
  double *Linv = nullptr, *XLw = nullptr;
  float *Linv32 = nullptr, *XLw32 = nullptr;
  // EIG
  double *Zt = nullptr, *w = nullptr, *XLt = nullptr, *planes = nullptr;
  float *Zt32 = nullptr, *planes32 = nullptr;
  // scratch for the rotated block (EIG)
  void* xt = nullptr;
  int64_t xt_cap = 0;
  // streaming ring (genotype bytes and outputs of one block per buffer); nring allocated
  uint8_t* ring[NRING] = {};
  void* oring[NRING] = {};
  size_t ring_bytes = 0, oring_bytes = 0;
  int nring = 0;
  // format conversion scratch: packed rows for the tensor-core path (int8 input), int8 rows for
  // the CUDA-core paths (packed input)
  uint8_t* pk = nullptr;
  int64_t pk_cap = 0;
  int8_t* u8 = nullptr;
  int64_t u8_cap = 0;
  // CUDA graph of the device work of one full block in ring slot i (host input and output),
  // captured on first use and replayed; valid while its key (buffers, block, format) holds
  struct BlockGraph {
    cudaGraphExec_t exec = nullptr;
    const void *ring = nullptr, *oring = nullptr;
    int64_t blk = 0;
    int fmt = -1;
    bool f64 = false, wald = false;
  };
  BlockGraph graphs[NRING];
  cudaStream_t st_cap = nullptr;  // graphs are captured here
  int64_t graph_launches = 0;
  // tensor-core state; split pieces per trait (CHOL) or of every U_j (EIG, pieces[0])
  TcState* tc = nullptr;
  std::vector<int> pieces;
  std::vector<void*> allocs;
  StageTimer timer;  // per-stage events (gwas_stage_timing)
};

namespace {

void* dalloc(gwas_handle h, size_t bytes) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    throw Fail{GWAS_ERR_OOM};
  }
  h->allocs.push_back(p);
  return p;
}

template <typename T>
T* dalloc_t(gwas_handle h, size_t count) {
  return (T*)dalloc(h, count * sizeof(T));
}

void dfree(gwas_handle h, void* p) {
  if (!p) return;
  for (size_t i = 0; i < h->allocs.size(); ++i)
    if (h->allocs[i] == p) {
      cudaFree(p);
      h->allocs.erase(h->allocs.begin() + i);
      return;
    }
}

void destroy_impl(gwas_handle h) {
  if (!h) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h->dev);
  if (h->st) cudaStreamSynchronize(h->st);
  if (h->st_lane) cudaStreamSynchronize(h->st_lane);
  if (h->st_h2d) cudaStreamSynchronize(h->st_h2d);
  if (h->st_d2h) cudaStreamSynchronize(h->st_d2h);
  if (h->tc) tc_destroy(h->tc);
  h->timer.destroy();
  for (auto& gph : h->graphs)
    if (gph.exec) cudaGraphExecDestroy(gph.exec);
  if (h->st_cap) cudaStreamDestroy(h->st_cap);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_flags) cudaFreeHost(h->h_flags);
  for (int i = 0; i < gwas_handle_s::NRING; ++i) {
    if (h->ev_loaded[i]) cudaEventDestroy(h->ev_loaded[i]);
    if (h->ev_computed[i]) cudaEventDestroy(h->ev_computed[i]);
    if (h->ev_drained[i]) cudaEventDestroy(h->ev_drained[i]);
  }
  if (h->ev_begin) cudaEventDestroy(h->ev_begin);
  if (h->ev_lane_done) cudaEventDestroy(h->ev_lane_done);
  if (h->st) cudaStreamDestroy(h->st);
  if (h->st_lane) cudaStreamDestroy(h->st_lane);
  if (h->st_h2d) cudaStreamDestroy(h->st_h2d);
  if (h->st_d2h) cudaStreamDestroy(h->st_d2h);
  delete h;
  cudaSetDevice(cur);
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    GW_CUDA(cudaSetDevice(dev));
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

void read_flags(gwas_handle h, cudaStream_t s) {
  GW_CUDA(cudaMemcpyAsync(h->h_flags, h->flags, sizeof(int) * FLAG_COUNT, cudaMemcpyDeviceToHost, s));
  GW_CUDA(cudaStreamSynchronize(s));
}

// After a synchronisation: a kernel of this handle whose bounded wait gave up makes the call
// fail with GWAS_ERR_TIMEOUT (the flag is cleared, so the handle stays usable).
void check_timeout(gwas_handle h, cudaStream_t s) {
  read_flags(h, s);
  if (h->h_flags[FLAG_TIMEOUT]) {
    GW_CUDA(cudaMemsetAsync(h->flags + FLAG_TIMEOUT, 0, sizeof(int), s));
    GW_CUDA(cudaStreamSynchronize(s));
    GW_REQUIRE(false, GWAS_ERR_TIMEOUT,
               "a tensor-core kernel gave up waiting (its outputs for this call are incomplete)");
  }
}

// The CHOL route of an EIG handle (traits past KAPPA_CHOL_ROUTE): Algorithm 3's setup for those
// traits only -- M_j, L_j, L_j^-1, L_j^-1 X_L, L_j^-1 y_j, S_TL, b0, the whitened residual --
// then a CHOL tensor-core state over them (three BF16 pieces of each augmented L_j^-1), which the
// EIG state runs after its own kernels.
void attach_chol_route(gwas_handle h, cudaStream_t s, const std::vector<int>& route,
                       const double* dPhi, const double* dXL, const double* dY, const double* h2,
                       const double* s2, const TcSetupArgs& eig_args) {
  const int n = h->n, q = h->q, tr = (int)route.size();
  const size_t nn = (size_t)n * n;
  double* Lr = dalloc_t<double>(h, (size_t)tr * nn);
  double* XLwr = dalloc_t<double>(h, (size_t)tr * q * n);
  double* ywr = dalloc_t<double>(h, (size_t)tr * n);
  double* rwr = dalloc_t<double>(h, (size_t)tr * n);
  double* Pr = dalloc_t<double>(h, (size_t)tr * q * q);  // kept: the CHOL kernel reads P_j, b0_j
  double* b0r = dalloc_t<double>(h, (size_t)tr * q);
  double* A = dalloc_t<double>(h, nn);
  double* work = dalloc_t<double>(h, nn > 3 * (size_t)n + 1 ? nn : 3 * (size_t)n + 1);
  for (int k = 0; k < tr; ++k) {
    const int j = route[k];
    double* Lk = Lr + (size_t)k * nn;
    form_M(s, n, dPhi, h2[j], s2[j], A);
    cholesky(s, n, A, h->flags);
    tri_inverse(s, n, A, Lk, work);
    gemm_f64(s, q, n, n, 1.0, dXL, n, 1, Lk, 1, n, 0.0, XLwr + (size_t)k * q * n, n, 1);
    gemm_f64(s, 1, n, n, 1.0, dY + (size_t)j * n, 0, 1, Lk, 1, n, 0.0, ywr + (size_t)k * n, 0, 1);
  }
  TraitPackArgs tp{n, q, tr, XLwr, (int64_t)q * n, ywr, nullptr, Pr, b0r, rwr, h->flags};
  trait_pack(s, tp);
  TcSetupArgs ta = eig_args;
  ta.algo = GWAS_ALGO_CHOL;
  ta.t = tr;
  ta.Linv = Lr;
  ta.XLw = XLwr;
  ta.rw = rwr;
  ta.P = Pr;
  ta.b0 = b0r;
  std::vector<int> three(tr, 3);
  ta.pieces = three.data();
  ta.fp8_lo = 0;
  TcState* rs = tc_setup(s, ta);
  try {
    tc_attach_chol_route(s, h->tc, rs, route);
  } catch (...) {
    tc_destroy(rs);
    throw;
  }
  for (double* p : {Lr, XLwr, ywr, rwr, A, work}) dfree(h, p);
}

void setup_impl(gwas_handle h, const double* Phi, const double* XL, const double* Y,
                const double* h2, const double* s2) {
  const int n = h->n, q = h->q, t = h->t;
  std::vector<int> route;  // EIG traits the CHOL kernel scans as well
  const size_t nn = (size_t)n * n;
  cudaStream_t s = h->st;
  double* dPhi = dalloc_t<double>(h, nn);
  double* dXL = dalloc_t<double>(h, (size_t)n * q);
  double* dY = dalloc_t<double>(h, (size_t)n * t);
  double* dh2 = dalloc_t<double>(h, t);
  double* ds2 = dalloc_t<double>(h, t);
  GW_CUDA(cudaMemcpyAsync(dPhi, Phi, nn * 8, cudaMemcpyHostToDevice, s));
  GW_CUDA(cudaMemcpyAsync(dXL, XL, (size_t)n * q * 8, cudaMemcpyHostToDevice, s));
  GW_CUDA(cudaMemcpyAsync(dY, Y, (size_t)n * t * 8, cudaMemcpyHostToDevice, s));
  GW_CUDA(cudaMemcpyAsync(dh2, h2, (size_t)t * 8, cudaMemcpyHostToDevice, s));
  GW_CUDA(cudaMemcpyAsync(ds2, s2, (size_t)t * 8, cudaMemcpyHostToDevice, s));
  GW_CUDA(cudaMemsetAsync(h->flags, 0, sizeof(int) * FLAG_COUNT, s));
  cudaEvent_t e0, e1;
  GW_CUDA(cudaEventCreate(&e0));
  GW_CUDA(cudaEventCreate(&e1));
  GW_CUDA(cudaEventRecord(e0, s));

  h->P = dalloc_t<double>(h, (size_t)t * q * q);
  h->b0 = dalloc_t<double>(h, (size_t)t * q);
  h->rw = dalloc_t<double>(h, (size_t)t * n);
  double* yw = dalloc_t<double>(h, (size_t)t * n);
  int sweeps = 0;
  if (h->algo == GWAS_ALGO_CHOL) {
    // Algorithm 3's setup for every trait: M_j, L_j, L_j^-1, L_j^-1 X_L, L_j^-1 y_j
    h->Linv = dalloc_t<double>(h, (size_t)t * nn);
    h->XLw = dalloc_t<double>(h, (size_t)t * q * n);
    double* A = dalloc_t<double>(h, nn);
    double* work = dalloc_t<double>(h, nn > 3 * (size_t)n + 1 ? nn : 3 * (size_t)n + 1);
    h->pieces.assign(t, 2);
    for (int j = 0; j < t; ++j) {
      double hj = h2[j], sj = s2[j];
      double* Lj = h->Linv + (size_t)j * nn;
      form_M(s, n, dPhi, hj, sj, A);
      cholesky(s, n, A, h->flags);
      tri_inverse(s, n, A, Lj, work);
      if (h->prec == GWAS_PREC_SPLIT_BF16) {
        read_flags(h, s);  // a failed factorisation is reported below; skip its estimate
        if (!h->h_flags[FLAG_NOT_SPD] &&
            condition_estimate(s, n, A, Lj, work, 24) > KAPPA_THIRD_PIECE)
          h->pieces[j] = 3;
      }
      // XLw_j (q x n, row k) = L^-1 X_L[:, k];  yw_j = L^-1 y_j
      gemm_f64(s, q, n, n, 1.0, dXL, n, 1, Lj, 1, n, 0.0, h->XLw + (size_t)j * q * n, n, 1);
      gemm_f64(s, 1, n, n, 1.0, dY + (size_t)j * n, 0, 1, Lj, 1, n, 0.0, yw + (size_t)j * n, 0, 1);
    }
    dfree(h, A);
    dfree(h, work);
    TraitPackArgs ta{n, q, t, h->XLw, (int64_t)q * n, yw, nullptr, h->P, h->b0, h->rw, h->flags};
    trait_pack(s, ta);
  } else {
    // Algorithm 4's setup: Phi = Z W Z^T, X~_L = Z^T X_L, Y~ = Z^T Y; then per trait
    // D_j, S_TL, b_T and the operand planes of the pair reduction.
    h->Zt = dalloc_t<double>(h, nn);
    h->w = dalloc_t<double>(h, n);
    double* U = dalloc_t<double>(h, nn);
    sweeps = eigh_f64(s, n, dPhi, h->Zt, h->w, U, h->flags);
    dfree(h, U);
    GW_REQUIRE(sweeps >= 0, GWAS_ERR_NOT_CONVERGED, "the eigensolver did not converge");
    h->XLt = dalloc_t<double>(h, (size_t)q * n);
    gemm_f64(s, q, n, n, 1.0, dXL, n, 1, h->Zt, 1, n, 0.0, h->XLt, n, 1);
    gemm_f64(s, t, n, n, 1.0, dY, n, 1, h->Zt, 1, n, 0.0, yw, n, 1);
    double* d = dalloc_t<double>(h, (size_t)t * n);
    eig_weights(s, n, t, h->w, dh2, ds2, d, h->flags);
    // conditioning of each M_j from the eigenvalues of Phi: one number decides the U pieces;
    // traits past KAPPA_CHOL_ROUTE are scanned by the CHOL kernel as well (route)
    h->pieces.assign(1, 2);
    route.clear();
    if (h->prec == GWAS_PREC_SPLIT_BF16) {
      std::vector<double> hw(n);
      GW_CUDA(cudaMemcpyAsync(hw.data(), h->w, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
      GW_CUDA(cudaStreamSynchronize(s));
      double wmin = hw[0], wmax = hw[0];
      for (int r = 1; r < n; ++r) {
        wmin = hw[r] < wmin ? hw[r] : wmin;
        wmax = hw[r] > wmax ? hw[r] : wmax;
      }
      for (int j = 0; j < t; ++j) {
        const double lo = h2[j] * wmin + 1.0 - h2[j], hi = h2[j] * wmax + 1.0 - h2[j];
        if (lo > 0.0 && hi / lo > KAPPA_THIRD_PIECE) h->pieces[0] = 3;
        if (lo > 0.0 && hi / lo > KAPPA_CHOL_ROUTE) route.push_back(j);
      }
    }
    TraitPackArgs ta{n, q, t, h->XLt, 0, yw, d, h->P, h->b0, h->rw, h->flags};
    trait_pack(s, ta);
    h->planes = dalloc_t<double>(h, (size_t)t * (q + 2) * h->ldp);
    eig_planes_f64(s, n, q, t, h->ldp, h->XLt, d, h->rw, h->planes);
    dfree(h, d);
  }
  dfree(h, yw);

  if (h->prec == GWAS_PREC_FP32) {
    h->P32 = dalloc_t<float>(h, (size_t)t * q * q);
    h->b032 = dalloc_t<float>(h, (size_t)t * q);
    convert_f64_to_f32(s, h->P, h->P32, (int64_t)t * q * q);
    convert_f64_to_f32(s, h->b0, h->b032, (int64_t)t * q);
    if (h->algo == GWAS_ALGO_CHOL) {
      h->Linv32 = dalloc_t<float>(h, (size_t)t * nn);
      h->XLw32 = dalloc_t<float>(h, (size_t)t * q * n);
      h->rw32 = dalloc_t<float>(h, (size_t)t * n);
      convert_f64_to_f32(s, h->Linv, h->Linv32, (int64_t)t * nn);
      convert_f64_to_f32(s, h->XLw, h->XLw32, (int64_t)t * q * n);
      convert_f64_to_f32(s, h->rw, h->rw32, (int64_t)t * n);
    } else {
      h->Zt32 = dalloc_t<float>(h, nn);
      h->planes32 = dalloc_t<float>(h, (size_t)t * (q + 2) * h->ldp);
      convert_f64_to_f32(s, h->Zt, h->Zt32, (int64_t)nn);
      convert_f64_to_f32(s, h->planes, h->planes32, (int64_t)t * (q + 2) * h->ldp);
    }
  } else if (h->prec == GWAS_PREC_SPLIT_BF16) {
    TcSetupArgs ta{};
    ta.algo = h->algo; ta.n = n; ta.q = q; ta.t = t;
    ta.Linv = h->Linv; ta.XLw = h->XLw; ta.rw = h->rw;
    ta.Zt = h->Zt; ta.planes = h->planes; ta.ldp = h->ldp;
    ta.P = h->P; ta.b0 = h->b0;
    ta.block_snps = h->block_snps;
    ta.out_snp = h->out_snp;
    ta.out_var = h->out_var;
    ta.gm = h->gm;
    ta.pieces = h->pieces.data();
    ta.fp8_lo = h->fp8 && h->algo == GWAS_ALGO_CHOL ? 1 : 0;
    ta.intercept = 1;
    for (int i = 0; i < n; ++i)
      if (XL[i] != 1.0) ta.intercept = 0;
    h->tc = tc_setup(s, ta);
    if (!route.empty()) attach_chol_route(h, s, route, dPhi, dXL, dY, h2, s2, ta);
  }
  GW_CUDA(cudaEventRecord(e1, s));
  GW_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  GW_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  h->setup_ms = ms;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  read_flags(h, s);
  GW_REQUIRE(!h->h_flags[FLAG_NOT_SPD], GWAS_ERR_NOT_SPD,
             "M_j = s2 (h2 Phi + (1-h2) I) is not positive definite");
  GW_REQUIRE(!h->h_flags[FLAG_STL_SINGULAR], GWAS_ERR_SINGULAR,
             "X_L^T M^-1 X_L is singular: covariates are collinear");
  GW_CUDA(cudaMemsetAsync(h->flags, 0, sizeof(int) * FLAG_COUNT, s));
  dfree(h, dPhi);
  dfree(h, dXL);
  dfree(h, dY);
  dfree(h, dh2);
  dfree(h, ds2);
  if (h->algo == GWAS_ALGO_EIG && h->prec != GWAS_PREC_FP64) {
    dfree(h, h->planes);
    h->planes = nullptr;
  }
  if (h->algo == GWAS_ALGO_CHOL && h->prec != GWAS_PREC_FP64) {
    dfree(h, h->Linv);
    h->Linv = nullptr;
  }
  GW_CUDA(cudaStreamSynchronize(s));
}

// Scratch of the EIG CUDA-core path: the rotated genetic columns of up to `snps` SNPs.
void ensure_xt(gwas_handle h, int64_t snps) {
  if (h->algo != GWAS_ALGO_EIG || h->prec == GWAS_PREC_SPLIT_BF16) return;
  if (snps <= h->xt_cap) return;
  if (h->xt) {
    GW_CUDA(cudaDeviceSynchronize());
    dfree(h, h->xt);
  }
  const size_t es = h->prec == GWAS_PREC_FP64 ? 8 : 4;
  h->xt = dalloc(h, (size_t)snps * h->gm.pr * h->ldp * es);
  h->xt_cap = snps;
}

enum { FMT_INT8 = 0, FMT_PACKED2 = 1 };

size_t row_bytes_of(gwas_handle h, int fmt) {
  return fmt == FMT_PACKED2 ? (size_t)packed_row_bytes(h->n) : (size_t)h->n;
}

// Grows a conversion scratch of `snps` rows of `row_bytes` (waits for queued work first).
template <typename T>
void ensure_rows(gwas_handle h, T*& buf, int64_t& cap, int64_t snps, size_t row_bytes) {
  if (snps <= cap) return;
  if (buf) {
    GW_CUDA(cudaDeviceSynchronize());
    dfree(h, buf);
    buf = nullptr;
  }
  buf = (T*)dalloc(h, (size_t)snps * row_bytes);
  cap = snps;
}

// SNPs converted per pass when a scan's input format differs from its kernels' format: the
// streaming block, or up to 1 GiB of converted rows for device-resident input.
int64_t convert_chunk(gwas_handle h, int64_t m, size_t row_bytes) {
  int64_t c = (int64_t)(((size_t)1 << 30) / row_bytes);
  c = m < c ? m : c;
  return c > h->block_snps ? c : (m < h->block_snps ? m : h->block_snps);
}

// CUDA-core scan of int8 rows already on the device; asynchronous on s.
void scan_block_simt(gwas_handle h, const int8_t* XR, int64_t m, void* B, void* wald,
                     bool out_f64, cudaStream_t s) {
  const int n = h->n, q = h->q, t = h->t;
  if (h->algo == GWAS_ALGO_CHOL) {
    for (int j = 0; j < t; ++j) {
      if (h->prec == GWAS_PREC_FP64) {
        CholScanArgs<double> a{n, q, t, j, h->Linv + (size_t)j * n * n, h->XLw + (size_t)j * q * n,
                               h->rw + (size_t)j * n, h->P + (size_t)j * q * q, h->b0 + (size_t)j * q,
                               XR, m, 0, B, wald, out_f64, 1e-12, h->flags};
        a.out_snp = h->out_snp;
        a.out_var = h->out_var;
        a.gm = h->gm;
        chol_scan_simt<double>(s, a);
      } else {
        CholScanArgs<float> a{n, q, t, j, h->Linv32 + (size_t)j * n * n, h->XLw32 + (size_t)j * q * n,
                              h->rw32 + (size_t)j * n, h->P32 + (size_t)j * q * q, h->b032 + (size_t)j * q,
                              XR, m, 0, B, wald, out_f64, 1e-5f, h->flags};
        a.out_snp = h->out_snp;
        a.out_var = h->out_var;
        a.gm = h->gm;
        chol_scan_simt<float>(s, a);
      }
    }
    return;
  }
  // EIG on CUDA cores: chunks that fit the scratch (same stream, so chunks serialise)
  const int64_t cap = h->xt_cap;
  for (int64_t off = 0; off < m; off += cap) {
    const int64_t mm = m - off < cap ? m - off : cap;
    const size_t ob = out_f64 ? 8 : 4;
    void* Bc = (char*)B + (size_t)off * t * h->pw * ob;
    void* Wc = wald ? (char*)wald + (size_t)off * t * ob : nullptr;
    if (h->prec == GWAS_PREC_FP64) {
      EigScanArgs<double> a{n, q, t, h->Zt, h->planes, h->ldp, h->P, h->b0, XR + off * n, mm, 0,
                            Bc, Wc, out_f64, 1e-12, (double*)h->xt, h->flags};
      a.out_snp = h->out_snp;
      a.out_var = h->out_var;
      a.gm = h->gm;
      eig_scan_simt<double>(s, a);
    } else {
      EigScanArgs<float> a{n, q, t, h->Zt32, h->planes32, h->ldp, h->P32, h->b032, XR + off * n, mm,
                           0, Bc, Wc, out_f64, 1e-5f, (float*)h->xt, h->flags};
      a.out_snp = h->out_snp;
      a.out_var = h->out_var;
      a.gm = h->gm;
      eig_scan_simt<float>(s, a);
    }
  }
}

// One block of m SNPs already on the device (int8 rows or packed rows, `fmt`), outputs on the
// device; asynchronous on s.  The tensor-core kernels read packed rows, the CUDA-core kernels
// int8 rows: input in the other format is converted chunk by chunk into the handle's scratch.
void scan_block(gwas_handle h, const void* X, int fmt, int64_t m, void* B, void* wald,
                bool out_f64, cudaStream_t s) {
  const int n = h->n, t = h->t, p = h->pw;
  const size_t rbi = row_bytes_of(h, fmt);
  const size_t ob = out_f64 ? 8 : 4;
  if (h->prec == GWAS_PREC_SPLIT_BF16) {
    TcScanArgs a{};
    a.flags = h->flags;
    a.timer = &h->timer;
    if (fmt == FMT_PACKED2) {
      GW_REQUIRE(((uintptr_t)X & 15) == 0, GWAS_ERR_ARG,
                 "packed genotypes on the device must start on a 16-byte boundary");
      if (h->validate) validate_packed(s, (const uint8_t*)X, m, n, h->flags);
      a.G = (const uint8_t*)X;
      a.m = m;
      a.B = (float*)B;
      a.wald = (float*)wald;
      tc_scan(s, h->tc, a);
      return;
    }
    const size_t rb = (size_t)packed_row_bytes(n);
    const int64_t chunk = convert_chunk(h, m, rb);
    ensure_rows(h, h->pk, h->pk_cap, chunk, rb);
    for (int64_t off = 0; off < m; off += chunk) {
      const int64_t mm = m - off < chunk ? m - off : chunk;
      cudaEvent_t ev = h->timer.begin(s, STAGE_PACK);
      pack_genotypes(s, (const int8_t*)X + off * n, mm, n, h->pk, h->flags, h->validate != 0);
      h->timer.end(s, ev);
      a.G = h->pk;
      a.m = mm;
      a.B = (float*)B + (size_t)off * t * p;
      a.wald = wald ? (float*)wald + (size_t)off * t : nullptr;
      tc_scan(s, h->tc, a);
    }
    return;
  }
  if (fmt == FMT_INT8) {
    if (h->validate) validate_genotypes(s, (const int8_t*)X, m * n, h->flags);
    cudaEvent_t ev = h->timer.begin(s, STAGE_SIMT);
    scan_block_simt(h, (const int8_t*)X, m, B, wald, out_f64, s);
    h->timer.end(s, ev);
    return;
  }
  const int64_t chunk = convert_chunk(h, m, (size_t)n);
  ensure_rows(h, h->u8, h->u8_cap, chunk, (size_t)n);
  for (int64_t off = 0; off < m; off += chunk) {
    const int64_t mm = m - off < chunk ? m - off : chunk;
    const uint8_t* src = (const uint8_t*)X + off * rbi;
    if (h->validate) validate_packed(s, src, mm, n, h->flags);
    cudaEvent_t ev = h->timer.begin(s, STAGE_PACK);
    unpack_genotypes(s, src, mm, n, h->u8);
    h->timer.end(s, ev);
    ev = h->timer.begin(s, STAGE_SIMT);
    scan_block_simt(h, h->u8, mm, (char*)B + (size_t)off * t * p * ob,
                    wald ? (char*)wald + (size_t)off * t * ob : nullptr, out_f64, s);
    h->timer.end(s, ev);
  }
}

// Conversion scratch a block of `blk` SNPs in format `fmt` needs, allocated ahead (no device
// allocation may happen while a graph is being captured).
void prepare_scratch(gwas_handle h, int fmt, int64_t blk) {
  if (h->prec == GWAS_PREC_SPLIT_BF16 && fmt == FMT_INT8) {
    const size_t rb = (size_t)packed_row_bytes(h->n);
    ensure_rows(h, h->pk, h->pk_cap, convert_chunk(h, blk, rb), rb);
  } else if (h->prec != GWAS_PREC_SPLIT_BF16 && fmt == FMT_PACKED2) {
    ensure_rows(h, h->u8, h->u8_cap, convert_chunk(h, blk, (size_t)h->n), (size_t)h->n);
  }
  ensure_xt(h, blk);
}

// The graph of ring slot `buf`'s device work for a full block: captured on first use (or when
// the slot's buffers or the block changed) on the handle's capture stream, replayed after.
cudaGraphExec_t block_graph(gwas_handle h, int buf, int fmt, int64_t blk, bool out_f64, bool wald) {
  gwas_handle_s::BlockGraph& g = h->graphs[buf];
  if (g.exec && g.ring == h->ring[buf] && g.oring == h->oring[buf] && g.blk == blk &&
      g.fmt == fmt && g.f64 == out_f64 && g.wald == wald)
    return g.exec;
  if (g.exec) {
    GW_CUDA(cudaGraphExecDestroy(g.exec));
    g.exec = nullptr;
  }
  prepare_scratch(h, fmt, blk);
  const size_t ob = out_f64 ? 8 : 4;
  void* Bo = h->oring[buf];
  void* Wo = wald ? (char*)h->oring[buf] + (size_t)blk * h->t * h->pw * ob : nullptr;
  const bool timer_on = h->timer.on;  // replays are not timed per stage
  h->timer.on = false;
  GW_CUDA(cudaStreamBeginCapture(h->st_cap, cudaStreamCaptureModeThreadLocal));
  try {
    scan_block(h, h->ring[buf], fmt, blk, Bo, Wo, out_f64, h->st_cap);
  } catch (...) {
    cudaGraph_t gr = nullptr;
    cudaStreamEndCapture(h->st_cap, &gr);
    if (gr) cudaGraphDestroy(gr);
    h->timer.on = timer_on;
    throw;
  }
  h->timer.on = timer_on;
  cudaGraph_t gr = nullptr;
  GW_CUDA(cudaStreamEndCapture(h->st_cap, &gr));
  cudaError_t e = cudaGraphInstantiate(&g.exec, gr, 0);
  cudaGraphDestroy(gr);
  GW_CUDA(e);
  g.ring = h->ring[buf];
  g.oring = h->oring[buf];
  g.blk = blk;
  g.fmt = fmt;
  g.f64 = out_f64;
  g.wald = wald;
  return g.exec;
}

// block_snps = 0: on the first streamed call the handle times the three stages of its pipeline
// -- the H2D copy of a block, the block's scan, the D2H copy of its outputs -- at each candidate
// block size, on the call's own first SNPs (written again by the scan that follows), and keeps
// the size that minimises the modelled time of this call: the pipeline's fill (the three stages
// of one block) plus, for every further block, its slowest stage (the scan shared by the lanes
// that run in parallel).
void tune_block(gwas_handle h, const void* X, int fmt, int64_t m, int xr_dev, void* B,
                void* wald, int out_dev, bool out_f64, cudaStream_t s, int lanes) {
  const int t = h->t, p = h->pw;
  const size_t ob = out_f64 ? 8 : 4;
  const size_t rbi = row_bytes_of(h, fmt);
  const int64_t out_cap = (int64_t)(2e9 / ((double)t * (p + 1) * 8));
  std::vector<int64_t> cands;
  for (int64_t b = 8192; b <= 262144 && b <= out_cap; b *= 2)
    if (b <= m || cands.empty()) cands.push_back(b < m ? b : m);
  if (cands.empty()) cands.push_back(out_cap < m ? (out_cap > 64 ? out_cap : 64) : m);
  const int64_t bmax = cands.back();
  uint8_t* gtmp = xr_dev ? nullptr : (uint8_t*)dalloc(h, (size_t)bmax * rbi);
  void* otmp = out_dev ? nullptr : dalloc(h, (size_t)bmax * t * (p + 1) * ob);
  prepare_scratch(h, fmt, bmax);
  cudaEvent_t ev[6];
  for (auto& e : ev) GW_CUDA(cudaEventCreate(&e));
  h->ntune = 0;
  double best = 1e300;
  int64_t best_b = cands[0];
  for (int rep = 0; rep < 2; ++rep) {  // the first pass warms up; the second is timed
    for (int64_t b : cands) {
      const void* src = X;
      if (!xr_dev) {
        GW_CUDA(cudaEventRecord(ev[0], h->st_h2d));
        GW_CUDA(cudaMemcpyAsync(gtmp, X, (size_t)b * rbi, cudaMemcpyHostToDevice, h->st_h2d));
        GW_CUDA(cudaEventRecord(ev[1], h->st_h2d));
        GW_CUDA(cudaStreamWaitEvent(s, ev[1], 0));
        src = gtmp;
      }
      void* Bo = out_dev ? B : otmp;
      void* Wo = !wald ? nullptr : out_dev ? wald : (char*)otmp + (size_t)b * t * p * ob;
      GW_CUDA(cudaEventRecord(ev[2], s));
      scan_block(h, src, fmt, b, Bo, Wo, out_f64, s);
      GW_CUDA(cudaEventRecord(ev[3], s));
      if (!out_dev) {
        GW_CUDA(cudaStreamWaitEvent(h->st_d2h, ev[3], 0));
        GW_CUDA(cudaEventRecord(ev[4], h->st_d2h));
        GW_CUDA(cudaMemcpyAsync(B, otmp, (size_t)b * t * p * ob, cudaMemcpyDeviceToHost,
                                h->st_d2h));
        if (wald)
          GW_CUDA(cudaMemcpyAsync(wald, Wo, (size_t)b * t * ob, cudaMemcpyDeviceToHost,
                                  h->st_d2h));
        GW_CUDA(cudaEventRecord(ev[5], h->st_d2h));
      }
      GW_CUDA(cudaDeviceSynchronize());
      if (rep == 0) continue;
      float tin = 0.f, tc = 0.f, tout = 0.f;
      if (!xr_dev) GW_CUDA(cudaEventElapsedTime(&tin, ev[0], ev[1]));
      GW_CUDA(cudaEventElapsedTime(&tc, ev[2], ev[3]));
      if (!out_dev) GW_CUDA(cudaEventElapsedTime(&tout, ev[4], ev[5]));
      const double nb = (double)((m + b - 1) / b);
      double slow = tc / lanes;
      slow = tin > slow ? tin : slow;
      slow = tout > slow ? tout : slow;
      const double T = tin + tc + tout + (nb - 1.0) * slow;
      if (h->ntune < 8) {
        h->tune_b[h->ntune] = b;
        h->tune_ms[h->ntune][0] = tin;
        h->tune_ms[h->ntune][1] = tc;
        h->tune_ms[h->ntune][2] = tout;
        ++h->ntune;
      }
      if (T < best) {
        best = T;
        best_b = b;
      }
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  dfree(h, gtmp);
  dfree(h, otmp);
  h->block_snps = (int)(best_b > 64 ? best_b : 64);
  h->block_tuned = true;
}

gwas_status scan_impl(gwas_handle h, const void* X, int fmt, int64_t m, int xr_dev, void* B,
                      void* wald, int out_dev, void* stream, bool out_f64) {
  GW_REQUIRE(h != nullptr, GWAS_ERR_ARG, "null handle");
  GW_REQUIRE(m >= 0, GWAS_ERR_ARG, "m < 0");
  if (m == 0) return GWAS_OK;
  GW_REQUIRE(X != nullptr && B != nullptr, GWAS_ERR_ARG, "null genotypes or B");
  GW_REQUIRE(!(out_f64 && h->prec == GWAS_PREC_SPLIT_BF16), GWAS_ERR_UNSUPPORTED,
             "gwas_scan_f64 needs the FP64 or FP32 precision mode");
  DeviceGuard dg(h->dev);
  cudaStream_t s = (cudaStream_t)stream;
  const int t = h->t, p = h->pw;
  const size_t ob = out_f64 ? 8 : 4;
  const size_t rbi = row_bytes_of(h, fmt);
  if (h->validate)  // each call reports only its own genotypes
    GW_CUDA(cudaMemsetAsync(h->flags + FLAG_GENOTYPE, 0, sizeof(int), s));
  if (xr_dev && out_dev) {
    ensure_xt(h, m < h->block_snps ? m : h->block_snps);
    scan_block(h, X, fmt, m, B, wald, out_f64, s);
    if (h->validate) {
      check_timeout(h, s);
      GW_REQUIRE(!h->h_flags[FLAG_GENOTYPE], GWAS_ERR_GENOTYPE, "genotype outside {0,1,2}");
    }
    return GWAS_OK;
  }
  // Streamed: H2D of genotype blocks through a ring of device buffers (copy stream), compute,
  // D2H of each block's outputs (second copy stream).  A block whose scan uses no scratch of
  // the handle (CHOL on the tensor cores from packed rows, or on CUDA cores from int8 rows)
  // alternates between two compute streams: the next block's kernel then fills the SMs that
  // the last wave of the current one leaves idle.  Other scans run their blocks in order on s.
  const bool two = h->algo == GWAS_ALGO_CHOL &&
                   (h->prec == GWAS_PREC_SPLIT_BF16 ? fmt == FMT_PACKED2 : fmt == FMT_INT8);
  const int nring = two ? gwas_handle_s::NRING : 2;
  if (h->block_auto && !h->block_tuned)
    tune_block(h, X, fmt, m, xr_dev, B, wald, out_dev, out_f64, s, two ? 2 : 1);
  const int64_t blk = h->block_snps;
  const size_t gbytes = (size_t)blk * rbi, obytes = (size_t)blk * t * (p + 1) * 8;
  if (h->ring_bytes < gbytes || h->oring_bytes < obytes || h->nring < nring) {
    GW_CUDA(cudaStreamSynchronize(s));
    GW_CUDA(cudaStreamSynchronize(h->st_lane));
    GW_CUDA(cudaStreamSynchronize(h->st_h2d));
    GW_CUDA(cudaStreamSynchronize(h->st_d2h));
    for (int i = 0; i < gwas_handle_s::NRING; ++i) {
      dfree(h, h->ring[i]);
      dfree(h, h->oring[i]);
      h->ring[i] = nullptr;
      h->oring[i] = nullptr;
    }
    h->nring = 0;
    const size_t gb = gbytes > h->ring_bytes ? gbytes : h->ring_bytes;
    const size_t obb = obytes > h->oring_bytes ? obytes : h->oring_bytes;
    for (int i = 0; i < nring; ++i) {
      h->ring[i] = (uint8_t*)dalloc(h, gb);
      h->oring[i] = dalloc(h, obb);
    }
    h->nring = nring;
    h->ring_bytes = gb;
    h->oring_bytes = obb;
  }
  ensure_xt(h, blk);
  if (two) {  // the second lane starts after the caller's prior work on s
    GW_CUDA(cudaEventRecord(h->ev_begin, s));
    GW_CUDA(cudaStreamWaitEvent(h->st_lane, h->ev_begin, 0));
  }
  const int nblocks = ceil_div(m, blk);
  for (int b = 0; b < nblocks; ++b) {
    const int buf = b % nring;
    cudaStream_t cs = two && (b & 1) ? h->st_lane : s;
    const int64_t off = (int64_t)b * blk;
    const int64_t mm = m - off < blk ? m - off : blk;
    const uint8_t* src = (const uint8_t*)X + off * rbi;
    if (!xr_dev) {
      GW_CUDA(cudaStreamWaitEvent(h->st_h2d, h->ev_computed[buf], 0));
      GW_CUDA(cudaMemcpyAsync(h->ring[buf], src, (size_t)mm * rbi, cudaMemcpyHostToDevice,
                              h->st_h2d));
      GW_CUDA(cudaEventRecord(h->ev_loaded[buf], h->st_h2d));
      GW_CUDA(cudaStreamWaitEvent(cs, h->ev_loaded[buf], 0));
      src = h->ring[buf];
    }
    void* Bo;
    void* Wo;
    if (out_dev) {
      Bo = (char*)B + (size_t)off * t * p * ob;
      Wo = wald ? (char*)wald + (size_t)off * t * ob : nullptr;
    } else {
      GW_CUDA(cudaStreamWaitEvent(cs, h->ev_drained[buf], 0));
      Bo = h->oring[buf];
      Wo = wald ? (char*)h->oring[buf] + (size_t)blk * t * p * ob : nullptr;
    }
    if (!xr_dev && !out_dev && mm == blk) {
      // a full block between ring slots: its device work is one captured graph
      GW_CUDA(cudaGraphLaunch(block_graph(h, buf, fmt, blk, out_f64, wald != nullptr), cs));
      ++h->graph_launches;
    } else {
      scan_block(h, src, fmt, mm, Bo, Wo, out_f64, cs);
    }
    GW_CUDA(cudaEventRecord(h->ev_computed[buf], cs));
    if (!out_dev) {
      GW_CUDA(cudaStreamWaitEvent(h->st_d2h, h->ev_computed[buf], 0));
      GW_CUDA(cudaMemcpyAsync((char*)B + (size_t)off * t * p * ob, Bo, (size_t)mm * t * p * ob,
                              cudaMemcpyDeviceToHost, h->st_d2h));
      if (wald)
        GW_CUDA(cudaMemcpyAsync((char*)wald + (size_t)off * t * ob, Wo, (size_t)mm * t * ob,
                                cudaMemcpyDeviceToHost, h->st_d2h));
      GW_CUDA(cudaEventRecord(h->ev_drained[buf], h->st_d2h));
    }
  }
  if (two) {  // work after the call on s sees both lanes' results
    GW_CUDA(cudaEventRecord(h->ev_lane_done, h->st_lane));
    GW_CUDA(cudaStreamWaitEvent(s, h->ev_lane_done, 0));
  }
  GW_CUDA(cudaStreamSynchronize(s));
  GW_CUDA(cudaStreamSynchronize(h->st_h2d));
  GW_CUDA(cudaStreamSynchronize(h->st_d2h));
  check_timeout(h, s);
  if (h->validate)
    GW_REQUIRE(!h->h_flags[FLAG_GENOTYPE], GWAS_ERR_GENOTYPE, "genotype outside {0,1,2}");
  return GWAS_OK;
}

}  // namespace

namespace gw {
// Internals the batch API (batch.cu) builds on.
TcState* handle_tc(gwas_handle h) { return h ? h->tc : nullptr; }
int handle_device(gwas_handle h) { return h->dev; }
int* handle_flags(gwas_handle h) { return h->flags; }
int handle_n(gwas_handle h) { return h->n; }
int handle_t(gwas_handle h) { return h->t; }
int handle_p(gwas_handle h) { return h->p; }
}  // namespace gw

GW_API void gwas_default_options(gwas_options* opt) {
  if (!opt) return;
  opt->algo = GWAS_ALGO_AUTO;
  opt->precision = GWAS_PREC_SPLIT_BF16;
  opt->block_snps = 0;
  opt->validate_genotypes = 0;
  opt->device = 0;
  opt->out_mode = GWAS_OUT_FULL;
  opt->genetic_model = GWAS_MODEL_ADDITIVE;
}

namespace gw {
GeneticModel genetic_model(int model) {
  GeneticModel g;
  switch (model) {
    case GWAS_MODEL_ADDITIVE: break;
    case GWAS_MODEL_DOMINANT: g.code[0][2] = 1; break;
    case GWAS_MODEL_RECESSIVE: g.code[0][1] = 0; g.code[0][2] = 1; break;
    case GWAS_MODEL_ADD_DOM:
      // working basis: the genotype indicators [x == 1, x == 2], which span the same columns
      // as (x, [x == 1]) but stay well conditioned when one homozygote class is rare (x and
      // [x == 1] then differ in a few individuals only); x = I1 + 2 I2 and [x == 1] = I1 give
      // b_additive = b_I2 / 2, b_dominance = b_I1 - b_I2 / 2
      g.pr = 2;
      g.code[0][1] = 1; g.code[0][2] = 0;
      g.code[1][1] = 0; g.code[1][2] = 1;
      g.tm[0][0] = 0.f; g.tm[0][1] = 0.5f;
      g.tm[1][0] = 1.f; g.tm[1][1] = -0.5f;
      break;
    default: GW_REQUIRE(false, GWAS_ERR_ARG, "bad genetic_model %d", model);
  }
  return g;
}
}  // namespace gw

GW_API gwas_status gwas_setup(const double* Phi, int n, const double* XL, int q, const double* Y,
                              int t, const double* h2, const double* s2, const gwas_options* opt,
                              gwas_handle* out) {
  if (out) *out = nullptr;
  gwas_handle h = nullptr;
  try {
    GW_REQUIRE(out != nullptr, GWAS_ERR_ARG, "out is NULL");
    GW_REQUIRE(Phi && XL && Y && h2 && s2, GWAS_ERR_ARG, "null input pointer");
    GW_REQUIRE(n >= 1 && n <= 16384, GWAS_ERR_ARG, "n=%d outside [1,16384]", n);
    GW_REQUIRE(q >= 1 && q <= 7, GWAS_ERR_ARG, "q=%d outside [1,7]", q);
    GW_REQUIRE(t >= 1, GWAS_ERR_ARG, "t=%d < 1", t);
    for (int j = 0; j < t; ++j) {
      GW_REQUIRE(h2[j] >= 0.0 && h2[j] < 1.0, GWAS_ERR_ARG, "h2[%d]=%g outside [0,1)", j, h2[j]);
      GW_REQUIRE(s2[j] > 0.0 && isfinite(s2[j]), GWAS_ERR_ARG, "s2[%d]=%g not > 0", j, s2[j]);
    }
    gwas_options o;
    gwas_default_options(&o);
    if (opt) o = *opt;
    GW_REQUIRE(o.algo >= 0 && o.algo <= 2, GWAS_ERR_ARG, "bad algo %d", o.algo);
    GW_REQUIRE(o.precision >= 0 && o.precision <= 3, GWAS_ERR_ARG, "bad precision %d", o.precision);
    GW_REQUIRE(o.block_snps >= 0, GWAS_ERR_ARG, "block_snps < 0");
    GW_REQUIRE(o.out_mode == GWAS_OUT_FULL || o.out_mode == GWAS_OUT_SNP ||
                   o.out_mode == GWAS_OUT_VAR,
               GWAS_ERR_ARG, "bad out_mode %d", o.out_mode);
    const GeneticModel gm = genetic_model(o.genetic_model);
    h = new gwas_handle_s();
    h->model = o.genetic_model;
    h->gm = gm;
    h->dev = o.device;
    h->n = n;
    h->q = q;
    h->p = q + gm.pr;
    h->t = t;
    h->algo = o.algo == GWAS_ALGO_AUTO ? (t == 1 ? GWAS_ALGO_CHOL : GWAS_ALGO_EIG) : o.algo;
    h->prec_opt = o.precision;
    h->fp8 = o.precision == GWAS_PREC_SPLIT_FP8;
    h->prec = h->fp8 ? GWAS_PREC_SPLIT_BF16 : o.precision;
    h->validate = o.validate_genotypes ? 1 : 0;
    h->out_snp = o.out_mode == GWAS_OUT_SNP ? 1 : 0;
    h->out_var = o.out_mode == GWAS_OUT_VAR ? 1 : 0;
    h->pw = h->out_snp ? 2 * gm.pr : h->out_var ? h->p + h->p * (h->p + 1) / 2 : h->p;
    h->ldp = (int)round_up(n, 64);
    if (h->algo == GWAS_ALGO_CHOL)
      GW_REQUIRE((double)t * n * n * 8.0 <= 64e9, GWAS_ERR_UNSUPPORTED,
                 "CHOL keeps one n x n factor per trait: t=%d, n=%d is too large (use EIG)", t, n);
    if (h->prec == GWAS_PREC_SPLIT_BF16) {
      tc_check_supported(h->algo, n, q, t);
      // Two working columns on the tensor cores are centred by the intercept: without it their
      // cross product g0^T M^-1 g1 is a large cancellation (both columns keep their means) that
      // the split-BF16 operands cannot resolve to the 1e-4 bound.
      bool ones = true;
      for (int i = 0; i < n; ++i) ones = ones && XL[i] == 1.0;
      GW_REQUIRE(gm.pr == 1 || ones, GWAS_ERR_UNSUPPORTED,
                 "a two-column genetic model on the tensor cores needs the intercept as column 0 "
                 "of X_L (use FP64 or FP32 without it)");
    }
    int ndev = 0;
    GW_CUDA(cudaGetDeviceCount(&ndev));
    GW_REQUIRE(h->dev >= 0 && h->dev < ndev, GWAS_ERR_ARG, "device %d not present", h->dev);
    DeviceGuard dg(h->dev);
    // default block: CHOL 64 Ki SNPs; EIG bounded so a block's FP64 outputs (B and wald)
    // stay <= 2 GB
    int64_t blk = o.block_snps > 0 ? o.block_snps : (h->algo == GWAS_ALGO_CHOL ? 65536 : 32768);
    const int64_t out_cap = (int64_t)(2e9 / ((double)t * (h->pw + 1) * 8));
    if (blk > out_cap) blk = out_cap;
    if (blk < 64) blk = 64;
    h->block_snps = (int)blk;
    h->block_auto = o.block_snps == 0;
    GW_CUDA(cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking));
    GW_CUDA(cudaStreamCreateWithFlags(&h->st_cap, cudaStreamNonBlocking));
    GW_CUDA(cudaStreamCreateWithFlags(&h->st_lane, cudaStreamNonBlocking));
    GW_CUDA(cudaStreamCreateWithFlags(&h->st_h2d, cudaStreamNonBlocking));
    GW_CUDA(cudaStreamCreateWithFlags(&h->st_d2h, cudaStreamNonBlocking));
    for (int i = 0; i < gwas_handle_s::NRING; ++i) {
      GW_CUDA(cudaEventCreateWithFlags(&h->ev_loaded[i], cudaEventDisableTiming));
      GW_CUDA(cudaEventCreateWithFlags(&h->ev_computed[i], cudaEventDisableTiming));
      GW_CUDA(cudaEventCreateWithFlags(&h->ev_drained[i], cudaEventDisableTiming));
    }
    GW_CUDA(cudaEventCreateWithFlags(&h->ev_begin, cudaEventDisableTiming));
    GW_CUDA(cudaEventCreateWithFlags(&h->ev_lane_done, cudaEventDisableTiming));
    h->flags = (int*)dalloc(h, sizeof(int) * FLAG_COUNT);
    GW_CUDA(cudaMallocHost(&h->h_flags, sizeof(int) * FLAG_COUNT));
    setup_impl(h, Phi, XL, Y, h2, s2);
    *out = h;
    set_error("%s", "");
    return GWAS_OK;
  } catch (const Fail& f) {
    destroy_impl(h);
    return f.st;
  } catch (...) {
    set_error("unexpected C++ exception in gwas_setup");
    destroy_impl(h);
    return GWAS_ERR_CUDA;
  }
}

GW_API gwas_status gwas_scan(gwas_handle h, const int8_t* XR, int64_t m, int xr_on_device,
                             float* B, float* wald, int out_on_device, void* stream) {
  try {
    return scan_impl(h, XR, FMT_INT8, m, xr_on_device, B, wald, out_on_device, stream, false);
  } catch (const Fail& f) {
    return f.st;
  } catch (...) {
    set_error("unexpected C++ exception in gwas_scan");
    return GWAS_ERR_CUDA;
  }
}

GW_API gwas_status gwas_scan_f64(gwas_handle h, const int8_t* XR, int64_t m, int xr_on_device,
                                 double* B, double* wald, int out_on_device, void* stream) {
  try {
    return scan_impl(h, XR, FMT_INT8, m, xr_on_device, B, wald, out_on_device, stream, true);
  } catch (const Fail& f) {
    return f.st;
  } catch (...) {
    set_error("unexpected C++ exception in gwas_scan_f64");
    return GWAS_ERR_CUDA;
  }
}

GW_API gwas_status gwas_scan_packed(gwas_handle h, const uint8_t* G, int64_t m, int g_on_device,
                                    float* B, float* wald, int out_on_device, void* stream) {
  try {
    return scan_impl(h, G, FMT_PACKED2, m, g_on_device, B, wald, out_on_device, stream, false);
  } catch (const Fail& f) {
    return f.st;
  } catch (...) {
    set_error("unexpected C++ exception in gwas_scan_packed");
    return GWAS_ERR_CUDA;
  }
}

GW_API int gwas_packed_row_bytes(int n) { return n >= 1 ? packed_row_bytes(n) : 0; }

GW_API gwas_status gwas_shard(int64_t m_total, int rank, int world, int64_t align, int64_t* start,
                              int64_t* count) {
  try {
    GW_REQUIRE(start != nullptr && count != nullptr, GWAS_ERR_ARG, "null start or count");
    GW_REQUIRE(m_total >= 0 && world >= 1 && rank >= 0 && rank < world && align >= 1, GWAS_ERR_ARG,
               "need m_total >= 0, world >= 1, 0 <= rank < world, align >= 1");
    const int64_t units = m_total / align + (m_total % align != 0);
    const int64_t u0 = units / world * rank + std::min<int64_t>(rank, units % world);
    const int64_t u1 = u0 + units / world + (rank < units % world);
    *start = std::min(u0 * align, m_total);
    *count = std::min(u1 * align, m_total) - *start;
    return GWAS_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

GW_API gwas_status gwas_wald_pvalues_dof(const float* wald, int64_t count, int dof, float* pval,
                                         int on_device, void* stream) {
  try {
    GW_REQUIRE(count >= 0, GWAS_ERR_ARG, "count < 0");
    GW_REQUIRE(dof == 1 || dof == 2, GWAS_ERR_ARG, "dof=%d: 1 or 2 degrees of freedom", dof);
    if (count == 0) return GWAS_OK;
    GW_REQUIRE(wald != nullptr && pval != nullptr, GWAS_ERR_ARG, "null wald or pval");
    if (on_device) {
      wald_pvalues((cudaStream_t)stream, wald, count, dof, pval);
      return GWAS_OK;
    }
    for (int64_t e = 0; e < count; ++e) {
      const double x = wald[e];
      pval[e] = x >= 0.0 ? (float)(dof == 2 ? exp(-0.5 * x) : erfc(sqrt(0.5 * x)))
                         : (x == x ? 1.f : (float)x);
    }
    return GWAS_OK;
  } catch (const Fail& f) {
    return f.st;
  } catch (...) {
    set_error("unexpected C++ exception in gwas_wald_pvalues");
    return GWAS_ERR_CUDA;
  }
}

GW_API gwas_status gwas_wald_pvalues(const float* wald, int64_t count, float* pval, int on_device,
                                     void* stream) {
  return gwas_wald_pvalues_dof(wald, count, 1, pval, on_device, stream);
}

GW_API gwas_status gwas_estimate(const double* Phi, int n, const double* XL, int q,
                                 const double* Y, int t, int method, int device, double* h2,
                                 double* s2, double* crit, double* ms) {
  std::vector<void*> mem;
  auto alloc = [&](size_t bytes) -> double* {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
      cudaGetLastError();
      set_error("cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
      throw Fail{GWAS_ERR_OOM};
    }
    mem.push_back(p);
    return (double*)p;
  };
  cudaStream_t s = nullptr;
  cudaEvent_t ev[3] = {};
  int prev = -1;
  gwas_status st = GWAS_OK;
  try {
    GW_REQUIRE(Phi && XL && Y && h2 && s2, GWAS_ERR_ARG, "null input or output pointer");
    GW_REQUIRE(n >= 2 && n <= 16384, GWAS_ERR_ARG, "n=%d outside [2,16384]", n);
    GW_REQUIRE(q >= 1 && q <= 7 && q < n, GWAS_ERR_ARG, "q=%d outside [1,min(7,n-1)]", q);
    GW_REQUIRE(t >= 1, GWAS_ERR_ARG, "t=%d < 1", t);
    GW_REQUIRE(method == GWAS_EST_ML || method == GWAS_EST_REML, GWAS_ERR_ARG, "bad method %d",
               method);
    int ndev = 0;
    GW_CUDA(cudaGetDeviceCount(&ndev));
    GW_REQUIRE(device >= 0 && device < ndev, GWAS_ERR_ARG, "device %d not present", device);
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    GW_CUDA(cudaSetDevice(device));
    GW_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    for (auto& e : ev) GW_CUDA(cudaEventCreate(&e));
    const size_t nn = (size_t)n * n;
    double* dPhi = alloc(nn * 8);
    double* dXL = alloc((size_t)n * q * 8);
    double* dY = alloc((size_t)n * t * 8);
    double* Zt = alloc(nn * 8);
    double* U = alloc(nn * 8);
    double* w = alloc((size_t)n * 8);
    double* XLt = alloc((size_t)q * n * 8);
    double* Yt = alloc((size_t)t * n * 8);
    double* out = alloc((size_t)3 * t * 8);
    double* tables = alloc(estimate_table_doubles(n) * 8);
    int* flags = (int*)alloc(sizeof(int) * FLAG_COUNT);
    GW_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * FLAG_COUNT, s));
    GW_CUDA(cudaMemcpyAsync(dPhi, Phi, nn * 8, cudaMemcpyHostToDevice, s));
    GW_CUDA(cudaMemcpyAsync(dXL, XL, (size_t)n * q * 8, cudaMemcpyHostToDevice, s));
    GW_CUDA(cudaMemcpyAsync(dY, Y, (size_t)n * t * 8, cudaMemcpyHostToDevice, s));
    GW_CUDA(cudaEventRecord(ev[0], s));
    // Phi = Z W Z^T; X~ = Z^T X_L (rows of XLt), y~_j = Z^T y_j (rows of Yt)
    const int sweeps = eigh_f64(s, n, dPhi, Zt, w, U, flags);
    GW_REQUIRE(sweeps >= 0, GWAS_ERR_NOT_CONVERGED, "the eigensolver did not converge");
    gemm_f64(s, q, n, n, 1.0, dXL, n, 1, Zt, 1, n, 0.0, XLt, n, 1);
    gemm_f64(s, t, n, n, 1.0, dY, n, 1, Zt, 1, n, 0.0, Yt, n, 1);
    GW_CUDA(cudaEventRecord(ev[1], s));
    // H(h) = h Phi + (1 - h) I must stay positive definite on the whole search interval
    std::vector<double> hw(n);
    GW_CUDA(cudaMemcpyAsync(hw.data(), w, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    GW_CUDA(cudaStreamSynchronize(s));
    for (int r = 0; r < n; ++r)
      GW_REQUIRE(0.999 * hw[r] + 0.001 > 0.0, GWAS_ERR_NOT_SPD,
                 "h Phi + (1 - h) I is not positive definite for h up to 0.999 (eigenvalue %g)",
                 hw[r]);
    estimate_traits(s, n, q, t, method, w, XLt, Yt, tables, out, out + t, out + 2 * t, flags);
    GW_CUDA(cudaEventRecord(ev[2], s));
    std::vector<double> hout((size_t)3 * t);
    int hflags[FLAG_COUNT];
    GW_CUDA(cudaMemcpyAsync(hout.data(), out, (size_t)3 * t * 8, cudaMemcpyDeviceToHost, s));
    GW_CUDA(cudaMemcpyAsync(hflags, flags, sizeof(hflags), cudaMemcpyDeviceToHost, s));
    GW_CUDA(cudaStreamSynchronize(s));
    GW_REQUIRE(!hflags[FLAG_STL_SINGULAR], GWAS_ERR_SINGULAR,
               "X_L^T H^-1 X_L is singular (collinear covariates)");
    for (int j = 0; j < t; ++j) {
      h2[j] = hout[j];
      s2[j] = hout[t + j];
      if (crit) crit[j] = hout[2 * t + j];
    }
    if (ms) {
      float a = 0.f, b = 0.f;
      GW_CUDA(cudaEventElapsedTime(&a, ev[0], ev[1]));
      GW_CUDA(cudaEventElapsedTime(&b, ev[1], ev[2]));
      ms[0] = a;
      ms[1] = b;
    }
  } catch (const Fail& f) {
    st = f.st;
  } catch (...) {
    set_error("unexpected C++ exception in gwas_estimate");
    st = GWAS_ERR_CUDA;
  }
  if (s) cudaStreamSynchronize(s);
  for (void* p : mem) cudaFree(p);
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (s) cudaStreamDestroy(s);
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}

GW_API gwas_status gwas_pack_genotypes(const int8_t* X, int64_t m, int n, uint8_t* G,
                                       int on_device, void* stream) {
  try {
    GW_REQUIRE(m >= 0 && n >= 1, GWAS_ERR_ARG, "bad sizes m=%lld n=%d", (long long)m, n);
    if (m == 0) return GWAS_OK;
    GW_REQUIRE(X != nullptr && G != nullptr, GWAS_ERR_ARG, "null X or G");
    if (on_device) {
      pack_genotypes((cudaStream_t)stream, X, m, n, G, nullptr, false);
      return GWAS_OK;
    }
    const int rb = packed_row_bytes(n);
    bool bad = false;
    for (int64_t i = 0; i < m; ++i) {
      const uint8_t* x = (const uint8_t*)X + i * n;
      uint8_t* g = G + i * rb;
      for (int b = 0; b < rb; ++b) {
        unsigned v = 0;
        for (int u = 0; u < 4; ++u) {
          const int k = 4 * b + u;
          if (k < n) {
            const unsigned c = x[k];
            bad |= c > 2;
            v |= (c > 2 ? 3u : c) << (2 * u);
          }
        }
        g[b] = (uint8_t)v;
      }
    }
    GW_REQUIRE(!bad, GWAS_ERR_GENOTYPE, "genotype outside {0,1,2} (packed as the invalid code 3)");
    return GWAS_OK;
  } catch (const Fail& f) {
    return f.st;
  } catch (...) {
    set_error("unexpected C++ exception in gwas_pack_genotypes");
    return GWAS_ERR_CUDA;
  }
}

GW_API gwas_status gwas_setup_timing(gwas_handle h, double* ms_setup) {
  if (!h || !ms_setup) {
    set_error("null argument");
    return GWAS_ERR_ARG;
  }
  *ms_setup = h->setup_ms;
  return GWAS_OK;
}

GW_API gwas_status gwas_info(gwas_handle h, int* n, int* q, int* t, int* algo, int* precision) {
  if (!h) {
    set_error("null handle");
    return GWAS_ERR_ARG;
  }
  if (n) *n = h->n;
  if (q) *q = h->q;
  if (t) *t = h->t;
  if (algo) *algo = h->algo;
  if (precision) *precision = h->prec_opt;
  return GWAS_OK;
}

GW_API int gwas_genetic_columns(gwas_handle h) { return h ? h->gm.pr : -1; }

GW_API gwas_status gwas_stream_info(gwas_handle h, int* block_snps, int* tuned,
                                    int64_t* graph_launches, int* ncand, int64_t* cand_snps,
                                    double* cand_ms) {
  if (!h) {
    set_error("null handle");
    return GWAS_ERR_ARG;
  }
  if (block_snps) *block_snps = h->block_snps;
  if (tuned) *tuned = h->block_tuned ? 1 : 0;
  if (graph_launches) *graph_launches = h->graph_launches;
  if (ncand) *ncand = h->ntune;
  for (int i = 0; i < h->ntune; ++i) {
    if (cand_snps) cand_snps[i] = h->tune_b[i];
    if (cand_ms)
      for (int k = 0; k < 3; ++k) cand_ms[3 * i + k] = h->tune_ms[i][k];
  }
  return GWAS_OK;
}

GW_API int64_t gwas_eig_chunk(gwas_handle h) {
  if (!h) return -1;
  return h->tc ? tc_eig_chunk(h->tc) : 0;
}

GW_API int gwas_chol_routed_traits(gwas_handle h) {
  return h ? (h->tc ? tc_chol_routed_traits(h->tc) : 0) : -1;
}

GW_API int gwas_fp8_traits(gwas_handle h) { return h ? (h->tc ? tc_fp8_traits(h->tc) : 0) : -1; }

GW_API int gwas_split_pieces(gwas_handle h) {
  if (!h) return -1;
  return h->tc ? tc_split_pieces(h->tc) : 0;
}

GW_API int64_t gwas_singular_count(gwas_handle h) {
  if (!h) return -1;
  try {
    DeviceGuard dg(h->dev);
    GW_CUDA(cudaDeviceSynchronize());
    read_flags(h, h->st);
    return h->h_flags[FLAG_SINGULAR];
  } catch (const Fail&) {
    return -1;
  }
}

GW_API gwas_status gwas_sync(gwas_handle h) {
  try {
    GW_REQUIRE(h != nullptr, GWAS_ERR_ARG, "null handle");
    DeviceGuard dg(h->dev);
    GW_CUDA(cudaDeviceSynchronize());
    check_timeout(h, h->st);
    return GWAS_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

GW_API gwas_status gwas_selftest_timeout(int device, int limit_ms) {
  try {
    GW_REQUIRE(limit_ms >= 1 && limit_ms <= 10000, GWAS_ERR_ARG, "limit_ms=%d outside [1,10000]",
               limit_ms);
    int ndev = 0;
    GW_CUDA(cudaGetDeviceCount(&ndev));
    GW_REQUIRE(device >= 0 && device < ndev, GWAS_ERR_ARG, "device %d not present", device);
    DeviceGuard dg(device);
    return selftest_wait_timeout(limit_ms);
  } catch (const Fail& f) {
    return f.st;
  }
}

GW_API gwas_status gwas_stage_timing(gwas_handle h, int enable) {
  try {
    GW_REQUIRE(h != nullptr, GWAS_ERR_ARG, "null handle");
    DeviceGuard dg(h->dev);
    GW_CUDA(cudaDeviceSynchronize());  // no recorded event is still pending
    h->timer.on = enable != 0;
    h->timer.stage.clear();
    h->timer.used = 0;
    return GWAS_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

GW_API gwas_status gwas_stage_times(gwas_handle h, double* ms, int64_t* launches) {
  try {
    GW_REQUIRE(h != nullptr && ms != nullptr, GWAS_ERR_ARG, "null handle or ms");
    DeviceGuard dg(h->dev);
    for (int i = 0; i < GWAS_NSTAGES; ++i) {
      ms[i] = 0.0;
      if (launches) launches[i] = 0;
    }
    StageTimer& tm = h->timer;
    for (size_t k = 0; k < tm.stage.size(); ++k) {
      cudaEvent_t e0 = tm.pool[2 * k], e1 = tm.pool[2 * k + 1];
      GW_CUDA(cudaEventSynchronize(e1));
      float t = 0.f;
      GW_CUDA(cudaEventElapsedTime(&t, e0, e1));
      const int st = tm.stage[k];
      if (st >= 0 && st < GWAS_NSTAGES) {
        ms[st] += t;
        if (launches) launches[st] += 1;
      }
    }
    tm.stage.clear();
    tm.used = 0;
    return GWAS_OK;
  } catch (const Fail& f) {
    return f.st;
  }
}

GW_API const char* gwas_last_error(void) { return gw::g_err.c_str(); }

GW_API void gwas_destroy(gwas_handle h) { destroy_impl(h); }

// ------------------------------------------------------------------------------------------
// gwas_scan_static: the CUDA-core EIG scan of a handle with its per-block scratch (the rotated
// genotypes Z^T X_R) in a fixed device array of this file instead of memory the call allocates.
// ------------------------------------------------------------------------------------------
namespace {

constexpr size_t STATIC_SCRATCH_BYTES = (size_t)16 << 20;  // 16 MiB on every device
static __device__ __align__(256) unsigned char g_scan_scratch[STATIC_SCRATCH_BYTES];

std::mutex g_scratch_mu;
constexpr int MAX_DEVICES = 64;
void* g_scratch_addr[MAX_DEVICES] = {};

// Device address of g_scan_scratch on the current device, looked up once per device.  In host
// code g_scan_scratch names a host-side stand-in, never the device array itself.
void* static_scratch(int dev) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  GW_REQUIRE(dev >= 0 && dev < MAX_DEVICES, GWAS_ERR_ARG, "device %d out of range", dev);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    GW_CUDA(cudaGetSymbolAddress(&ptr, g_scan_scratch));
    GW_REQUIRE(ptr != nullptr, GWAS_ERR_CUDA, "no device address for the static scratch");
    g_scratch_addr[dev] = ptr;
  }
  return g_scratch_addr[dev];
}

}  // namespace

GW_API gwas_status gwas_scan_static(gwas_handle h, const int8_t* XR, int64_t m, float* B,
                                    float* wald, void* stream) {
  try {
    GW_REQUIRE(h != nullptr, GWAS_ERR_ARG, "null handle");
    GW_REQUIRE(m >= 0, GWAS_ERR_ARG, "m < 0");
    if (m == 0) return GWAS_OK;
    GW_REQUIRE(XR != nullptr && B != nullptr, GWAS_ERR_ARG, "null XR or B");
    GW_REQUIRE(h->algo == GWAS_ALGO_EIG &&
                   (h->prec == GWAS_PREC_FP64 || h->prec == GWAS_PREC_FP32),
               GWAS_ERR_UNSUPPORTED,
               "gwas_scan_static needs an EIG handle with FP64 or FP32 precision");
    const size_t es = h->prec == GWAS_PREC_FP64 ? 8 : 4;
    const size_t per_snp = (size_t)h->gm.pr * h->ldp * es;
    GW_REQUIRE((size_t)m * per_snp <= STATIC_SCRATCH_BYTES, GWAS_ERR_ARG,
               "m=%lld SNPs need %zu bytes of scratch; the static scratch holds %zu bytes "
               "(at most %zu SNPs per call for this handle)",
               (long long)m, (size_t)m * per_snp, STATIC_SCRATCH_BYTES,
               STATIC_SCRATCH_BYTES / per_snp);
    DeviceGuard dg(h->dev);
    void* xt = static_scratch(h->dev);
    cudaStream_t s = (cudaStream_t)stream;
    const int n = h->n, q = h->q, t = h->t;
    if (h->validate) {  // as gwas_scan: each call reports only its own genotypes
      GW_CUDA(cudaMemsetAsync(h->flags + FLAG_GENOTYPE, 0, sizeof(int), s));
      validate_genotypes(s, XR, m * n, h->flags);
    }
    if (h->prec == GWAS_PREC_FP64) {
      EigScanArgs<double> a{n, q, t, h->Zt, h->planes, h->ldp, h->P, h->b0, XR, m, 0,
                            B, wald, false, 1e-12, (double*)xt, h->flags};
      a.out_snp = h->out_snp;
      a.out_var = h->out_var;
      a.gm = h->gm;
      eig_scan_simt<double>(s, a);
    } else {
      EigScanArgs<float> a{n, q, t, h->Zt32, h->planes32, h->ldp, h->P32, h->b032, XR, m, 0,
                           B, wald, false, 1e-5f, (float*)xt, h->flags};
      a.out_snp = h->out_snp;
      a.out_var = h->out_var;
      a.gm = h->gm;
      eig_scan_simt<float>(s, a);
    }
    if (h->validate) {  // synchronous then: the flag is read back into pinned host memory
      read_flags(h, s);
      GW_REQUIRE(!h->h_flags[FLAG_GENOTYPE], GWAS_ERR_GENOTYPE, "genotype outside {0,1,2}");
    }
    return GWAS_OK;
  } catch (const Fail& f) {
    return f.st;
  } catch (...) {
    set_error("unexpected C++ exception in gwas_scan_static");
    return GWAS_ERR_CUDA;
  }
}
