// Host side of the split-BF16 tensor-core path: operand splitting, tensor maps, dispatch.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <limits>
#include <mutex>
#include <vector>

#include "tc.cuh"
#include "tc_kernels.cuh"

namespace gw {

namespace {

constexpr int QMAX = 7;

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static std::mutex mu;  // looked up once, possibly from several host threads
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    GW_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000,
                                             cudaEnableDefault, &q));
    GW_REQUIRE(q == cudaDriverEntryPointSuccess && ptr, GWAS_ERR_CUDA,
               "cuTensorMapEncodeTiled not available from the driver");
    fn = (PFN_cuTensorMapEncodeTiled_v12000)ptr;
  }
  return fn;
}

}  // namespace

// 2-D BF16 row-major matrix [rows][cols] (cols * 2 bytes a multiple of 16, base 16-byte
// aligned), boxes of 64 columns x box_rows rows, 128-byte swizzle; out-of-range reads are zero.
CUtensorMap make_map_bf16(const void* base, int64_t rows, int64_t cols, int box_rows) {
  GW_REQUIRE(cols % 8 == 0 && ((uintptr_t)base & 15) == 0 && box_rows >= 1 && box_rows <= 256,
             GWAS_ERR_ARG, "tensor map arguments not TMA-aligned");
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                           strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  GW_REQUIRE(r == CUDA_SUCCESS, GWAS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return m;
}

// 2-D uint8 map over packed genotype rows [rows][row_bytes] (row_bytes a multiple of 16, base
// 16-byte aligned), boxes of 16 bytes x box_rows rows, no swizzle; rows past the end read as zero.
CUtensorMap make_map_packed(const void* base, int64_t rows, int row_bytes, int box_rows) {
  GW_REQUIRE(row_bytes % 16 == 0 && ((uintptr_t)base & 15) == 0 && rows >= 1 &&
                 rows <= ((int64_t)1 << 32) && box_rows >= 1 && box_rows <= 256,
             GWAS_ERR_ARG, "packed genotypes not TMA-aligned (base and rows need 16 bytes)");
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)row_bytes, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
  cuuint32_t box[2] = {16, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims,
                           strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  GW_REQUIRE(r == CUDA_SUCCESS, GWAS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return m;
}

// 2-D uint8 map over [rows][cols] bytes, boxes of 64 bytes x box_rows rows, 64-byte swizzle.
CUtensorMap make_map_u8_sw64(const void* base, int64_t rows, int64_t cols, int box_rows) {
  GW_REQUIRE(cols % 16 == 0 && ((uintptr_t)base & 15) == 0 && box_rows >= 1 && box_rows <= 256,
             GWAS_ERR_ARG, "tensor map arguments not TMA-aligned");
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols};
  cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims,
                           strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  GW_REQUIRE(r == CUDA_SUCCESS, GWAS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return m;
}

// Per-trait constants of the FP16 + E4M3 split (SPLIT_FP8): see CholTcParams.
struct FP8Consts {
  std::vector<float> unscale, lsa;
  double k2 = 0.0;
};

struct TcState {
  int algo = 0, n = 0, q = 0, t = 0;
  int kpad = 0, rpad = 0, num_sms = 0;
  std::vector<void*> allocs;
  // CHOL, per trait: split L^-1 (hi rows then lo rows) and its tensor maps
  std::vector<CholMaps> lmaps;
  std::vector<int> lpieces;         // split pieces of each trait's matrix (2 or 3)
  std::vector<uint8_t> lfp8;        // trait's split is FP16 hi + E4M3 lo (SPLIT_FP8)
  std::vector<FP8Consts> lconst;    // per trait: the FP8 split's scales and lo-row sums
  __nv_bfloat16* Lsplit = nullptr;  // per trait (pieces rpad) x kpad, traits one after another
                                    // (an FP8 trait: its FP16 hi piece, then the E4M3 lo bytes
                                    // in the space of half a piece)
  const double* P = nullptr;        // t x q x q (owned by the handle)
  const double* b0 = nullptr;       // t x q
  // EIG: split operands, FP32 null-model blocks, per-block scratch and tensor maps
  __nv_bfloat16 *Zsplit = nullptr, *Usplit = nullptr, *dsplit = nullptr, *xsq = nullptr;
  float *P32 = nullptr, *b032 = nullptr, *sbuf = nullptr;
  // EIG: per-SNP centres of the current chunk (NULL: no intercept, no centring)
  float* mu = nullptr;
  // CHOL states of an EIG handle's badly conditioned traits: local trait k is global jmap[k] of
  // tglobal traits (empty jmap: the identity)
  TcState* route = nullptr;
  std::vector<int> jmap;
  int tglobal = 0;
  int64_t mcap = 0;    // SNPs per chunk the scratch holds
  int64_t chunk = 0;   // SNPs per chunk the scan uses (<= mcap; 0: mcap)
  bool intercept = false;
  int out_snp = 0;
  int out_var = 0;
  int traits_ac = 0;
  int upieces = 2;  // split pieces of U
  GeneticModel gm;
  CUtensorMap mapZ, mapU, mapD, mapX;
};

namespace {
void* tc_alloc(TcState* st, size_t bytes) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    throw Fail{GWAS_ERR_OOM};
  }
  st->allocs.push_back(p);
  return p;
}
}  // namespace

void tc_check_supported(int algo, int n, int q, int t) {
  (void)algo;
  GW_REQUIRE(q >= 1 && q <= QMAX, GWAS_ERR_UNSUPPORTED, "q=%d outside [1,%d]", q, QMAX);
  GW_REQUIRE(n >= 1 && t >= 1, GWAS_ERR_ARG, "bad sizes");
}

TcState* tc_setup(cudaStream_t s, const TcSetupArgs& a) {
  TcState* st = new TcState();
  try {
    st->algo = a.algo;
    st->n = a.n;
    st->q = a.q;
    st->t = a.t;
    st->P = a.P;
    st->b0 = a.b0;
    st->intercept = a.intercept != 0;
    st->out_snp = a.out_snp;
    st->out_var = a.out_var;
    st->gm = a.gm;
    int dev = 0;
    GW_CUDA(cudaGetDevice(&dev));
    GW_CUDA(cudaDeviceGetAttribute(&st->num_sms, cudaDevAttrMultiProcessorCount, dev));
    const int n = a.n, q = a.q, t = a.t;
    st->kpad = (int)round_up(n, 64);
    st->rpad = (int)round_up(n, 256);
    if (a.algo == GWAS_ALGO_CHOL) {
      // Per trait, the split rows of [L^-1; (M^-1 X_L)^T; (M^-1 r)^T]: M^-1 X_L = L^-T (L^-1 X_L)
      // and M^-1 r = L^-T (L^-1 r) are linear in the genotypes, so the whitening product also
      // yields a_k and c (Algorithm 3) in q + 1 extra accumulator columns.
      // (SPLIT_FP8: one more augmented row, w)
      st->rpad = (int)round_up(n + q + 1 + (a.fp8_lo ? 1 : 0), 256);
      const size_t piece = (size_t)st->rpad * st->kpad;  // elements of one piece
      size_t total = 0;
      for (int j = 0; j < t; ++j) {
        st->lpieces.push_back(a.pieces && a.pieces[j] == 3 ? 3 : 2);
        st->lfp8.push_back(a.fp8_lo && st->lpieces[j] == 2 ? 1 : 0);
        total += st->lfp8[j] ? piece + piece / 2 : piece * st->lpieces[j];
      }
      st->Lsplit = (__nv_bfloat16*)tc_alloc(st, total * 2);
      GW_CUDA(cudaMemsetAsync(st->Lsplit, 0, total * 2, s));
      double* Ut = (double*)tc_alloc(st, (size_t)(q + 1) * n * 8);
      double* rmax = nullptr;  // FP8: row maxima, row scales, w (natural column order)
      float* ls = nullptr;      // FP8: the sums of the lo rows of one trait
      if (a.fp8_lo) {
        rmax = (double*)tc_alloc(st, (size_t)(3 * n + 2 * (q + 2)) * 8);
        ls = (float*)tc_alloc(st, (size_t)(n + q + 2) * 4);
      }
      size_t off = 0;
      for (int j = 0; j < t; ++j) {
        const int np = st->lpieces[j];
        const double* Li = a.Linv + (size_t)j * n * n;
        if (st->lfp8[j]) {
          // FP16 hi + E4M3 lo.  Row groups (the rows of L^-1; each augmented row) are scaled by
          // powers of two that bring their largest magnitude into (2^13, 2^14]: FP16 keeps its
          // full precision there and lo (<= 2^-11 of it) stays inside E4M3's range.  One more
          // augmented row, w = sum_{r < n} lsum_r (hi + lo)_r (lsum_r: the sum of row r's lo
          // piece), lets the epilogue remove the centring term the lo product misses.
          __half* hi = reinterpret_cast<__half*>(st->Lsplit + off);
          uint8_t* lo = reinterpret_cast<uint8_t*>(st->Lsplit + off + piece);
          off += piece + piece / 2;
          gemm_f64(s, q, n, n, 1.0, a.XLw + (size_t)j * q * n, n, 1, Li, n, 1, 0.0, Ut, n, 1);
          gemm_f64(s, 1, n, n, 1.0, a.rw + (size_t)j * n, n, 1, Li, n, 1, 0.0,
                   Ut + (size_t)q * n, n, 1);
          const int na = q + 2;  // augmented rows: X_L's q, the residual, w
          double* dmax = rmax;
          double* dsc = rmax + (n + na);
          double* wnat = rmax + 2 * (n + na);
          rowmax_abs(s, Li, n, n, n, dmax);
          rowmax_abs(s, Ut, q + 1, n, n, dmax + n);
          std::vector<double> hm(n + na), hs(n + na);
          GW_CUDA(cudaMemcpyAsync(hm.data(), dmax, (size_t)(n + q + 1) * 8, cudaMemcpyDeviceToHost, s));
          GW_CUDA(cudaStreamSynchronize(s));
          auto exp_of = [](double mx) { return mx > 0.0 ? 14 - (int)ceil(log2(mx)) : 0; };
          double mL = 0.0;
          for (int r = 0; r < n; ++r) mL = hm[r] > mL ? hm[r] : mL;
          std::vector<float> us(na + 1);
          const int eL = exp_of(mL);
          us[0] = ldexpf(1.f, -eL);
          for (int r = 0; r < n; ++r) hs[r] = ldexp(1.0, eL);
          for (int k = 0; k <= q; ++k) {
            const int e = exp_of(hm[n + k]);
            us[1 + k] = ldexpf(1.f, -e);
            hs[n + k] = ldexp(1.0, e);
          }
          GW_CUDA(cudaMemcpyAsync(dsc, hs.data(), (size_t)(n + q + 1) * 8, cudaMemcpyHostToDevice, s));
          const size_t aug = (size_t)n * st->kpad;
          split_f16_e4m3(s, Li, n, n, n, dsc, hi, lo, st->kpad);
          split_f16_e4m3(s, Ut, q + 1, n, n, dsc + n, hi + aug, lo + aug, st->kpad);
          e4m3_row_sums(s, lo, n + q + 1, st->kpad, ls);
          e4m3_weighted_col_sums(s, hi, lo, n, st->kpad, n, ls, wnat);
          rowmax_abs(s, wnat, 1, n, n, dmax + n + q + 1);
          GW_CUDA(cudaMemcpyAsync(hm.data() + n + q + 1, dmax + n + q + 1, 8,
                                  cudaMemcpyDeviceToHost, s));
          GW_CUDA(cudaStreamSynchronize(s));
          const int ew = exp_of(hm[n + q + 1]);
          us[na] = ldexpf(1.f, -ew);
          hs[n + q + 1] = ldexp(1.0, ew);
          GW_CUDA(cudaMemcpyAsync(dsc + n + q + 1, &hs[n + q + 1], 8, cudaMemcpyHostToDevice, s));
          const size_t wrow = (size_t)(n + q + 1) * st->kpad;
          split_f16_e4m3(s, wnat, 1, n, n, dsc + n + q + 1, hi + wrow, lo + wrow, st->kpad);
          e4m3_row_sums(s, lo + wrow, 1, st->kpad, ls + n + q + 1);
          std::vector<float> hls(n + na);
          GW_CUDA(cudaMemcpyAsync(hls.data(), ls, hls.size() * 4, cudaMemcpyDeviceToHost, s));
          // the stream must be done with hs before the next trait reuses the buffers
          GW_CUDA(cudaStreamSynchronize(s));
          FP8Consts fc;
          fc.unscale = us;
          fc.lsa.assign(hls.begin() + n, hls.end());
          fc.k2 = 0.0;
          for (int r = 0; r < n; ++r) fc.k2 += (double)hls[r] * hls[r];
          st->lconst.push_back(fc);
          CholMaps mp;
          for (int r = 0; r < 4; ++r) {
            mp.m[r] = make_map_bf16(hi, st->rpad, st->kpad, 256 - 64 * r);
            mp.m8[r] = make_map_u8_sw64(lo, st->rpad, st->kpad, 256 - 64 * r);
          }
          st->lmaps.push_back(mp);
          continue;
        }
        st->lconst.push_back(FP8Consts());
        __nv_bfloat16* hi = st->Lsplit + off;
        __nv_bfloat16* lo = hi + piece;
        __nv_bfloat16* lo2 = np == 3 ? lo + piece : nullptr;
        off += piece * np;
        split_bf16(s, Li, n, n, n, hi, lo, st->kpad, lo2);
        gemm_f64(s, q, n, n, 1.0, a.XLw + (size_t)j * q * n, n, 1, Li, n, 1, 0.0, Ut, n, 1);
        gemm_f64(s, 1, n, n, 1.0, a.rw + (size_t)j * n, n, 1, Li, n, 1, 0.0, Ut + (size_t)q * n,
                 n, 1);
        const size_t aug = (size_t)n * st->kpad;  // the q + 1 augmented rows follow L^-1's n
        split_bf16(s, Ut, q + 1, n, n, hi + aug, lo + aug, st->kpad, lo2 ? lo2 + aug : nullptr);
        CholMaps mp;
        for (int r = 0; r < 4; ++r) {
          mp.m[r] = make_map_bf16(hi, (int64_t)np * st->rpad, st->kpad, 256 - 64 * r);
          mp.m8[r] = mp.m[r];  // unused
        }
        st->lmaps.push_back(mp);
      }
      GW_CUDA(cudaStreamSynchronize(s));
      cudaFree(Ut);
      st->allocs.erase(std::find(st->allocs.begin(), st->allocs.end(), (void*)Ut));
      for (void* tmp : {(void*)rmax, (void*)ls}) {
        if (!tmp) continue;
        cudaFree(tmp);
        st->allocs.erase(std::find(st->allocs.begin(), st->allocs.end(), tmp));
      }
      chol_tc_prepare();
      return st;
    }
    // EIG.  Z^T split (rows = eigenvectors).
    const int kp = st->kpad, q1 = q + 1, q2 = q + 2;
    const size_t zrows = (size_t)st->rpad;
    // U_j takes a third BF16 piece when some M_j is badly conditioned; Z^T (orthonormal), d_j
    // and the squared planes (positive sums) keep two: at that conditioning the FP32 accumulation
    // of the contractions, not their operands' 16 bits, bounds s_ij
    st->upieces = a.pieces && a.pieces[0] == 3 ? 3 : 2;
    st->Zsplit = (__nv_bfloat16*)tc_alloc(st, 2 * zrows * kp * 2);
    GW_CUDA(cudaMemsetAsync(st->Zsplit, 0, 2 * zrows * kp * 2, s));
    split_bf16(s, a.Zt, n, n, n, st->Zsplit, st->Zsplit + zrows * kp, kp);
    // U_j = Z [d_j o X~_L | d_j o r~_j] = M_j^-1 [X_L | r_j], one row per (trait, column):
    // Uall[row][c] = sum_r planes[row][r] Z^T[r][c] over all q+2 plane rows (the last is unused)
    double* Uall = (double*)tc_alloc(st, (size_t)t * q2 * a.ldp * 8);
    gemm_f64(s, t * q2, n, n, 1.0, a.planes, a.ldp, 1, a.Zt, n, 1, 0.0, Uall, a.ldp, 1);
    const size_t upiece = (size_t)t * q1 * kp;
    st->Usplit = (__nv_bfloat16*)tc_alloc(st, (size_t)st->upieces * upiece * 2);
    split_bf16_rows(s, Uall, t * q1, n, a.ldp, q2, q1, 0, st->Usplit, st->Usplit + upiece, kp,
                    st->upieces == 3 ? st->Usplit + 2 * upiece : nullptr);
    // d_j (the last plane row of each trait), split
    st->dsplit = (__nv_bfloat16*)tc_alloc(st, (size_t)2 * t * kp * 2);
    split_bf16_rows(s, a.planes, t, n, a.ldp, q2, 1, q + 1, st->dsplit,
                    st->dsplit + (size_t)t * kp, kp);
    st->P32 = (float*)tc_alloc(st, (size_t)t * q * q * 4);
    st->b032 = (float*)tc_alloc(st, (size_t)t * q * 4);
    convert_f64_to_f32(s, a.P, st->P32, (int64_t)t * q * q);
    convert_f64_to_f32(s, a.b0, st->b032, (int64_t)t * q);
    GW_CUDA(cudaStreamSynchronize(s));
    cudaFree(Uall);
    st->allocs.erase(std::find(st->allocs.begin(), st->allocs.end(), (void*)Uall));
    // traits per AC column block: T (q+1) columns, the last trait's load of QP columns in range
    st->traits_ac = eig_ac_traits(q);
    // SNPs per internal chunk: at least the streaming block, up to 32 Ki while the s scratch
    // (t x chunk FP32) stays within 4 GB, so that many-trait scans keep every SM busy
    // (a two-column genetic model has three squared planes per SNP: x0 x0, x0 x1, x1 x1)
    const int np = a.gm.pr == 2 ? 3 : 1;
    int64_t cap = (int64_t)(4e9 / (4.0 * t * np));
    cap = cap < 32768 ? cap : 32768;
    cap = cap > a.block_snps ? cap : a.block_snps;
    st->mcap = round_up(cap > 128 ? cap : 128, 128);
    st->xsq = (__nv_bfloat16*)tc_alloc(st, (size_t)2 * np * st->mcap * kp * 2);
    st->sbuf = (float*)tc_alloc(st, (size_t)t * np * st->mcap * 4);
    // With an intercept in X_L, each SNP is centred by a multiple of 1/64 near its mean: the
    // estimates of b_snp and its Wald statistic are unchanged, the intercept is corrected
    // exactly, and the large intercept-direction component no longer cancels in
    // sigma = x^T M^-1 x - a^T S_TL^-1 a (which would amplify the BF16 splitting error).
    if (a.intercept) st->mu = (float*)tc_alloc(st, (size_t)st->mcap * a.gm.pr * 4);
    st->mapZ = make_map_bf16(st->Zsplit, 2 * (int64_t)zrows, kp, 256);
    st->mapU = make_map_bf16(st->Usplit, (int64_t)st->upieces * t * q1, kp, 256);
    st->mapD = make_map_bf16(st->dsplit, 2 * (int64_t)t, kp, 256);
    st->mapX = make_map_bf16(st->xsq, 2 * (int64_t)np * st->mcap, kp, 128);
    eig_tc_prepare();
    return st;
  } catch (...) {
    tc_destroy(st);
    throw;
  }
}

double tc_scan_work(const TcState* st, int64_t m) {
  const double kp = st->kpad, rp = st->rpad, t = st->t, q1 = st->q + 1;
  if (st->algo == GWAS_ALGO_CHOL) return 2.0 * kp * rp * t * (double)m;  // ~ half the square x 2 pieces x 2 flops
  return (4.0 * rp * kp + t * kp * (6.0 + 4.0 * q1)) * (double)m +
         (st->route ? tc_scan_work(st->route, m) : 0.0);
}

void tc_attach_chol_route(cudaStream_t s, TcState* st, TcState* route,
                          const std::vector<int>& jmap) {
  GW_REQUIRE(st && route && st->algo == GWAS_ALGO_EIG && route->algo == GWAS_ALGO_CHOL &&
                 (int)jmap.size() == route->t,
             GWAS_ERR_ARG, "bad CHOL route");
  route->jmap = jmap;
  route->tglobal = st->t;
  st->route = route;
  // NaN as the first entry of P_j in the a/c kernel's FP32 constants: that kernel then leaves
  // the trait out of its singular count (its outputs are overwritten by the CHOL pass)
  const float nanv = std::numeric_limits<float>::quiet_NaN();
  for (int j : jmap)
    GW_CUDA(cudaMemcpyAsync(st->P32 + (size_t)j * st->q * st->q, &nanv, 4,
                            cudaMemcpyHostToDevice, s));
  GW_CUDA(cudaStreamSynchronize(s));
}

int tc_chol_routed_traits(const TcState* st) {
  return st && st->route ? st->route->t : 0;
}

void tc_scan(cudaStream_t s, TcState* st, const TcScanArgs& a) {
  if (a.m <= 0) return;
  GW_REQUIRE(st != nullptr, GWAS_ERR_ARG, "no tensor-core state");
  const int ctas = a.max_ctas > 0 && a.max_ctas < st->num_sms ? a.max_ctas : st->num_sms;
  const int rb = packed_row_bytes(st->n);
  if (st->algo == GWAS_ALGO_CHOL) {
    const CUtensorMap mapG = make_map_packed(a.G, a.m, rb, CHOL_TC_BM / st->gm.pr);
    for (int j = 0; j < st->t; ++j) {
      CholTcParams p{};
      p.m = a.m;
      p.n = st->n;
      p.q = st->q;
      p.t = st->tglobal > 0 ? st->tglobal : st->t;
      p.j = st->jmap.empty() ? j : st->jmap[j];
      p.kpad = st->kpad;
      p.rpad = st->rpad;
      p.P = st->P + (size_t)j * st->q * st->q;
      p.b0 = st->b0 + (size_t)j * st->q;
      p.centre = st->intercept ? 1 : 0;
      p.out_snp = st->out_snp;
      p.out_var = st->out_var;
      p.G = a.G;
      p.row_bytes = rb;
      p.gp = st->gm.pr;
      p.code[0] = st->gm.code_word(0);
      p.code[1] = st->gm.code_word(1);
      for (int e = 0; e < 4; ++e) p.tm[e] = st->gm.tm[e / 2][e % 2];
      p.pieces = st->lpieces[j];
      p.fp8 = st->lfp8[j];
      p.naug = st->q + 1 + (p.fp8 ? 1 : 0);
      if (p.fp8) {
        const FP8Consts& fc = st->lconst[j];
        for (size_t g = 0; g < fc.unscale.size() && g < 10; ++g) p.unscale[g] = fc.unscale[g];
        for (size_t g = 0; g < fc.lsa.size() && g < 9; ++g) p.lsa[g] = fc.lsa[g];
        p.k2 = fc.k2;
      }
      p.B = a.B;
      p.W = a.wald;
      p.flags = a.flags;
      cudaEvent_t ev = a.timer ? a.timer->begin(s, STAGE_CHOL) : nullptr;
      chol_tc_launch(s, st->lmaps[j], mapG, p, ctas);
      if (ev) a.timer->end(s, ev);
    }
    return;
  }
  const int n = st->n, q = st->q, t = st->t, q1 = q + 1;
  const int64_t ck = st->chunk > 0 && st->chunk < st->mcap ? st->chunk : st->mcap;
  for (int64_t off = 0; off < a.m; off += ck) {
    const int64_t mm = a.m - off < ck ? a.m - off : ck;
    EigTcParams p{};
    p.m = mm;
    p.n = n;
    p.q = q;
    p.t = t;
    p.kpad = st->kpad;
    const int gp = st->gm.pr, np = gp == 2 ? 3 : 1;
    p.a_piece_rows = (int)(np * st->mcap);
    p.xsq = st->xsq;
    p.sbuf = st->sbuf;
    p.lds = np * st->mcap;
    p.xplane = round_up(mm, 128);  // gp = 2: rows of each squared plane of this chunk
    p.flags = a.flags;
    p.gp = st->gm.pr;
    p.code[0] = st->gm.code_word(0);
    p.code[1] = st->gm.code_word(1);
    for (int e = 0; e < 4; ++e) p.tm[e] = st->gm.tm[e / 2][e % 2];
    // ROT: Xsq = (Z^T x)^2 for this chunk (Algorithm 4's rotation, squared and split)
    const uint8_t* Gc = a.G + off * rb;
    const CUtensorMap mapG = make_map_packed(Gc, mm, rb, 128 / gp);
    StageTimer* tm = a.timer;
    cudaEvent_t ev = nullptr;
    if (st->mu) {
      ev = tm ? tm->begin(s, STAGE_CENTRES) : nullptr;
      const uint32_t codes[2] = {st->gm.code_word(0), st->gm.code_word(1)};
      snp_centres_packed(s, Gc, mm, n, st->mu, st->gm.pr, codes);
      if (ev) tm->end(s, ev);
    }
    p.mu = st->mu;
    p.nblk = st->rpad / 256;
    p.pieces = 2;  // Z^T (and, in SQ, the squared planes and d_j): two pieces
    p.b_piece_rows = st->rpad;
    p.b_rows_per_blk = 256;
    ev = tm ? tm->begin(s, STAGE_ROT) : nullptr;
    eig_tc_launch(s, 0, st->mapZ, st->mapZ, mapG, p, ctas);
    if (ev) tm->end(s, ev);
    // SQ: s_ij = sum_r Xsq[i][r] d_j[r] (gp = 2: over the rows of all three planes)
    p.m = gp == 2 ? 3 * p.xplane : mm;
    p.nblk = (t + 255) / 256;
    p.b_piece_rows = t;
    p.b_rows_per_blk = 256;
    ev = tm ? tm->begin(s, STAGE_SQ) : nullptr;
    eig_tc_launch(s, 1, st->mapX, st->mapD, mapG, p, ctas);
    if (ev) tm->end(s, ev);
    // AC: a_ij, c_ij from the genotypes against U, then the bordered solve (Algorithm 4)
    p.m = mm;
    p.nblk = (t + st->traits_ac - 1) / st->traits_ac;
    p.b_piece_rows = t * q1;
    p.b_rows_per_blk = st->traits_ac * q1;
    p.traits_per_blk = st->traits_ac;
    p.pieces = st->upieces;
    p.P = st->P32;
    p.b0 = st->b032;
    const int pp = q + gp;  // coefficients per pair
    p.B = a.B + (size_t)off * t * (st->out_snp ? 2 * gp : st->out_var ? pp + pp * (pp + 1) / 2 : pp);
    p.out_snp = st->out_snp;
    p.out_var = st->out_var;
    p.W = a.wald ? a.wald + (size_t)off * t : nullptr;
    ev = tm ? tm->begin(s, STAGE_AC) : nullptr;
    eig_tc_launch(s, 2, st->mapU, st->mapU, mapG, p, ctas);
    if (ev) tm->end(s, ev);
  }
  // the badly conditioned traits again, with the CHOL kernel (their outputs overwritten)
  if (st->route) tc_scan(s, st->route, a);
}

int64_t tc_eig_chunk(const TcState* st) {
  if (!st || st->algo == GWAS_ALGO_CHOL) return 0;
  return st->chunk > 0 && st->chunk < st->mcap ? st->chunk : st->mcap;
}

int64_t tc_eig_chunk_capacity(const TcState* st) {
  return st && st->algo != GWAS_ALGO_CHOL ? st->mcap : 0;
}

void tc_set_eig_chunk(TcState* st, int64_t snps) {
  if (!st || st->algo == GWAS_ALGO_CHOL) return;
  snps = round_up(snps < 128 ? 128 : snps, 128);
  st->chunk = snps < st->mcap ? snps : st->mcap;
}

int tc_fp8_traits(const TcState* st) {
  int k = 0;
  if (st)
    for (uint8_t v : st->lfp8) k += v;
  return k;
}

int tc_split_pieces(const TcState* st) {
  if (!st) return 0;
  int np = st->algo == GWAS_ALGO_CHOL ? 2 : st->upieces;
  for (int v : st->lpieces) np = v > np ? v : np;
  return np;
}

void tc_destroy(TcState* st) {
  if (!st) return;
  tc_destroy(st->route);
  for (void* p : st->allocs) cudaFree(p);
  delete st;
}

}  // namespace gw
