// Host side of the split-BF16 tensor-core path: operand splitting, tensor maps, dispatch.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <vector>

#include "tc.cuh"
#include "tc_kernels.cuh"

namespace gw {

namespace {

constexpr int QMAX = 7;

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
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

struct TcState {
  int algo = 0, n = 0, q = 0, t = 0;
  int kpad = 0, rpad = 0, num_sms = 0;
  std::vector<void*> allocs;
  // CHOL, per trait: split L^-1 (hi rows then lo rows) and its two tensor maps
  std::vector<CUtensorMap> lmap256, lmap128;
  __nv_bfloat16* Lsplit = nullptr;  // t x (2 rpad) x kpad
  float* XLw32 = nullptr;           // t x q x n
  float* rw32 = nullptr;            // t x n
  const double* P = nullptr;        // t x q x q (owned by the handle)
  const double* b0 = nullptr;       // t x q
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
  GW_REQUIRE(algo == GWAS_ALGO_CHOL, GWAS_ERR_UNSUPPORTED,
             "split-BF16 tensor-core EIG path is not available in this build");
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
    int dev = 0;
    GW_CUDA(cudaGetDevice(&dev));
    GW_CUDA(cudaDeviceGetAttribute(&st->num_sms, cudaDevAttrMultiProcessorCount, dev));
    const int n = a.n, q = a.q, t = a.t;
    st->kpad = (int)round_up(n, 64);
    st->rpad = (int)round_up(n, 256);
    const size_t per = (size_t)2 * st->rpad * st->kpad;
    st->Lsplit = (__nv_bfloat16*)tc_alloc(st, per * t * 2);
    GW_CUDA(cudaMemsetAsync(st->Lsplit, 0, per * t * 2, s));
    st->XLw32 = (float*)tc_alloc(st, (size_t)t * q * n * 4);
    st->rw32 = (float*)tc_alloc(st, (size_t)t * n * 4);
    convert_f64_to_f32(s, a.XLw, st->XLw32, (int64_t)t * q * n);
    convert_f64_to_f32(s, a.rw, st->rw32, (int64_t)t * n);
    for (int j = 0; j < t; ++j) {
      __nv_bfloat16* hi = st->Lsplit + per * j;
      __nv_bfloat16* lo = hi + (size_t)st->rpad * st->kpad;
      split_bf16(s, a.Linv + (size_t)j * n * n, n, n, n, hi, lo, st->kpad);
      st->lmap256.push_back(make_map_bf16(hi, 2 * (int64_t)st->rpad, st->kpad, 256));
      st->lmap128.push_back(make_map_bf16(hi, 2 * (int64_t)st->rpad, st->kpad, 128));
    }
    chol_tc_prepare();
    return st;
  } catch (...) {
    tc_destroy(st);
    throw;
  }
}

void tc_scan(cudaStream_t s, TcState* st, const TcScanArgs& a) {
  if (a.m <= 0) return;
  GW_REQUIRE(st != nullptr, GWAS_ERR_ARG, "no tensor-core state");
  for (int j = 0; j < st->t; ++j) {
    CholTcParams p{};
    p.XR = a.XR;
    p.m = a.m;
    p.n = st->n;
    p.q = st->q;
    p.t = st->t;
    p.j = j;
    p.kpad = st->kpad;
    p.rpad = st->rpad;
    p.XLw = st->XLw32 + (size_t)j * st->q * st->n;
    p.rw = st->rw32 + (size_t)j * st->n;
    p.P = st->P + (size_t)j * st->q * st->q;
    p.b0 = st->b0 + (size_t)j * st->q;
    p.B = a.B;
    p.W = a.wald;
    p.flags = a.flags;
    chol_tc_launch(s, st->lmap256[j], st->lmap128[j], p, st->num_sms);
  }
}

void tc_destroy(TcState* st) {
  if (!st) return;
  for (void* p : st->allocs) cudaFree(p);
  delete st;
}

}  // namespace gw
