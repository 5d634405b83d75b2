// Tensor-core split-BF16 scan (tcgen05 / TMEM / TMA, sm_103a).
//
// CHOL (Algorithm 3 lines 4 and 8-11).  One CTA owns 128 SNPs.  For each block of 256 rows of
// L^-1 it accumulates D = X^T (L^-1)^T, i.e. D[snp][r] = (L^-1 x_snp)_r, in TMEM over only the
// columns c <= r that L^-1 can have nonzero (the triangular solve of "Sequences of GLS'", as one
// product with the precomputed inverse).  L^-1 = hi + lo with BF16 pieces; genotypes are exact in
// BF16, so D = X^T hi^T + X^T lo^T carries ~16 significant bits of L^-1 with FP32 accumulation.
// The epilogue reduces each D row block straight out of TMEM into the bordered-system entries
//   s = x'^T x',  c = r'^T x',  a_k = (L^-1 X_L)_k^T x'
// (FP32 over 32 columns, FP64 across chunks) and finishes with the Schur-complement solve in FP64.
// X' = L^-1 X_R is never written to memory.
//
// Warp roles (320 threads): 0-3 epilogue (one SNP per thread = one TMEM lane), 4 TMA producer of
// the L^-1 tiles, 5 MMA issuer and TMEM owner, 6-9 genotype converters (int8 global -> BF16
// swizzled shared tiles).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <vector>

#include "tc.cuh"
#include "tc_ptx.cuh"

namespace gw {
using namespace tc;

namespace {

constexpr int BM = 128;                 // SNPs per CTA tile
constexpr int BN = 256;                 // rows of L^-1 per accumulator block
constexpr int BK = 64;                  // K per pipeline step (one 128-byte swizzle row)
constexpr int SA = 3;                   // genotype tile ring
constexpr int SB = 4;                   // L^-1 tile ring (one piece per slot)
constexpr int A_BYTES = BM * BK * 2;    // 16 KB
constexpr int B_BYTES = BN * BK * 2;    // 32 KB
constexpr int QMAX = 7;
constexpr int CST_FLOATS = (QMAX + 1) * BN;
constexpr int NUM_THREADS = 320;
constexpr int TMEM_COLS = 512;          // two 256-column accumulators
constexpr uint64_t WAIT_NS = 4000000000ull;

struct __align__(8) Bars {
  uint64_t a_full[SA], a_empty[SA], b_full[SB], b_empty[SB], acc_full[2], acc_empty[2], done;
  uint32_t tmem_base;
  int abort;
};

constexpr size_t SMEM_BYTES = 1024 + SA * A_BYTES + SB * B_BYTES + CST_FLOATS * 4 + sizeof(Bars);

struct CholTcParams {
  const int8_t* XR;
  int64_t m;
  int n, q, t, j;
  int kpad, rpad, nblocks;
  const float* XLw;   // q x n, this trait
  const float* rw;    // n
  const double* P;    // q x q
  const double* b0;   // q
  float* B;
  float* W;
  int* flags;
  int aligned8;
};

__device__ __forceinline__ int chol_ksteps(int nb, int kpad) {
  const int k = (nb + 1) * (BN / BK);
  const int kmax = kpad / BK;
  return k < kmax ? k : kmax;
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    chol_tc_kernel(const __grid_constant__ CUtensorMap tmapL, const CholTcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = sA + SA * A_BYTES;
  float* cst = (float*)(sB + SB * B_BYTES);
  Bars* bars = (Bars*)(cst + CST_FLOATS);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t s0 = (int64_t)blockIdx.x * BM;
  int* tflag = p.flags + FLAG_TIMEOUT;

  if (threadIdx.x == 0) {
    for (int i = 0; i < SA; ++i) {
      mbar_init(&bars->a_full[i], 128);
      mbar_init(&bars->a_empty[i], 1);
    }
    for (int i = 0; i < SB; ++i) {
      mbar_init(&bars->b_full[i], 1);
      mbar_init(&bars->b_empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bars->acc_full[i], 1);
      mbar_init(&bars->acc_empty[i], 4);
    }
    mbar_init(&bars->done, 1);
    bars->abort = 0;
    fence_mbar_init();
  }
  if (warp == 5) {
    tmem_alloc(&bars->tmem_base, TMEM_COLS);
    tmem_relinquish();
  }
  if (warp == 4 && lane == 0) prefetch_tensormap(&tmapL);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  volatile int* abort = &bars->abort;

  if (warp == 4) {
    // ---------------------------------------------------------------- L^-1 tiles via TMA
    if (lane == 0) {
      int bs = 0;
      uint32_t bph = 0;
      bool ok = true;
      for (int nb = 0; nb < p.nblocks && ok; ++nb) {
        const int nk = chol_ksteps(nb, p.kpad);
        for (int ks = 0; ks < nk && ok; ++ks)
          for (int piece = 0; piece < 2 && ok; ++piece) {
            ok = mbar_wait(&bars->b_empty[bs], bph ^ 1, abort, tflag, WAIT_NS);
            if (!ok) break;
            mbar_arrive_expect_tx(&bars->b_full[bs], B_BYTES);
            tma_load_2d(sB + bs * B_BYTES, &tmapL, &bars->b_full[bs], ks * BK,
                        piece * p.rpad + nb * BN);
            if (++bs == SB) { bs = 0; bph ^= 1; }
          }
      }
    }
  } else if (warp == 5) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      int as = 0, bs = 0;
      uint32_t aph = 0, bph = 0;
      bool ok = true;
      const uint32_t idesc = idesc_bf16(BM, BN);
      for (int nb = 0; nb < p.nblocks && ok; ++nb) {
        const int buf = nb & 1;
        ok = mbar_wait(&bars->acc_empty[buf], ((nb >> 1) & 1) ^ 1, abort, tflag, WAIT_NS);
        if (!ok) break;
        tc_fence_after();
        const uint32_t dt = tmem + buf * BN;
        const int nk = chol_ksteps(nb, p.kpad);
        for (int ks = 0; ks < nk && ok; ++ks) {
          ok = mbar_wait(&bars->a_full[as], aph, abort, tflag, WAIT_NS);
          if (!ok) break;
          tc_fence_after();
          const uint64_t ad = sw128_desc(sA + as * A_BYTES);
          for (int piece = 0; piece < 2 && ok; ++piece) {
            ok = mbar_wait(&bars->b_full[bs], bph, abort, tflag, WAIT_NS);
            if (!ok) break;
            tc_fence_after();
            const uint64_t bd = sw128_desc(sB + bs * B_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
              mma_bf16(dt, ad + 2 * kk, bd + 2 * kk, idesc, (ks | piece | kk) != 0);
            mma_commit(&bars->b_empty[bs]);
            if (++bs == SB) { bs = 0; bph ^= 1; }
          }
          mma_commit(&bars->a_empty[as]);
          if (++as == SA) { as = 0; aph ^= 1; }
        }
        if (ok) mma_commit(&bars->acc_full[buf]);
      }
      // every MMA issued by this thread has finished before TMEM is released
      mma_commit(&bars->done);
      mbar_wait(&bars->done, 0, abort, tflag, WAIT_NS);
    }
  } else if (warp >= 6) {
    // ---------------------------------------------------------------- genotype converters
    const int ct = threadIdx.x - 192;
    int as = 0;
    uint32_t aph = 0;
    bool ok = true;
    for (int nb = 0; nb < p.nblocks && ok; ++nb) {
      const int nk = chol_ksteps(nb, p.kpad);
      for (int ks = 0; ks < nk && ok; ++ks) {
        uint2 v[8];
#pragma unroll
        for (int l = 0; l < 8; ++l) {
          const int e = ct + 128 * l, r = e >> 3, jc = e & 7;
          const int64_t snp = s0 + r;
          const int k = ks * BK + jc * 8;
          v[l] = make_uint2(0u, 0u);
          if (snp < p.m && k < p.n) {
            const int8_t* src = p.XR + snp * p.n + k;
            if (p.aligned8) {
              v[l] = __ldg(reinterpret_cast<const uint2*>(src));
            } else {
              uint32_t w[2] = {0u, 0u};
#pragma unroll
              for (int b = 0; b < 8; ++b)
                if (k + b < p.n) w[b >> 2] |= (uint32_t)(uint8_t)src[b] << (8 * (b & 3));
              v[l] = make_uint2(w[0], w[1]);
            }
          }
        }
        ok = mbar_wait(&bars->a_empty[as], aph ^ 1, abort, tflag, WAIT_NS);
        if (!ok) break;
        uint8_t* tile = sA + as * A_BYTES;
#pragma unroll
        for (int l = 0; l < 8; ++l) {
          const int e = ct + 128 * l, r = e >> 3, jc = e & 7;
          uint8_t* dst = tile + (r >> 3) * 1024 + (r & 7) * 128 + ((jc ^ (r & 7)) << 4);
          *reinterpret_cast<uint4*>(dst) = i8x8_to_bf16x8(v[l]);
        }
        fence_proxy_async_smem();
        mbar_arrive(&bars->a_full[as]);
        if (++as == SA) { as = 0; aph ^= 1; }
      }
    }
  } else {
    // ---------------------------------------------------------------- epilogue (warps 0-3)
    const int q = p.q;
    double S = 0.0, C = 0.0, A[QMAX];
#pragma unroll
    for (int k = 0; k < QMAX; ++k) A[k] = 0.0;
    bool ok = true;
    for (int nb = 0; nb < p.nblocks; ++nb) {
      const int buf = nb & 1;
      named_bar(1, 128);  // the previous block's constants are no longer read
      for (int e = threadIdx.x; e < (q + 1) * BN; e += 128) {
        const int k = e / BN, i = e % BN, r = nb * BN + i;
        cst[e] = r < p.n ? (k < q ? p.XLw[(int64_t)k * p.n + r] : p.rw[r]) : 0.f;
      }
      named_bar(1, 128);
      if (ok) ok = mbar_wait(&bars->acc_full[buf], (nb >> 1) & 1, abort, tflag, WAIT_NS);
      if (!ok) continue;
      tc_fence_after();
      const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16) + buf * BN;
      for (int c = 0; c < BN / 32; ++c) {
        float v[32];
        tmem_ld32(base + 32 * c, v);
        float ss = 0.f, cc = 0.f, aa[QMAX];
#pragma unroll
        for (int k = 0; k < QMAX; ++k) aa[k] = 0.f;
        const float* cr = cst + 32 * c;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float x = v[i];
          ss = fmaf(x, x, ss);
          cc = fmaf(cr[q * BN + i], x, cc);
#pragma unroll
          for (int k = 0; k < QMAX; ++k)
            if (k < q) aa[k] = fmaf(cr[k * BN + i], x, aa[k]);
        }
        S += ss;
        C += cc;
#pragma unroll
        for (int k = 0; k < QMAX; ++k) A[k] += aa[k];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->acc_empty[buf]);
    }
    const int64_t snp = s0 + 32 * warp + lane;
    if (ok && snp < p.m) {
      double v[QMAX], aPa = 0.0;
#pragma unroll
      for (int k = 0; k < QMAX; ++k) {
        double acc = 0.0;
        if (k < q) {
#pragma unroll
          for (int l = 0; l < QMAX; ++l)
            if (l < q) acc += p.P[k * q + l] * A[l];
          aPa += A[k] * acc;
        }
        v[k] = acc;
      }
      const double sigma = S - aPa;
      const int pp = q + 1;
      float* Bo = p.B + (snp * p.t + p.j) * pp;
      if (sigma > 1e-5 * S) {
        const double bs = C / sigma;
#pragma unroll
        for (int k = 0; k < QMAX; ++k)
          if (k < q) Bo[k] = (float)(p.b0[k] - v[k] * bs);
        Bo[q] = (float)bs;
        if (p.W) p.W[snp * p.t + p.j] = (float)(bs * C);
      } else {
        for (int k = 0; k < pp; ++k) Bo[k] = __int_as_float(0x7fc00000);
        if (p.W) p.W[snp * p.t + p.j] = __int_as_float(0x7fc00000);
        atomicAdd(&p.flags[FLAG_SINGULAR], 1);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 5) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

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

// 2-D BF16 row-major matrix [rows][cols] (cols * 2 bytes a multiple of 16), box 64 x box_rows,
// 128-byte swizzle.
CUtensorMap make_map_bf16(const void* base, int64_t rows, int64_t cols, int box_rows) {
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

}  // namespace

struct TcState {
  int algo = 0, n = 0, q = 0, t = 0;
  int kpad = 0, rpad = 0;
  std::vector<void*> allocs;
  // CHOL: per trait
  std::vector<CUtensorMap> lmaps;
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
    const int n = a.n, q = a.q, t = a.t;
    st->kpad = (int)round_up(n, BK);
    st->rpad = (int)round_up(n, BN);
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
      st->lmaps.push_back(make_map_bf16(hi, 2 * (int64_t)st->rpad, st->kpad, BN));
    }
    GW_CUDA(cudaFuncSetAttribute(chol_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)SMEM_BYTES));
    return st;
  } catch (...) {
    tc_destroy(st);
    throw;
  }
}

void tc_scan(cudaStream_t s, TcState* st, const TcScanArgs& a) {
  if (a.m <= 0) return;
  GW_REQUIRE(st != nullptr, GWAS_ERR_ARG, "no tensor-core state");
  const int64_t tiles = (a.m + BM - 1) / BM;
  GW_REQUIRE(tiles <= 0x7fffffff, GWAS_ERR_ARG, "block too large");
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
    p.nblocks = st->rpad / BN;
    p.XLw = st->XLw32 + (size_t)j * st->q * st->n;
    p.rw = st->rw32 + (size_t)j * st->n;
    p.P = st->P + (size_t)j * st->q * st->q;
    p.b0 = st->b0 + (size_t)j * st->q;
    p.B = a.B;
    p.W = a.wald;
    p.flags = a.flags;
    p.aligned8 = (st->n % 8 == 0) && ((uintptr_t)a.XR % 8 == 0);
    chol_tc_kernel<<<(unsigned)tiles, NUM_THREADS, SMEM_BYTES, s>>>(st->lmaps[j], p);
    GW_CHECK_LAUNCH();
  }
}

void tc_destroy(TcState* st) {
  if (!st) return;
  for (void* p : st->allocs) cudaFree(p);
  delete st;
}

}  // namespace gw
