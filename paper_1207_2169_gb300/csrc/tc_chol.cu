// CHOL fused whiten-and-reduce on the tensor cores (tcgen05 / TMEM / TMA, sm_103a).
//
// Algorithm 3 lines 4 and 8-11 for one trait.  A persistent CTA walks 128-SNP tiles.  For each
// block of 256 rows of L^-1 it accumulates D[snp][r] = (L^-1 x_snp)_r in TMEM, over only the
// K range c <= r where L^-1 can be nonzero (the aggregated triangular solve of "Sequences of
// GLS'", done as one product with the precomputed inverse).  L^-1 = hi + lo in BF16 pieces and
// genotypes are exact in BF16, so D = X hi^T + X lo^T carries ~16 significant bits of L^-1 with
// FP32 accumulation.  Where a K step lies entirely above the diagonal of the lower 128 rows of a
// block, only the upper 128 rows are multiplied.  The epilogue reduces each finished block
// straight out of TMEM into the bordered-system entries of every SNP,
//     s = x'^T x',   c = r'^T x',   a_k = (L^-1 X_L)_k^T x'     (x' = L^-1 x),
// in FP32 over 32 columns and FP64 across them, and finishes each tile with the Schur-complement
// solve in FP64.  X' = L^-1 X_R is never written to memory.
//
// Warp roles (448 threads):
//   0-3  epilogue: one SNP per thread (TMEM lane 32*warp + lane)
//   4    TMA producers: lane 0 the L^-1 tiles, lane 1 the 2-bit packed genotype slices
//   5    MMA issuer (one elected lane); owns the 512 TMEM columns (two 256-column accumulators)
//   6-13 genotype converters: packed slices (shared memory) -> BF16 tiles in the
//        128-byte-swizzled K-major layout
#include "tc_kernels.cuh"
#include "tc_ptx.cuh"

namespace gw {
using namespace tc;

namespace {

constexpr int BM = CHOL_TC_BM;
constexpr int BN = 256;
constexpr int BK = 64;
constexpr int SA = 4;                   // genotype tile ring
constexpr int SB = 4;                   // L^-1 tile ring (one piece per slot)
constexpr int A_BYTES = BM * BK * 2;    // 16 KB
constexpr int B_BYTES = BN * BK * 2;    // 32 KB
constexpr int QMAX = 7;
constexpr int CST_FLOATS = 4096;  // 16 KB: per-row epilogue constants
constexpr int PR = 8;                   // packed-genotype slice ring
constexpr int PK_BYTES = BM * 16;       // 64 genotypes of 128 SNPs, 2-bit codes: 2 KB
constexpr int NCONV = 8;                // genotype converter warps: 2 threads per row
constexpr int NUM_THREADS = 192 + 32 * NCONV;
constexpr int TMEM_COLS = 512;
constexpr uint64_t WAIT_NS = 4000000000ull;

struct __align__(8) Bars {
  uint64_t a_full[SA], a_empty[SA], b_full[SB], b_empty[SB], pk_full[PR], pk_empty[PR];
  uint64_t acc_full[2], acc_empty[2], done;
  uint32_t tmem_base;
  int abort;
};

constexpr size_t SMEM_BYTES =
    1024 + SA * A_BYTES + SB * B_BYTES + PR * PK_BYTES + CST_FLOATS * 4 + sizeof(Bars);

__device__ __forceinline__ int ksteps(int nb, int kpad) {
  const int k = (nb + 1) * (BN / BK);
  const int kmax = kpad / BK;
  return k < kmax ? k : kmax;
}
// K steps at or beyond this one only meet the upper 128 rows of block nb (the lower rows of
// L^-1 are zero there).
__device__ __forceinline__ int half_from(int nb) { return nb * (BN / BK) + 2; }

// (tile, block, k-step) sequence shared by every role of a CTA.
struct Step {
  int64_t tile;
  int nb, ks;
};
__device__ __forceinline__ void advance(Step& s, int nblocks, int kpad) {
  if (++s.ks < ksteps(s.nb, kpad)) return;
  s.ks = 0;
  if (++s.nb < nblocks) return;
  s.nb = 0;
  s.tile += gridDim.x;
}

// QM: compile-time bound on q (3 or 7), so the epilogue's per-column arrays stay in registers.
template <int QM>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    chol_tc_kernel(const __grid_constant__ CUtensorMap map256,
                   const __grid_constant__ CUtensorMap map128,
                   const __grid_constant__ CUtensorMap mapG, const CholTcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = sA + SA * A_BYTES;
  uint8_t* sP = sB + SB * B_BYTES;
  float* cst = (float*)(sP + PR * PK_BYTES);
  Bars* bars = (Bars*)(cst + CST_FLOATS);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t ntiles = (p.m + BM - 1) / BM;
  const int nblocks = p.rpad / BN;
  int* tflag = p.flags + FLAG_TIMEOUT;

  if (threadIdx.x == 0) {
    for (int i = 0; i < SA; ++i) {
      mbar_init(&bars->a_full[i], NCONV);  // one arrive per converter warp
      mbar_init(&bars->a_empty[i], 1);
    }
    for (int i = 0; i < SB; ++i) {
      mbar_init(&bars->b_full[i], 1);
      mbar_init(&bars->b_empty[i], 1);
    }
    for (int i = 0; i < PR; ++i) {
      mbar_init(&bars->pk_full[i], 1);
      mbar_init(&bars->pk_empty[i], NCONV);
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
  if (warp == 4 && lane == 0) {
    prefetch_tensormap(&map256);
    prefetch_tensormap(&map128);
    prefetch_tensormap(&mapG);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  volatile int* abort = &bars->abort;

  if (warp == 4) {
    // ------------------------------------------------------------ L^-1 tiles via TMA
    if (lane == 0) {
      int bs = 0;
      uint32_t bph = 0;
      for (Step st{blockIdx.x, 0, 0}; st.tile < ntiles; advance(st, nblocks, p.kpad)) {
        const bool half = st.ks >= half_from(st.nb);
        bool ok = true;
        for (int piece = 0; piece < 2; ++piece) {
          ok = mbar_wait(&bars->b_empty[bs], bph ^ 1, abort, tflag, WAIT_NS);
          if (!ok) break;
          const int y = piece * p.rpad + st.nb * BN;
          if (half) {
            mbar_arrive_expect_tx(&bars->b_full[bs], B_BYTES / 2);
            tma_load_2d(sB + bs * B_BYTES + B_BYTES / 2, &map128, &bars->b_full[bs], st.ks * BK,
                        y + BN / 2);
          } else {
            mbar_arrive_expect_tx(&bars->b_full[bs], B_BYTES);
            tma_load_2d(sB + bs * B_BYTES, &map256, &bars->b_full[bs], st.ks * BK, y);
          }
          if (++bs == SB) { bs = 0; bph ^= 1; }
        }
        if (!ok) break;
      }
    } else if (lane == 1) {
      // packed genotype slices (64 genotypes x 128 SNPs, 2 KB) via TMA, in the K-step order the
      // converters consume them; rows past m read as zero
      int ps = 0;
      uint32_t pph = 0;
      for (Step st{blockIdx.x, 0, 0}; st.tile < ntiles; advance(st, nblocks, p.kpad)) {
        if (!mbar_wait(&bars->pk_empty[ps], pph ^ 1, abort, tflag, WAIT_NS)) break;
        mbar_arrive_expect_tx(&bars->pk_full[ps], PK_BYTES);
        tma_load_2d(sP + ps * PK_BYTES, &mapG, &bars->pk_full[ps], st.ks * 16,
                    (int32_t)(st.tile * BM));
        if (++ps == PR) { ps = 0; pph ^= 1; }
      }
    }
  } else if (warp == 5) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int as = 0, bs = 0, buf = 0;
      uint32_t aph = 0, bph = 0, accph = 0;
      bool ok = true;
      const uint32_t id_full = idesc_bf16(BM, BN), id_half = idesc_bf16(BM, BN / 2);
      for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        for (int nb = 0; nb < nblocks && ok; ++nb) {
          ok = mbar_wait(&bars->acc_empty[buf], accph ^ 1, abort, tflag, WAIT_NS);
          if (!ok) break;
          tc_fence_after();
          const uint32_t dt = tmem + buf * BN;
          const int nk = ksteps(nb, p.kpad), hf = half_from(nb);
          for (int ks = 0; ks < nk && ok; ++ks) {
            ok = mbar_wait(&bars->a_full[as], aph, abort, tflag, WAIT_NS);
            if (!ok) break;
            tc_fence_after();
            const uint64_t ad = sw128_desc(sA + as * A_BYTES);
            const bool half = ks >= hf;
            for (int piece = 0; piece < 2; ++piece) {
              ok = mbar_wait(&bars->b_full[bs], bph, abort, tflag, WAIT_NS);
              if (!ok) break;
              tc_fence_after();
              const uint64_t bd = sw128_desc(sB + bs * B_BYTES + (half ? B_BYTES / 2 : 0));
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(half ? dt + BN / 2 : dt, ad + 2 * kk, bd + 2 * kk,
                         half ? id_half : id_full, (ks | piece | kk) != 0);
              mma_commit(&bars->b_empty[bs]);
              if (++bs == SB) { bs = 0; bph ^= 1; }
            }
            mma_commit(&bars->a_empty[as]);
            if (++as == SA) { as = 0; aph ^= 1; }
          }
          if (ok) mma_commit(&bars->acc_full[buf]);
          if (++buf == 2) { buf = 0; accph ^= 1; }
        }
      }
      mma_commit(&bars->done);  // TMEM is released only after every issued MMA retired
      mbar_wait(&bars->done, 0, abort, tflag, WAIT_NS);
    }
  } else if (warp >= 6) {
    // ------------------------------------------------------------ genotype converters
    // Thread ct converts half hh of row r of each K step: packed bytes 8 hh .. 8 hh + 7 (32
    // genotypes) into BF16 chunks 4 hh .. 4 hh + 3 of the row's swizzled 128-byte line.
    const int ct = threadIdx.x - 192;
    const int r = ct >> 1, hh = ct & 1;
    const uint32_t line = (r >> 3) * 1024 + (r & 7) * 128;
    int64_t total = 0;
    {
      int per_tile = 0;
      for (int nb = 0; nb < nblocks; ++nb) per_tile += ksteps(nb, p.kpad);
      const int64_t mine = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
      total = mine * per_tile;
    }
    int as = 0, ps = 0;
    uint32_t aph = 0, pph = 0;
    for (int64_t g = 0; g < total; ++g) {
      // warp-uniform exits: every lane leaves together if any wait gave up
      if (!__all_sync(0xffffffffu, mbar_wait(&bars->pk_full[ps], pph, abort, tflag, WAIT_NS))) break;
      const uint2 w = *reinterpret_cast<const uint2*>(sP + ps * PK_BYTES + r * 16 + hh * 8);
      // the slot is refilled by TMA (async proxy): order these generic reads before it
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->pk_empty[ps]);
      if (++ps == PR) { ps = 0; pph ^= 1; }
      uint4 o[4];
      packed8_to_bf16x32(w, GENO_LO, GENO_HI, o);
      if (!__all_sync(0xffffffffu, mbar_wait(&bars->a_empty[as], aph ^ 1, abort, tflag, WAIT_NS)))
        break;
      uint8_t* dst = sA + as * A_BYTES + line;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int j = 4 * hh + i;
        *reinterpret_cast<uint4*>(dst + ((j ^ (r & 7)) << 4)) = o[i];
      }
      // every lane's writes are ordered before the async proxy, then one arrive per warp
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(&bars->a_full[as]);
      if (++as == SA) { as = 0; aph ^= 1; }
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 0-3)
    const int q = p.q;
    int buf = 0;
    uint32_t accph = 0;
    bool ok = true;
    // Per-row constants [k][row] (k < q: L^-1 X_L columns, k = q: whitened residual).  When all
    // rows fit they are loaded once; otherwise the 256 rows of each block are reloaded.
    const bool resident = (q + 1) * p.rpad <= CST_FLOATS;
    const int cstride = resident ? p.rpad : BN;
    if (resident) {
      for (int e = threadIdx.x; e < (q + 1) * p.rpad; e += 128) {
        const int k = e / p.rpad, r = e % p.rpad;
        cst[e] = r < p.n ? (k < q ? p.XLw[(int64_t)k * p.n + r] : p.rw[r]) : 0.f;
      }
      named_bar(1, 128);
    }
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
      double S = 0.0, C = 0.0, A[QM];
#pragma unroll
      for (int k = 0; k < QM; ++k) A[k] = 0.0;
      for (int nb = 0; nb < nblocks; ++nb) {
        if (!resident) {
          named_bar(1, 128);  // the previous block's constants are no longer read
          for (int e = threadIdx.x; e < (q + 1) * BN; e += 128) {
            const int k = e / BN, i = e % BN, r = nb * BN + i;
            cst[e] = r < p.n ? (k < q ? p.XLw[(int64_t)k * p.n + r] : p.rw[r]) : 0.f;
          }
          named_bar(1, 128);
        }
        const float* cb = resident ? cst + nb * BN : cst;
        if (ok) ok = __all_sync(0xffffffffu, mbar_wait(&bars->acc_full[buf], accph, abort, tflag, WAIT_NS));
        if (ok) {
          tc_fence_after();
          const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16) + buf * BN;
          // FP32 over the block's 256 rows (two levels: 32-row chunks, then chunks), FP64 over
          // blocks.
          float bs_ = 0.f, bc = 0.f, ba[QM];
#pragma unroll
          for (int k = 0; k < QM; ++k) ba[k] = 0.f;
          uint32_t ra[32];
          auto chunk = [&](const uint32_t (&r)[32], int c) {
            float ss = 0.f, cc = 0.f, aa[QM];
#pragma unroll
            for (int k = 0; k < QM; ++k) aa[k] = 0.f;
            const float* cr = cb + 32 * c;
#pragma unroll
            for (int i4 = 0; i4 < 8; ++i4) {
              const float4 cv = *reinterpret_cast<const float4*>(cr + q * cstride + 4 * i4);
              float4 av[QM];
#pragma unroll
              for (int k = 0; k < QM; ++k)
                if (k < q) av[k] = *reinterpret_cast<const float4*>(cr + k * cstride + 4 * i4);
              const float x[4] = {__uint_as_float(r[4 * i4]), __uint_as_float(r[4 * i4 + 1]),
                                  __uint_as_float(r[4 * i4 + 2]), __uint_as_float(r[4 * i4 + 3])};
              const float cw[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                ss = fmaf(x[e], x[e], ss);
                cc = fmaf(cw[e], x[e], cc);
#pragma unroll
                for (int k = 0; k < QM; ++k) {
                  if (k < q) {
                    const float w = e == 0 ? av[k].x : e == 1 ? av[k].y : e == 2 ? av[k].z : av[k].w;
                    aa[k] = fmaf(w, x[e], aa[k]);
                  }
                }
              }
            }
            bs_ += ss;
            bc += cc;
#pragma unroll
            for (int k = 0; k < QM; ++k) ba[k] += aa[k];
          };
          // one 32-column TMEM load at a time: the epilogue has slack, and its registers go to
          // the eight converter warps (448 threads leave 128 registers per thread)
#pragma unroll 1
          for (int c = 0; c < BN / 32; ++c) {
            tmem_ld32_async(base + 32 * c, ra);
            tmem_wait32(ra);
            chunk(ra, c);
          }
          S += bs_;
          C += bc;
#pragma unroll
          for (int k = 0; k < QM; ++k) A[k] += ba[k];
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bars->acc_empty[buf]);
        }
        if (++buf == 2) { buf = 0; accph ^= 1; }
      }
      const int64_t snp = tile * BM + 32 * warp + lane;
      if (ok && snp < p.m) {
        double v[QM], aPa = 0.0;
#pragma unroll
        for (int k = 0; k < QM; ++k) {
          double acc = 0.0;
          if (k < q) {
#pragma unroll
            for (int l = 0; l < QM; ++l)
              if (l < q) acc += __ldg(&p.P[k * q + l]) * A[l];
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
          for (int k = 0; k < QM; ++k)
            if (k < q) Bo[k] = (float)(__ldg(&p.b0[k]) - v[k] * bs);
          Bo[q] = (float)bs;
          if (p.W) p.W[snp * p.t + p.j] = (float)(bs * C);
        } else {
          for (int k = 0; k < pp; ++k) Bo[k] = __int_as_float(0x7fc00000);
          if (p.W) p.W[snp * p.t + p.j] = __int_as_float(0x7fc00000);
          atomicAdd(&p.flags[FLAG_SINGULAR], 1);
        }
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

}  // namespace

void chol_tc_prepare() {
  GW_CUDA(cudaFuncSetAttribute(chol_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)SMEM_BYTES));
  GW_CUDA(cudaFuncSetAttribute(chol_tc_kernel<QMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)SMEM_BYTES));
}

void chol_tc_launch(cudaStream_t s, const CUtensorMap& map256, const CUtensorMap& map128,
                    const CUtensorMap& mapG, const CholTcParams& p, int num_sms) {
  if (p.m <= 0) return;
  GW_REQUIRE(p.q >= 1 && p.q <= QMAX, GWAS_ERR_ARG, "q=%d outside [1,%d]", p.q, QMAX);
  const int64_t tiles = (p.m + BM - 1) / BM;
  const unsigned grid = (unsigned)(tiles < num_sms ? tiles : num_sms);
  if (p.q <= 3)
    chol_tc_kernel<3><<<grid, NUM_THREADS, SMEM_BYTES, s>>>(map256, map128, mapG, p);
  else
    chol_tc_kernel<QMAX><<<grid, NUM_THREADS, SMEM_BYTES, s>>>(map256, map128, mapG, p);
  GW_CHECK_LAUNCH();
}

}  // namespace gw
