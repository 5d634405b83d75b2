// EIG on the tensor cores (tcgen05 / TMEM / TMA, sm_103a): Algorithm 4's per-SNP work.
//
// Per SNP i and trait j the bordered system needs three reductions over the n individuals:
//     a_ij[k] = x_i^T M_j^-1 X_L[:,k],   c_ij = x_i^T M_j^-1 r_j,   s_ij = x_i^T M_j^-1 x_i,
// with r_j = y_j - X_L b0_j the null-model residual.  With Phi = Z W Z^T, M_j^-1 = Z D_j Z^T.
// a and c are linear in the raw genotypes, so they are contracted against the precomputed
// columns U_j = Z D_j Z^T [X_L | r_j] (exact genotype operand, U split hi + lo: 2 products);
// s needs the eigenbasis: s_ij = sum_r (Z^T x_i)_r^2 d_j[r].  Three kernels share one template:
//   ROT  Xsq = (Z^T X_R)^2, written as hi + lo BF16 planes  (A: genotypes, B: Z^T split)
//   SQ   s_ij = Xsq_i . d_j                                  (A: Xsq split, B: d split, 3 products)
//   AC   a, c from the genotypes, then the Schur-complement solve in FP32 with s_ij
//                                                            (A: genotypes, B: U split)
// A persistent CTA walks (128-SNP tile, 256-column block) work items, eight SNP tiles per
// column block at a time so that both operands are reused from L2.
//
// Warp roles (448 threads): 0-3 epilogue (one SNP per TMEM lane), 11 TMA producers (lane 0: the
// B operand and SQ's A operand; lane 1: 2-bit packed genotype slices for ROT and AC), 7 MMA
// issuer and TMEM owner (two 256-column FP32 accumulators), 4-6, 8-10, 12-13 genotype converters
// (packed slices in shared memory -> centred BF16 tiles; ROT and AC).
#include <mutex>

#include "tc_kernels.cuh"
#include "tc_ptx.cuh"

namespace gw {
using namespace tc;

namespace {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 64;
constexpr int SA_MAX = 6;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int NCONV = 8;                 // genotype converter warps (ROT, AC): 2 threads per row
// Warp roles.  A warp issues on SMSP (warp % 4) and may read only TMEM lanes 32 (warp % 4) ..
// +31.  The single-thread MMA issuer (7) and TMA producers (11) share SMSP 3 with epilogue warps
// only, so converter bursts never delay their issue.  ROT and SQ: 14 warps, epilogue 0-3,
// converters 4-6, 8-10, 12-13.  AC is epilogue-bound: 20 warps in five warpgroups, epilogue
// warps 0-3 and 12-15 (each set takes half of a work item's traits), converters 4-6, 8-10,
// 16-17, warps 18-19 idle.
constexpr int MMA_WARP = 7;
constexpr int TMA_WARP = 11;

enum { EPI_ROT = 0, EPI_SQ = 1, EPI_AC = 2 };
// the 20-warp layout: AC with q <= 3 (larger q would need more staging memory than fits)
__host__ __device__ constexpr bool wide_of(int epi, int qq) { return epi == EPI_AC && qq <= 3; }
__host__ __device__ constexpr int nwarps_of(int epi, int qq) { return wide_of(epi, qq) ? 20 : 14; }
__host__ __device__ constexpr int nepi_of(int epi, int qq) { return wide_of(epi, qq) ? 8 : 4; }
// A-tile ring depth.  SQ reads its A tiles (the squared planes, rows 2 KB apart) by TMA, mostly
// from DRAM: six slots (three K steps of hi + lo) keep more of them in flight than four (the
// SQ kernel 9 % faster); its shared memory has room, having no packed-slice ring.
__host__ __device__ constexpr int sa_of(int epi, int qq) {
  return wide_of(epi, qq) ? 3 : epi == EPI_SQ ? 6 : 4;
}
// converter warps -> 0 .. 7
template <bool WIDE>
__device__ __forceinline__ int conv_index(int warp) {
  return warp < MMA_WARP ? warp - 4 : warp < TMA_WARP ? warp - 5 : (WIDE ? warp - 10 : warp - 6);
}
template <bool WIDE>
__device__ __forceinline__ bool is_epilogue(int warp) {
  return warp < 4 || (WIDE && warp >= 12 && warp < 16);
}
template <bool WIDE>
__device__ __forceinline__ bool is_idle(int warp) {
  return WIDE && warp >= 18;
}
constexpr int PR = 8;                    // packed-genotype slice ring
constexpr int PK_BYTES = BM * 16;        // 64 genotypes of 128 SNPs, 2-bit codes: 2 KB
constexpr int TMEM_COLS = 512;
constexpr int GROUP_M = 8;
constexpr int QMAX = 7;
constexpr uint64_t WAIT_NS = 4000000000ull;

// B-tile ring depth: AC gives one slot to the shared memory that stages its output rows.
__host__ __device__ constexpr int sb_of(int epi) { return epi == EPI_AC ? 3 : 4; }
// AC is compiled per q (QQ = q, 1..7); ROT and SQ use QQ = 0.  QP = TMEM columns loaded per
// trait (q + 1 rounded up to 4 or 8).
__host__ __device__ constexpr int qp_of(int qq) { return qq + 1 <= 4 ? 4 : 8; }
// AC staging row stride in floats: 8 traits x (q + 1) coefficients.  For q = 3 each trait is one
// float4 and rows are 36 floats (16-byte aligned, conflict-free float4 access); otherwise rows
// are 8 QP + 1 floats (odd: conflict-free scalar access).
__host__ __device__ constexpr int stg_rb(int qq) { return qq == 3 ? 36 : 8 * qp_of(qq) + 1; }
// AC shared floats: P_j, b0_j of a block (<= 2048), then per epilogue warp (eight) a staging
// area of 32 rows of coefficients and 32 x 9 Wald values.
__host__ __device__ constexpr int stg_b(int qq) { return 32 * stg_rb(qq); }
constexpr int STG_W = 32 * 9;
constexpr int PB_FLOATS = 2048;
// q = 3: the 64 traits of a block fill the accumulator (the epilogue loads 8 of them at once)
static_assert(eig_ac_traits(3) * 4 == BN, "AC block of q = 3 is not one accumulator");
__host__ __device__ constexpr int cst_of(int epi, int qq) {
  return epi == EPI_AC ? PB_FLOATS + nepi_of(epi, qq) * (stg_b(qq) + STG_W) : 0;
}

template <int NSB>
struct __align__(8) BarsT {
  uint64_t a_full[SA_MAX], a_empty[SA_MAX], b_full[NSB], b_empty[NSB], pk_full[PR], pk_empty[PR];
  uint64_t acc_full[2], acc_empty[2], done;
  uint32_t tmem_base;
  int abort;
};

__host__ __device__ constexpr size_t smem_of(int epi, int qp) {
  return 1024 + (size_t)sa_of(epi, qp) * A_BYTES + (size_t)sb_of(epi) * B_BYTES + (epi == EPI_SQ ? 0 : PR * PK_BYTES) +
         (size_t)cst_of(epi, qp) * 4 + sizeof(BarsT<4>);
}

__device__ __forceinline__ void work_coords(int64_t w, int64_t mtiles, int nblk, int64_t& tile,
                                            int& nb) {
  const int64_t per_group = (int64_t)GROUP_M * nblk;
  const int64_t g = w / per_group;
  const int64_t r = w % per_group;
  const int64_t first = g * GROUP_M;
  const int64_t rows = mtiles - first < GROUP_M ? mtiles - first : GROUP_M;
  nb = (int)(r / rows);
  tile = first + r % rows;
}

// With GP = 2 working columns per SNP (a two-column genetic model) a ROT or AC tile holds 64
// SNPs: A row r is column (r / 16) % 2 of SNP (r / 32) 16 + r % 16, so that a SNP's two rows sit in
// lanes l and l + 16 of one epilogue warp.
template <int GP>
__device__ __forceinline__ int row_snp(int r) { return GP == 1 ? r : (r >> 5) * 16 + (r & 15); }
template <int GP>
__device__ __forceinline__ int row_col(int r) { return GP == 1 ? 0 : (r >> 4) & 1; }

// The bordered solve of one (SNP, trait) pair with a two-column genetic block, in FP32 (Algorithm
// 4's per-pair solve in the model's working basis): a0, a1 = (a_k, c) of the two centred working
// columns, S00, S01, S11 their s entries, Pj = P_j (q x q) then b0_j (q).  V = P [a0 a1],
// Sigma = S_RR - [a0 a1]^T V, b_w = Sigma^-1 c, b_L = b0 - V b_w (the intercept absorbing
// mu . b_w), wald = b_w . c; reported b_R = tm b_w, Var = R Var_c R^T as in the CHOL kernel's
// pair solve.  Returns 1 for a singular pair (a pivot of Sigma's Cholesky at most 1e-5 of the
// matching S_kk: NaN outputs), else 0.  Writes the pair's row of B (and W) directly.
template <int QQ>
__device__ __noinline__ int ac_pair(const EigTcParams& p, const float* Pj, const float* a0,
                                    const float* a1, float S00, float S01, float S11, float m0,
                                    float m1, int64_t snp, int j) {
  constexpr int P2 = QQ + 2;
  float v[2][QQ > 0 ? QQ : 1];
#pragma unroll
  for (int k = 0; k < QQ; ++k) {
    float x0 = 0.f, x1 = 0.f;
#pragma unroll
    for (int l = 0; l < QQ; ++l) {
      x0 = fmaf(Pj[k * QQ + l], a0[l], x0);
      x1 = fmaf(Pj[k * QQ + l], a1[l], x1);
    }
    v[0][k] = x0;
    v[1][k] = x1;
  }
  float g00 = S00, g01 = S01, g11 = S11;
#pragma unroll
  for (int k = 0; k < QQ; ++k) {
    g00 = fmaf(-a0[k], v[0][k], g00);
    g01 = fmaf(-a0[k], v[1][k], g01);
    g11 = fmaf(-a1[k], v[1][k], g11);
  }
  const float piv1 = g11 - g01 * g01 / g00;
  const bool ok = g00 > 1e-5f * S00 && piv1 > 1e-5f * S11;
  const int pw = p.out_snp ? 4 : p.out_var ? P2 + P2 * (P2 + 1) / 2 : P2;
  float* Bo = p.B + (snp * p.t + j) * pw;
  const float nanv = __int_as_float(0x7fc00000);
  if (!ok) {
    for (int k = 0; k < pw; ++k) Bo[k] = nanv;
    if (p.W) p.W[snp * p.t + j] = nanv;
    return 1;
  }
  const float det = g00 * piv1;
  const float si[2][2] = {{g11 / det, -g01 / det}, {-g01 / det, g00 / det}};
  const float c0 = a0[QQ], c1 = a1[QQ];
  const float bw[2] = {si[0][0] * c0 + si[0][1] * c1, si[1][0] * c0 + si[1][1] * c1};
  const float mu[2] = {p.mu ? m0 : 0.f, p.mu ? m1 : 0.f};
  const float tm[2][2] = {{p.tm[0], p.tm[1]}, {p.tm[2], p.tm[3]}};
  if (p.W) p.W[snp * p.t + j] = bw[0] * c0 + bw[1] * c1;
  const float bR[2] = {tm[0][0] * bw[0] + tm[0][1] * bw[1], tm[1][0] * bw[0] + tm[1][1] * bw[1]};
  float vr[2][2];
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float x = 0.f;
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int z = 0; z < 2; ++z) x += tm[g][u] * si[u][z] * tm[h][z];
      vr[g][h] = x;
    }
  if (p.out_snp) {
    Bo[0] = bR[0];
    Bo[1] = bR[1];
    Bo[2] = sqrtf(vr[0][0]);
    Bo[3] = sqrtf(vr[1][1]);
    return 0;
  }
#pragma unroll
  for (int k = 0; k < QQ; ++k) {
    float b = Pj[QQ * QQ + k] - v[0][k] * bw[0] - v[1][k] * bw[1];
    if (k == 0) b -= mu[0] * bw[0] + mu[1] * bw[1];
    Bo[k] = b;
  }
  Bo[QQ] = bR[0];
  Bo[QQ + 1] = bR[1];
  if (!p.out_var) return 0;
  auto vc = [&](int r, int c) -> float {
    if (r >= QQ && c >= QQ) return si[r - QQ][c - QQ];
    if (c >= QQ) return -(v[0][r] * si[0][c - QQ] + v[1][r] * si[1][c - QQ]);
    if (r >= QQ) return -(v[0][c] * si[0][r - QQ] + v[1][c] * si[1][r - QQ]);
    float x = Pj[r * QQ + c];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int z = 0; z < 2; ++z) x += v[u][r] * si[u][z] * v[z][c];
    return x;
  };
  auto rterms = [&](int r, int* idx, float* cf) -> int {
    if (r >= QQ) {
      idx[0] = QQ; cf[0] = tm[r - QQ][0];
      idx[1] = QQ + 1; cf[1] = tm[r - QQ][1];
      return 2;
    }
    idx[0] = r; cf[0] = 1.f;
    if (r != 0) return 1;
    idx[1] = QQ; cf[1] = -mu[0];
    idx[2] = QQ + 1; cf[2] = -mu[1];
    return 3;
  };
  for (int r = 0; r < P2; ++r)
    for (int c = r; c < P2; ++c) {
      int ir[3], ic[3];
      float fr[3], fc[3];
      const int nr = rterms(r, ir, fr), nc = rterms(c, ic, fc);
      float x = 0.f;
      for (int u = 0; u < nr; ++u)
        for (int z = 0; z < nc; ++z) x += fr[u] * fc[z] * vc(ir[u], ic[z]);
      Bo[P2 + r * P2 - r * (r - 1) / 2 + (c - r)] = x;
    }
  return 0;
}

// 4 or 8 consecutive FP32 TMEM columns of this warp's lanes (no wait).
template <int QP>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, uint32_t (&r)[QP]);
template <>
__device__ __forceinline__ void tmem_ld_cols<4>(uint32_t taddr, uint32_t (&r)[4]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}
template <>
__device__ __forceinline__ void tmem_ld_cols<8>(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

// VAR (AC only): the epilogue writes b and the packed Var(b) per pair (GWAS_OUT_VAR), compiled
// apart so that the other output modes keep their register allocation.
// NP: BF16 pieces of the B operand of ROT and AC (2, or 3 for AC when some M_j is badly
// conditioned); a compile-time bound keeps the producer's and issuer's piece loops unrolled.
template <int EPI, int QQ, bool VAR = false, int GP = 1, int NP = 2>
__global__ void __launch_bounds__(32 * nwarps_of(EPI, QQ), 1)
    eig_tc_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                  const __grid_constant__ CUtensorMap mapG, const EigTcParams p) {
  // rows of a tile are SNPs (SQ: rows of the squared planes); ROT and AC with GP = 2 hold 64 SNPs
  constexpr int TS = EPI == EPI_SQ ? BM : BM / GP;
  constexpr int PKB = TS * 16;  // bytes of one packed slice (64 genotypes of TS SNPs)
  constexpr int QP = qp_of(QQ);
  constexpr bool CONV = EPI != EPI_SQ;  // A operand = genotypes through the converters
  constexpr int SB = sb_of(EPI);
  constexpr bool WIDE = wide_of(EPI, QQ);
  constexpr int SA = sa_of(EPI, QQ);
  constexpr int NEPI = nepi_of(EPI, QQ);
  using Bars = BarsT<SB>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = sA + SA * A_BYTES;
  uint8_t* sP = sB + SB * B_BYTES;
  float* cst = (float*)(sP + (CONV ? PR * PK_BYTES : 0));
  Bars* bars = (Bars*)(cst + cst_of(EPI, QQ));
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t mtiles = (p.m + TS - 1) / TS;
  const int64_t nwork = mtiles * p.nblk;
  const int nk = p.kpad / BK;
  int* tflag = p.flags + FLAG_TIMEOUT;

  if (threadIdx.x == 0) {
    for (int i = 0; i < SA; ++i) {
      mbar_init(&bars->a_full[i], CONV ? NCONV : 1);  // converters: one arrive per warp
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
      mbar_init(&bars->acc_empty[i], NEPI);
    }
    mbar_init(&bars->done, 1);
    bars->abort = 0;
    fence_mbar_init();
  }
  if (warp == MMA_WARP) {
    tmem_alloc(&bars->tmem_base, TMEM_COLS);
    tmem_relinquish();
  }
  if (warp == TMA_WARP && lane == 0) {
    if (!CONV) prefetch_tensormap(&mapA);
    if (CONV) prefetch_tensormap(&mapG);
    prefetch_tensormap(&mapB);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  volatile int* abort = &bars->abort;

  if (warp == TMA_WARP) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int as = 0, bs = 0;
      uint32_t aph = 0, bph = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
        int64_t tile;
        int nb;
        work_coords(w, mtiles, p.nblk, tile, nb);
        for (int ks = 0; ks < nk && ok; ++ks) {
          if (!CONV) {
            for (int piece = 0; piece < 2 && ok; ++piece) {
              ok = mbar_wait(&bars->a_empty[as], aph ^ 1, abort, tflag, WAIT_NS);
              if (!ok) break;
              mbar_arrive_expect_tx(&bars->a_full[as], A_BYTES);
              tma_load_2d(sA + as * A_BYTES, &mapA, &bars->a_full[as], ks * BK,
                          (int32_t)(piece * p.a_piece_rows + tile * BM));
              if (++as == SA) { as = 0; aph ^= 1; }
            }
          }
          // B pieces: ROT and AC NP against the exact genotype operand; SQ hi, lo
          constexpr int NBP = CONV ? NP : 2;
          for (int piece = 0; piece < NBP && ok; ++piece) {
            ok = mbar_wait(&bars->b_empty[bs], bph ^ 1, abort, tflag, WAIT_NS);
            if (!ok) break;
            mbar_arrive_expect_tx(&bars->b_full[bs], B_BYTES);
            tma_load_2d(sB + bs * B_BYTES, &mapB, &bars->b_full[bs], ks * BK,
                        piece * p.b_piece_rows + nb * p.b_rows_per_blk);
            if (++bs == SB) { bs = 0; bph ^= 1; }
          }
        }
      }
    } else if (lane == 1 && CONV) {
      // packed genotype slices (64 genotypes x TS SNPs) via TMA, in the order the converters
      // consume them; rows past m read as zero
      int ps = 0;
      uint32_t pph = 0;
      bool ok = true;
      for (int64_t w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
        int64_t tile;
        int nb;
        work_coords(w, mtiles, p.nblk, tile, nb);
        for (int ks = 0; ks < nk; ++ks) {
          ok = mbar_wait(&bars->pk_empty[ps], pph ^ 1, abort, tflag, WAIT_NS);
          if (!ok) break;
          mbar_arrive_expect_tx(&bars->pk_full[ps], PKB);
          tma_load_2d(sP + ps * PK_BYTES, &mapG, &bars->pk_full[ps], ks * 16, (int32_t)(tile * TS));
          if (++ps == PR) { ps = 0; pph ^= 1; }
        }
      }
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int as = 0, bs = 0, buf = 0;
      uint32_t aph = 0, bph = 0, accph = 0;
      bool ok = true;
      const uint32_t idesc = idesc_bf16(BM, BN);
      for (int64_t w = blockIdx.x; w < nwork && ok; w += gridDim.x) {
        ok = mbar_wait(&bars->acc_empty[buf], accph ^ 1, abort, tflag, WAIT_NS);
        if (!ok) break;
        tc_fence_after();
        const uint32_t dt = tmem + buf * BN;
        for (int ks = 0; ks < nk && ok; ++ks) {
          if (CONV) {
            // products (x, U_hi), (x, U_lo) (and (x, U_lo2)) -- the genotype operand is exact
            ok = mbar_wait(&bars->a_full[as], aph, abort, tflag, WAIT_NS);
            if (!ok) break;
            tc_fence_after();
            const uint64_t ad = sw128_desc(sA + as * A_BYTES);
            for (int piece = 0; piece < NP && ok; ++piece) {
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
          } else {
            // products (A_hi, B_hi), (A_lo, B_hi), (A_hi, B_lo)
            const int a0 = as, b0s = bs;
            int a1 = as + 1 == SA ? 0 : as + 1;
            int b1 = bs + 1 == SB ? 0 : bs + 1;
            const uint32_t aph1 = a1 == 0 ? aph ^ 1 : aph, bph1 = b1 == 0 ? bph ^ 1 : bph;
            ok = mbar_wait(&bars->a_full[a0], aph, abort, tflag, WAIT_NS) &&
                 mbar_wait(&bars->a_full[a1], aph1, abort, tflag, WAIT_NS) &&
                 mbar_wait(&bars->b_full[b0s], bph, abort, tflag, WAIT_NS);
            if (!ok) break;
            tc_fence_after();
            const uint64_t ah = sw128_desc(sA + a0 * A_BYTES), al = sw128_desc(sA + a1 * A_BYTES);
            const uint64_t bh = sw128_desc(sB + b0s * B_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              mma_bf16(dt, ah + 2 * kk, bh + 2 * kk, idesc, (ks | kk) != 0);
              mma_bf16(dt, al + 2 * kk, bh + 2 * kk, idesc, 1u);
            }
            mma_commit(&bars->b_empty[b0s]);
            ok = mbar_wait(&bars->b_full[b1], bph1, abort, tflag, WAIT_NS);
            if (!ok) break;
            tc_fence_after();
            const uint64_t bl = sw128_desc(sB + b1 * B_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) mma_bf16(dt, ah + 2 * kk, bl + 2 * kk, idesc, 1u);
            mma_commit(&bars->b_empty[b1]);
            mma_commit(&bars->a_empty[a0]);
            mma_commit(&bars->a_empty[a1]);
            as = a1 + 1 == SA ? 0 : a1 + 1;
            if (as == 0 || a1 == 0) aph ^= 1;
            bs = b1 + 1 == SB ? 0 : b1 + 1;
            if (bs == 0 || b1 == 0) bph ^= 1;
          }
        }
        if (ok) mma_commit(&bars->acc_full[buf]);
        if (++buf == 2) { buf = 0; accph ^= 1; }
      }
      mma_commit(&bars->done);
      mbar_wait(&bars->done, 0, abort, tflag, WAIT_NS);
    }
  } else if (!is_epilogue<WIDE>(warp) && !is_idle<WIDE>(warp)) {
    // ------------------------------------------------------------ genotype converters
    // Thread ct converts half hh of row r of each K step: packed bytes 8 hh .. 8 hh + 7 (32
    // genotypes) into BF16 chunks 4 hh .. 4 hh + 3 of the row's swizzled 128-byte line, through
    // the row's byte tables of g - mu (mu = 0 without centring).  Codes past n are 0 and map to
    // -mu; the B operand is zero there, so they add nothing.
    if (CONV) {
      const int ct = conv_index<WIDE>(warp) * 32 + lane;
      const int r = ct >> 1, hh = ct & 1;
      const int srow = row_snp<GP>(r), gk = row_col<GP>(r);  // the row's SNP and working column
      const uint32_t line = (r >> 3) * 1024 + (r & 7) * 128;
      const int64_t mine = blockIdx.x < nwork ? (nwork - 1 - blockIdx.x) / gridDim.x + 1 : 0;
      int as = 0, ps = 0;
      uint32_t aph = 0, pph = 0, lutlo = 0, luthi = 0;
      int64_t cur_tile = -1;
      bool ok = true;
      for (int64_t i = 0; i < mine && ok; ++i) {
        int64_t tile;
        int nb;
        work_coords(blockIdx.x + i * gridDim.x, mtiles, p.nblk, tile, nb);
        if (tile != cur_tile) {
          cur_tile = tile;
          const int64_t snp = tile * TS + srow;
          coded_lut(p.mu && snp < p.m ? p.mu[snp * GP + gk] : 0.f, p.code[gk], lutlo, luthi);
        }
        for (int ks = 0; ks < nk; ++ks) {
          // warp-uniform exits: every lane leaves together if any wait gave up
          ok = __all_sync(0xffffffffu, mbar_wait(&bars->pk_full[ps], pph, abort, tflag, WAIT_NS));
          if (!ok) break;
          const uint2 w = *reinterpret_cast<const uint2*>(sP + ps * PK_BYTES + srow * 16 + hh * 8);
          // the slot is refilled by TMA (async proxy): order these generic reads before it
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bars->pk_empty[ps]);
          if (++ps == PR) { ps = 0; pph ^= 1; }
          uint4 o[4];
          packed8_to_bf16x32(w, lutlo, luthi, o);
          ok = __all_sync(0xffffffffu, mbar_wait(&bars->a_empty[as], aph ^ 1, abort, tflag, WAIT_NS));
          if (!ok) break;
          uint8_t* dst = sA + as * A_BYTES + line;
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = 4 * hh + u;
            *reinterpret_cast<uint4*>(dst + ((j ^ (r & 7)) << 4)) = o[u];
          }
          // every lane's writes are ordered before the async proxy, then one arrive per warp
          fence_proxy_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bars->a_full[as]);
          if (++as == SA) { as = 0; aph ^= 1; }
        }
      }
    }
  } else if (is_epilogue<WIDE>(warp)) {
    // ------------------------------------------------------------ epilogue
    // ew: epilogue warp 0 .. NEPI-1; it reads TMEM lanes (SNPs) 32 qd .. 32 qd + 31 and, in AC,
    // the trait batches of its set (the two warpgroups take alternate batches of 8 traits)
    const int ew = warp < 4 ? warp : warp - 8, qd = warp & 3, set = ew >> 2;
    constexpr int NSETS = NEPI / 4;
    int buf = 0;
    uint32_t accph = 0;
    bool ok = true;
    // AC is compiled for one q, so the Schur loops below are fully unrolled
    const int q = EPI == EPI_AC ? QQ : p.q, q1 = q + 1;
    // AC constants of trait block nb, flattened: per trait P_j (q x q) then b0_j (q); 0 past t
    constexpr int ET = 32 * NEPI;  // epilogue threads
    constexpr int PF_REGS = (eig_ac_traits(QQ > 0 ? QQ : 1) * (QQ * QQ + QQ) + ET - 1) / ET;
    static_assert(PF_REGS * ET <= PB_FLOATS, "AC constants exceed their shared-memory area");
    const int et = 32 * ew + lane;
    float pf[EPI == EPI_AC ? PF_REGS : 1];
    bool have_pf = false;
    auto const_at = [&](int nbk, int e) -> float {
      const int per = q * q + q;
      const int jl = e / per, u = e - jl * per, j = nbk * p.traits_per_blk + jl;
      if (jl >= p.traits_per_blk || j >= p.t) return 0.f;
      return u < q * q ? __ldg(&p.P[(int64_t)j * q * q + u]) : __ldg(&p.b0[(int64_t)j * q + u - q * q]);
    };
    for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
      int64_t tile;
      int nb;
      work_coords(w, mtiles, p.nblk, tile, nb);
      // this lane's row: working column egk of SNP snp (GP = 1: the SNP of TMEM lane 32 qd + lane)
      const int erow = 32 * qd + lane, egk = row_col<GP>(erow);
      const int64_t snp = tile * TS + row_snp<GP>(erow);
      const float mu_snp = (p.mu && snp < p.m) ? p.mu[snp * GP + egk] : 0.f;
      if (EPI == EPI_AC) {
        // P_j and b0_j of this block's traits, FP32, into shared memory: from the registers
        // loaded during the previous work item, then the next item's are loaded (their global
        // latency hides behind this item)
        named_bar(1, ET);
        if (have_pf) {
#pragma unroll
          for (int i = 0; i < PF_REGS; ++i) cst[et + ET * i] = pf[i];
        } else {
#pragma unroll
          for (int i = 0; i < PF_REGS; ++i) cst[et + ET * i] = const_at(nb, et + ET * i);
        }
        named_bar(1, ET);
        const int64_t wn = w + gridDim.x;
        have_pf = wn < nwork;
        if (have_pf) {
          int64_t tn;
          int nbn;
          work_coords(wn, mtiles, p.nblk, tn, nbn);
#pragma unroll
          for (int i = 0; i < PF_REGS; ++i) pf[i] = const_at(nbn, et + ET * i);
        }
      }
      if (ok) ok = __all_sync(0xffffffffu, mbar_wait(&bars->acc_full[buf], accph, abort, tflag, WAIT_NS));
      if (ok) {
        tc_fence_after();
        const uint32_t base = tmem + ((uint32_t)(32 * qd) << 16) + buf * BN;
        if (EPI == EPI_ROT) {
          // 32 products of rotated values, split into NP BF16 pieces (each the rounding of what
          // the previous leave), into row `row` of each piece's planes
          auto store_split = [&](int64_t row, int col0, const float* x, const float* y) {
            float rem[32];
#pragma unroll
            for (int i = 0; i < 32; ++i) rem[i] = x[i] * y[i];
#pragma unroll
            for (int pc = 0; pc < NP; ++pc) {
              uint32_t pk[16];
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                const __nv_bfloat16 h0 = __float2bfloat16_rn(rem[2 * i]);
                const __nv_bfloat16 h1 = __float2bfloat16_rn(rem[2 * i + 1]);
                rem[2 * i] -= __bfloat162float(h0);
                rem[2 * i + 1] -= __bfloat162float(h1);
                pk[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
              }
              uint4* dst = reinterpret_cast<uint4*>(p.xsq + (pc * p.a_piece_rows + row) * p.kpad + col0);
#pragma unroll
              for (int u = 0; u < 4; ++u)
                dst[u] = make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
            }
          };
          for (int c = 0; c < BN / 32; ++c) {
            float v[32];
            tmem_ld32(base + 32 * c, v);
            const int col0 = nb * BN + 32 * c;
            if (GP == 2) {
              // three planes per SNP (stride xplane rows): (Z^T g0)^2, (Z^T g0)(Z^T g1),
              // (Z^T g1)^2; the partner row (the SNP's other working column) is 16 lanes away
              float w2[32];
#pragma unroll
              for (int i = 0; i < 32; ++i) w2[i] = __shfl_xor_sync(0xffffffffu, v[i], 16);
              if (snp < p.m && col0 < p.kpad) {
                if (egk == 0) {
                  store_split(snp, col0, v, v);
                  store_split(p.xplane + snp, col0, v, w2);
                } else {
                  store_split(2 * p.xplane + snp, col0, v, v);
                }
              }
            } else if (snp < p.m && col0 < p.kpad) {
              store_split(snp, col0, v, v);
            }
          }
        } else if (EPI == EPI_SQ) {
          for (int c = 0; c < BN / 32; ++c) {
            float v[32];
            tmem_ld32(base + 32 * c, v);
            if (snp < p.m) {
#pragma unroll
              for (int i = 0; i < 32; ++i) {
                const int j = nb * BN + 32 * c + i;
                if (j < p.t) p.sbuf[(int64_t)j * p.lds + snp] = v[i];
              }
            }
          }
        } else {
          // Per batch of 8 traits: TMEM -> (a, c), s from the SQ pass (loaded one batch ahead,
          // read-only path), FP32 Schur solve, results staged per warp in shared memory and
          // written row by row so every store is contiguous within one SNP's output.
          const int T = p.traits_per_blk;
          const int j0 = nb * T;
          const int jend = (j0 + T < p.t ? j0 + T : p.t);
          float* stgB = cst + PB_FLOATS + ew * (stg_b(QQ) + STG_W);
          float* stgW = stgB + stg_b(QQ);
          constexpr int RB = stg_rb(QQ);
          const bool live = snp < p.m;
          constexpr int STEP = 8 * NSETS;  // this warp's batches: 8 set, 8 set + STEP, ...
          float snext[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int j = j0 + 8 * set + u;
            snext[u] = (live && j < jend) ? __ldg(&p.sbuf[(int64_t)j * p.lds + snp]) : 1.f;
          }
          int nsing = 0;
          bool released = false;
          const int64_t row0 = tile * BM + 32 * qd;
          // GP = 2: the centre of the SNP's second working column (held by the partner lane)
          const float mu_pair = __shfl_down_sync(0xffffffffu, mu_snp, 16);
          for (int j8 = 8 * set; j8 < T; j8 += STEP) {
            float scur[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) scur[u] = snext[u];
            if (j8 + STEP < T) {
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int j = j0 + j8 + STEP + u;
                snext[u] = (live && j < jend) ? __ldg(&p.sbuf[(int64_t)j * p.lds + snp]) : 1.f;
              }
            }
            uint32_t r[8][QP];
            if (QQ == 3) {
              // q + 1 = 4 columns per trait: the batch's 32 columns are contiguous, one load
              // (T = 64, so the batch ends at column 4 (j8 + 8) <= 256 of the accumulator)
              tmem_ld32_async(base + j8 * 4, *reinterpret_cast<uint32_t(*)[32]>(&r[0][0]));
            } else {
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                // columns of traits past the block end are not read (their loads would leave the
                // accumulator); those lanes of r are unused
                const int jl = j8 + u < T ? j8 + u : 0;
                tmem_ld_cols<QP>(base + jl * q1, r[u]);
              }
            }
            // the wait names every destination register, so no use is scheduled before it
#pragma unroll
            for (int h = 0; h < QP / 4; ++h)
              tmem_wait32(*reinterpret_cast<uint32_t(*)[32]>(&r[4 * h][0]));
            if (j8 + STEP >= T) {
              // this warp's last columns are in registers: hand the accumulator back to the
              // MMA issuer before solving them
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&bars->acc_empty[buf]);
              released = true;
            }
            const int nval = jend - (j0 + j8) < 8 ? jend - (j0 + j8) : 8;  // valid traits
            if (GP == 2) {
              // a SNP's two working columns: the column-0 lanes (0-15) solve each pair with the
              // partner lane's a and c and the SNP's three s planes, writing their rows directly
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                if (u >= nval) continue;
                float a0[QQ + 1], a1[QQ + 1];
#pragma unroll
                for (int k = 0; k <= QQ; ++k) {
                  a0[k] = __uint_as_float(r[u][k]);
                  a1[k] = __shfl_down_sync(0xffffffffu, a0[k], 16);
                }
                const int j = j0 + j8 + u;
                if (egk == 0 && live) {
                  const float* sj = p.sbuf + (int64_t)j * p.lds;
                  // a trait the CHOL kernel scans afterwards (P_j[0] is NaN) is not counted here
                  const float* Pu = cst + (j8 + u) * (QQ * QQ + QQ);
                  nsing += (Pu[0] == Pu[0]) &
                           ac_pair<QQ>(p, Pu, a0, a1, __ldg(sj + snp), __ldg(sj + p.xplane + snp),
                                       __ldg(sj + 2 * p.xplane + snp), mu_snp, mu_pair, snp, j);
                }
              }
              continue;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              if (u >= nval) continue;
              const float* Pj = cst + (j8 + u) * (QQ * QQ + QQ);
              float a[QQ + 1], vq[QQ + 1], aPa = 0.f;
#pragma unroll
              for (int k = 0; k < QQ; ++k) a[k] = __uint_as_float(r[u][k]);
              const float cval = __uint_as_float(r[u][QQ]);
#pragma unroll
              for (int k = 0; k < QQ; ++k) {
                float acc = 0.f;
#pragma unroll
                for (int l = 0; l < QQ; ++l) acc = fmaf(Pj[k * QQ + l], a[l], acc);
                aPa = fmaf(a[k], acc, aPa);
                vq[k] = acc;
              }
              const float s = scur[u];
              const float sigma = s - aPa;
              float o[QQ + 1];
              float wv;
              if (sigma > 1e-5f * s) {
                const float bs = __fdividef(cval, sigma);
#pragma unroll
                for (int k = 0; k < QQ; ++k) o[k] = Pj[QQ * QQ + k] - vq[k] * bs;
                // centred SNP x - mu: the intercept (column 0 of X_L) absorbs mu * b_snp
                if (p.mu) o[0] -= mu_snp * bs;
                o[QQ] = bs;
                wv = bs * cval;
              } else {
#pragma unroll
                for (int k = 0; k <= QQ; ++k) o[k] = __int_as_float(0x7fc00000);
                wv = __int_as_float(0x7fc00000);
                // a trait the CHOL kernel scans afterwards (P_j[0] is NaN) is not counted here
                nsing += live && Pj[0] == Pj[0];
              }
              if (VAR) {
                // b, then Var(b) as a packed upper triangle, written by this thread straight to
                // its SNP's row (no staging): [[P + v v^T / sigma, -v / sigma], [., 1 / sigma]]
                // of the centred SNP, mapped back by b = T b_c, T = I - mu e_0 e_q^T, which
                // changes only row and column 0 (the intercept)
                if (live) {
                  constexpr int PWV = (QQ + 1) + (QQ + 1) * (QQ + 2) / 2;
                  float* dst = p.B + (snp * p.t + (j0 + j8 + u)) * PWV;
                  const bool okp = sigma > 1e-5f * s;
                  const float inv = 1.f / sigma, mu = p.mu ? mu_snp : 0.f;
#pragma unroll
                  for (int k = 0; k <= QQ; ++k) dst[k] = o[k];
#pragma unroll
                  for (int r = 0; r <= QQ; ++r)
#pragma unroll
                    for (int c = r; c <= QQ; ++c) {
                      float x;
                      if (c < QQ)
                        x = Pj[r * QQ + c] + vq[r] * vq[c] * inv;
                      else
                        x = r < QQ ? -vq[r] * inv : inv;
                      if (r == 0) x -= mu * (c < QQ ? -vq[c] * inv : inv);
                      if (r == 0 && c == 0) x -= mu * (-vq[0] * inv) - mu * mu * inv;
                      dst[(QQ + 1) + r * (QQ + 1) - r * (r - 1) / 2 + (c - r)] =
                          okp ? x : __int_as_float(0x7fc00000);
                    }
                  if (p.W) p.W[snp * p.t + j0 + j8 + u] = wv;
                }
                continue;
              }
              if (p.out_snp) {
                // (b_snp, standard error 1 / sqrt(sigma)) per pair
                float* so = stgB + lane * RB + 2 * u;
                so[0] = o[QQ];
                so[1] = sigma > 1e-5f * s ? rsqrtf(sigma) : __int_as_float(0x7fc00000);
              } else if (QQ == 3) {
                float* so = stgB + lane * RB + u * (QQ + 1);
                *reinterpret_cast<float4*>(so) = make_float4(o[0], o[1], o[2], o[QQ]);
              } else {
                float* so = stgB + lane * RB + u * (QQ + 1);
#pragma unroll
                for (int k = 0; k <= QQ; ++k) so[k] = o[k];
              }
              stgW[lane * 9 + u] = wv;
            }
            if (VAR) continue;  // written above, per thread
            __syncwarp();
            // Write the warp's 32 SNP rows: each row holds nval (q+1) contiguous floats of B
            // and nval of wald; consecutive lanes take consecutive floats of a row.
            const int64_t jb = j0 + j8;
            const int pw = p.out_snp ? 2 : q1;  // values per pair in B
            // float4 stores need B 16-byte aligned (the ABI promises only float alignment) and,
            // for SNP mode (2 floats per pair), an even t
            const bool vec_ok = (reinterpret_cast<uintptr_t>(p.B) & 15) == 0;
            if (QQ == 3 && nval == 8 && p.out_snp && vec_ok && (p.t & 1) == 0) {
              // SNP mode: (b_snp, se) of 8 traits = 4 float4 per row, 8 rows per instruction
#pragma unroll
              for (int it = 0; it < 4; ++it) {
                const int rr = it * 8 + (lane >> 2), c4 = lane & 3;
                const int64_t sn = row0 + rr;
                if (sn < p.m) {
                  const float4 v = *reinterpret_cast<const float4*>(stgB + rr * RB + c4 * 4);
                  *reinterpret_cast<float4*>(p.B + (sn * p.t + jb) * 2 + c4 * 4) = v;
                }
              }
            } else if (QQ == 3 && nval == 8 && !p.out_snp && vec_ok) {
              // 8 float4 per row, 4 rows per instruction
#pragma unroll
              for (int it = 0; it < 8; ++it) {
                const int rr = it * 4 + (lane >> 3), c4 = lane & 7;
                const int64_t sn = row0 + rr;
                if (sn < p.m) {
                  const float4 v = *reinterpret_cast<const float4*>(stgB + rr * RB + c4 * 4);
                  *reinterpret_cast<float4*>(p.B + (sn * p.t + jb) * 4 + c4 * 4) = v;
                }
              }
            } else {
              const int nb_f = nval * pw;
              for (int e = lane; e < 32 * nb_f; e += 32) {
                const int rr = e / nb_f, c = e - rr * nb_f;
                const int64_t sn = row0 + rr;
                if (sn < p.m) p.B[(sn * p.t + jb) * pw + c] = stgB[rr * RB + c];
              }
            }
            if (p.W) {
              if (nval == 8) {
#pragma unroll
                for (int it = 0; it < 8; ++it) {
                  const int rr = it * 4 + (lane >> 3), c = lane & 7;
                  const int64_t sn = row0 + rr;
                  if (sn < p.m) p.W[sn * p.t + jb + c] = stgW[rr * 9 + c];
                }
              } else {
                for (int e = lane; e < 32 * nval; e += 32) {
                  const int rr = e / nval, c = e - rr * nval;
                  const int64_t sn = row0 + rr;
                  if (sn < p.m) p.W[sn * p.t + jb + c] = stgW[rr * 9 + c];
                }
              }
            }
            __syncwarp();
          }
          if (!released) {  // a warp with no batch in this block (fewer than 9 traits)
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars->acc_empty[buf]);
          }
          if (nsing) atomicAdd(&p.flags[FLAG_SINGULAR], nsing);
        }
        if (EPI != EPI_AC) {  // AC hands the accumulator back inside its batch loop
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&bars->acc_empty[buf]);
        }
      }
      if (++buf == 2) { buf = 0; accph ^= 1; }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

template <int EPI, int QQ, bool VAR = false, int GP = 1, int NP = 2>
void prepare_one() {
  constexpr size_t SMEM = smem_of(EPI, QQ);
  static_assert(SMEM <= 232448, "shared memory over the sm_103 opt-in limit");
  GW_CUDA(cudaFuncSetAttribute(eig_tc_kernel<EPI, QQ, VAR, GP, NP>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM));
}

template <int EPI, int QQ, bool VAR = false, int GP = 1, int NP = 2>
void launch_one(cudaStream_t s, const CUtensorMap& mapA, const CUtensorMap& mapB,
                const CUtensorMap& mapG, const EigTcParams& p, int num_sms) {
  constexpr size_t SMEM = smem_of(EPI, QQ);
  constexpr int TS = EPI == EPI_SQ ? BM : BM / GP;
  const int64_t work = ((p.m + TS - 1) / TS) * p.nblk;
  const unsigned grid = (unsigned)(work < num_sms ? work : num_sms);
  eig_tc_kernel<EPI, QQ, VAR, GP, NP>
      <<<grid, 32 * nwarps_of(EPI, QQ), SMEM, s>>>(mapA, mapB, mapG, p);
  GW_CHECK_LAUNCH();
}

// AC per q; two working columns solve each pair in ac_pair, which writes every output mode
template <bool VAR, int GP, int NP>
void launch_ac(cudaStream_t s, const CUtensorMap& mapA, const CUtensorMap& mapB,
               const CUtensorMap& mapG, const EigTcParams& p, int num_sms) {
  switch (p.q) {
    case 1: launch_one<EPI_AC, 1, VAR, GP, NP>(s, mapA, mapB, mapG, p, num_sms); break;
    case 2: launch_one<EPI_AC, 2, VAR, GP, NP>(s, mapA, mapB, mapG, p, num_sms); break;
    case 3: launch_one<EPI_AC, 3, VAR, GP, NP>(s, mapA, mapB, mapG, p, num_sms); break;
    case 4: launch_one<EPI_AC, 4, VAR, GP, NP>(s, mapA, mapB, mapG, p, num_sms); break;
    case 5: launch_one<EPI_AC, 5, VAR, GP, NP>(s, mapA, mapB, mapG, p, num_sms); break;
    case 6: launch_one<EPI_AC, 6, VAR, GP, NP>(s, mapA, mapB, mapG, p, num_sms); break;
    default: launch_one<EPI_AC, 7, VAR, GP, NP>(s, mapA, mapB, mapG, p, num_sms); break;
  }
}

template <bool VAR, int GP, int NP>
void prepare_ac() {
  prepare_one<EPI_AC, 1, VAR, GP, NP>();
  prepare_one<EPI_AC, 2, VAR, GP, NP>();
  prepare_one<EPI_AC, 3, VAR, GP, NP>();
  prepare_one<EPI_AC, 4, VAR, GP, NP>();
  prepare_one<EPI_AC, 5, VAR, GP, NP>();
  prepare_one<EPI_AC, 6, VAR, GP, NP>();
  prepare_one<EPI_AC, 7, VAR, GP, NP>();
}

}  // namespace

void eig_tc_prepare() {
  // attributes belong to the current device: set once per device (setups may run on several
  // host threads at once)
  static std::mutex mu;
  static uint64_t done_mask = 0;
  std::lock_guard<std::mutex> lock(mu);
  int dev = 0;
  GW_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = 1ull << (dev & 63);
  if (done_mask & bit) return;
  prepare_one<EPI_ROT, 0>();
  prepare_one<EPI_ROT, 0, false, 2>();
  prepare_one<EPI_SQ, 0>();
  prepare_ac<false, 1, 2>();
  prepare_ac<true, 1, 2>();
  prepare_ac<false, 2, 2>();
  prepare_ac<false, 1, 3>();
  prepare_ac<true, 1, 3>();
  prepare_ac<false, 2, 3>();
  done_mask |= bit;
}

void eig_tc_launch(cudaStream_t s, int stage, const CUtensorMap& mapA, const CUtensorMap& mapB,
                   const CUtensorMap& mapG, const EigTcParams& p, int num_sms) {
  if (p.m <= 0 || p.nblk <= 0) return;
  GW_REQUIRE(p.q >= 1 && p.q <= QMAX, GWAS_ERR_ARG, "q out of range");
  GW_REQUIRE(p.gp == 1 || p.gp == 2, GWAS_ERR_ARG, "genetic columns %d outside [1,2]", p.gp);
  GW_REQUIRE(p.pieces == 2 || p.pieces == 3, GWAS_ERR_ARG, "split pieces %d outside [2,3]",
             p.pieces);
  switch (stage) {
    case 0:
      GW_REQUIRE(p.pieces == 2, GWAS_ERR_ARG, "the rotation takes two split pieces");
      if (p.gp == 2)
        launch_one<EPI_ROT, 0, false, 2>(s, mapA, mapB, mapG, p, num_sms);
      else
        launch_one<EPI_ROT, 0>(s, mapA, mapB, mapG, p, num_sms);
      break;
    case 1: launch_one<EPI_SQ, 0>(s, mapA, mapB, mapG, p, num_sms); break;
    default:
      if (p.pieces == 3) {
        if (p.gp == 2)
          launch_ac<false, 2, 3>(s, mapA, mapB, mapG, p, num_sms);
        else if (p.out_var)
          launch_ac<true, 1, 3>(s, mapA, mapB, mapG, p, num_sms);
        else
          launch_ac<false, 1, 3>(s, mapA, mapB, mapG, p, num_sms);
      } else if (p.gp == 2) {
        launch_ac<false, 2, 2>(s, mapA, mapB, mapG, p, num_sms);
      } else if (p.out_var) {
        launch_ac<true, 1, 2>(s, mapA, mapB, mapG, p, num_sms);
      } else {
        launch_ac<false, 1, 2>(s, mapA, mapB, mapG, p, num_sms);
      }
  }
}

}  // namespace gw
