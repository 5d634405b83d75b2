// CHOL fused whiten-and-reduce on the tensor cores (tcgen05 / TMEM / TMA, sm_103a).
//
// Algorithm 3's per-SNP work (whitening, bordered solve) for one trait.  A persistent CTA walks 128-SNP tiles.  The B
// operand is L^-1 augmented with q + 1 rows: u_k = M^-1 X_L[:,k] (k < q) and M^-1 r (r the
// null residual), so one product gives, per SNP, the whitened genotypes x' = L^-1 x (columns
// < n) and, being linear in x, a_k = x^T M^-1 X_L[:,k] and c = x^T M^-1 r (columns n .. n+q).
// For each block of 256 rows it accumulates D[snp][r] in TMEM over only the K range c <= r
// where L^-1 can be nonzero (the aggregated triangular solve of "Sequences of GLS'", done as
// one product with the precomputed inverse); the augmented rows take the full K range.  On the
// diagonal of a block a K step of 64 columns multiplies only the rows it meets (narrower MMAs
// into the matching accumulator columns), and the last block stops at row n + q.  The
// augmented matrix is split into BF16 hi + lo pieces and genotypes are exact in BF16, so
// D = X hi^T + X lo^T carries ~16 significant bits with FP32 accumulation (a third piece,
// ~24 bits, for a trait whose M is badly conditioned).  The FP8 variant (SPLIT_FP8) splits it
// into an FP16 hi piece and an E4M3 lo piece instead (each row group scaled by a power of two):
// the hi product takes the centred genotypes in FP16 (kind::f16), the lo product the uncentred
// codes in E4M3 (kind::f8f6f4, twice the rate), both into the same accumulator, ~15 bits in
// all; both 8- and 16-bit genotype tiles, and both pieces, hold their K columns in the order the
// converters produce the E4M3 bytes in (e4m3_k_slot within every group of 16).  The lo product
// misses the centring term mu (lo 1): accumulator row r holds x'_r + mu lsum_r.  One more
// augmented row, w = sum_r lsum_r (hi + lo)_r, yields w . (x - mu) = sum_r lsum_r x'_r, from which
// the epilogue corrects s, a and c with a few scalar operations per SNP; it also removes the
// power-of-two scales.  The epilogue sums
// s = x'^T x' out of TMEM (FP32 within a block, FP64 across blocks), picks up a and c, and
// finishes each tile with the Schur-complement solve in FP64.  X' is never written to memory.
// With an intercept in X_L each SNP is centred by mu, the multiple of 1/64 nearest its mean
// (exact in BF16): s - a^T P a then no longer cancels the large intercept component, whose BF16
// splitting errors in s and in a are not correlated; b_snp and the Wald statistic are unchanged
// and the intercept estimate is corrected by -mu b_snp.
//
// Warp roles (448 threads):
//   0-3  epilogue: one SNP per thread (TMEM lane 32*warp + lane)
//   11   TMA producers: lane 0 the L^-1 tiles, lane 1 the 2-bit packed genotype slices
//   7    MMA issuer (one elected lane); owns the 512 TMEM columns (two 256-column accumulators)
//   4-6, 8-10, 12-13  genotype converters: packed slices (shared memory) -> BF16 (FP8 variant:
//        FP16) tiles in the 128-byte-swizzled K-major layout, and in the FP8 variant also E4M3
//        tiles of 64-byte rows in the 64-byte-swizzled layout
#include <mutex>

#include "tc_kernels.cuh"
#include "tc_ptx.cuh"

namespace gw {
using namespace tc;

namespace {

constexpr int BM = CHOL_TC_BM;
constexpr int BN = 256;
constexpr int BK = 64;
constexpr int A_BYTES = BM * BK * 2;    // 16 KB
constexpr int B_BYTES = BN * BK * 2;    // 32 KB
constexpr int A8_BYTES = BM * BK;       // FP8 variant: E4M3 genotype tile, 8 KB
constexpr int B8_BYTES = BN * BK;       // FP8 variant: E4M3 lo tile, 16 KB
constexpr int QMAX = 7;
constexpr int PK_BYTES = BM * 16;       // 64 genotypes of 128 SNPs, 2-bit codes: 2 KB
constexpr int NCONV = 8;                // genotype converter warps: 2 threads per row
constexpr int NUM_THREADS = 192 + 32 * NCONV;
// Warp roles.  A warp issues on SMSP (warp % 4); the single-thread MMA issuer and TMA producers
// share SMSP 3 with only an epilogue warp, so converter bursts never delay their issue.
constexpr int MMA_WARP = 7;
constexpr int TMA_WARP = 11;
// converter warps 4, 5, 6, 8, 9, 10, 12, 13 -> 0 .. 7
__device__ __forceinline__ int conv_index(int warp) {
  return warp < MMA_WARP ? warp - 4 : warp < TMA_WARP ? warp - 5 : warp - 6;
}
constexpr int TMEM_COLS = 512;
constexpr uint64_t WAIT_NS = 4000000000ull;

template <int SA, int SB, int PR>
struct __align__(8) BarsT {
  uint64_t a_full[SA], a_empty[SA], b_full[SB], b_empty[SB], pk_full[PR], pk_empty[PR];
  uint64_t acc_full[2], acc_empty[2], mu_full[2], mu_empty[2], done;
  uint32_t tmem_base;
  int abort;
  float mu[2][BM];  // SNP centres of the tiles in flight (epilogue -> converters)
};

// Shared-memory rings.  BF16: slots of one genotype tile (A) and of one piece of one K step (B).
// FP8: an A slot holds the FP16 tile and then the E4M3 tile of one K step, a B slot the FP16 hi
// tile and then the E4M3 lo tile of one K step.
template <bool F8>
struct Layout {
  static constexpr int SA = 3;                                   // genotype slots
  static constexpr int SB = F8 ? 3 : 5;                          // L^-1 slots
  static constexpr int PR = F8 ? 4 : 8;                          // packed-slice slots
  static constexpr int A_SLOT = F8 ? A_BYTES + A8_BYTES : A_BYTES;
  static constexpr int B_SLOT = F8 ? B_BYTES + B8_BYTES : B_BYTES;
  using Bars = BarsT<SA, SB, PR>;
  static constexpr size_t SMEM =
      1024 + (size_t)SA * A_SLOT + (size_t)SB * B_SLOT + (size_t)PR * PK_BYTES + sizeof(Bars);
  static_assert(SMEM <= 232448, "shared memory over the sm_103 opt-in limit");
};

__device__ __forceinline__ int ksteps(int nb, int kpad) {
  const int k = (nb + 1) * (BN / BK);
  const int kmax = kpad / BK;
  return k < kmax ? k : kmax;
}
// Rows of block nb that K step ks meets, in units of 64: L^-1 is lower triangular, so a K step
// on the diagonal (ks = 4 nb + j) meets only rows 64 j .. 255 of the block; j = 0 below it.
__device__ __forceinline__ int diag_skip(int nb, int ks) {
  const int j = ks - nb * (BN / BK);
  return j > 0 ? j : 0;
}

// Live accumulator columns of block nb: rows of the augmented matrix below n + naug, rounded
// up to the MMA's N granularity (16).
__device__ __forceinline__ int block_cols(int nb, int n, int naug) {
  const int live = n + naug - nb * BN;
  const int c = (live + 15) & ~15;
  return c < BN ? c : BN;
}

// With GP = 2 genetic columns per SNP a tile holds 64 SNPs: A row r is column (r / 16) % 2 of SNP
// (r / 32) 16 + r % 16, so that a SNP's two rows sit in lanes l and l + 16 of one epilogue warp.
template <int GP>
__device__ __forceinline__ int row_snp(int r) { return GP == 1 ? r : (r >> 5) * 16 + (r & 15); }
template <int GP>
__device__ __forceinline__ int row_col(int r) { return GP == 1 ? 0 : (r >> 4) & 1; }

// (tile, block, k-step) sequence shared by every role of a CTA.  A tile's blocks run from the
// last (the longest K range) down to the first: after a tile's last block the epilogue has its
// per-tile work to do (the bordered solves of the tile, the centres of a later tile) while the
// tensor cores start the next tile, and the two longest blocks give it the most time to do it
// before it must hand an accumulator back.
struct Step {
  int64_t tile;
  int nb, ks;
};
__device__ __forceinline__ void advance(Step& s, int nblocks, int kpad) {
  if (++s.ks < ksteps(s.nb, kpad)) return;
  s.ks = 0;
  if (--s.nb >= 0) return;
  s.nb = nblocks - 1;
  s.tile += gridDim.x;
}

// The bordered solve of one SNP with a two-column genetic block, in FP64 (Algorithm 3's per-SNP
// solve with X_R,i = [g0 | g1], the working basis of the model): a0, a1 = X_L^T M^-1 g_k
// (centred columns), c = g_k^T M^-1 r0, S00, S01, S11 = g_k^T M^-1 g_l.  V = P [a0 a1],
// Sigma = S_RR - [a0 a1]^T V, b_w = Sigma^-1 c, b_L = b0 - V b_w, wald = b_w . c (2 d.o.f.),
// singular when a pivot of Sigma's Cholesky is at most 1e-5 of the matching S_kk.  Centred
// columns g_k - mu_k: the intercept absorbs sum_k mu_k b_w,k.  Reported: b_R = tm b_w and
// Var(b) = R Var_c R^T, Var_c the centred working-basis Var, R the map b_c -> reported b
// (row 0: e_0 - sum_k mu_k e_(q+k); rows q + g: sum_k tm[g][k] e_(q+k); other rows e_r).
template <int QM>
__device__ __noinline__ void solve_pair(const CholTcParams& p, const float* a0, const float* a1,
                                        float c0, float c1, double S00, double S01, double S11,
                                        float m0, float m1, int64_t snp) {
  const int q = p.q;
  double v[2][QM];
#pragma unroll
  for (int k = 0; k < QM; ++k) {
    double x0 = 0.0, x1 = 0.0;
    if (k < q) {
#pragma unroll
      for (int l = 0; l < QM; ++l)
        if (l < q) {
          const double pk = __ldg(&p.P[k * q + l]);
          x0 += pk * (double)a0[l];
          x1 += pk * (double)a1[l];
        }
    }
    v[0][k] = x0;
    v[1][k] = x1;
  }
  double g00 = S00, g01 = S01, g11 = S11;
#pragma unroll
  for (int k = 0; k < QM; ++k)
    if (k < q) {
      g00 -= (double)a0[k] * v[0][k];
      g01 -= (double)a0[k] * v[1][k];
      g11 -= (double)a1[k] * v[1][k];
    }
  const double piv1 = g11 - g01 * g01 / g00;
  const bool ok = g00 > 1e-5 * S00 && piv1 > 1e-5 * S11;
  const int p2 = q + 2;
  const int pw = p.out_snp ? 4 : p.out_var ? p2 + p2 * (p2 + 1) / 2 : p2;
  float* Bo = p.B + (snp * p.t + p.j) * pw;
  const float nanv = __int_as_float(0x7fc00000);
  if (!ok) {
    for (int k = 0; k < pw; ++k) Bo[k] = nanv;
    if (p.W) p.W[snp * p.t + p.j] = nanv;
    atomicAdd(&p.flags[FLAG_SINGULAR], 1);
    return;
  }
  const double det = g00 * piv1;
  const double si[2][2] = {{g11 / det, -g01 / det}, {-g01 / det, g00 / det}};
  const double bw[2] = {si[0][0] * c0 + si[0][1] * c1, si[1][0] * c0 + si[1][1] * c1};
  const double mu[2] = {p.centre ? (double)m0 : 0.0, p.centre ? (double)m1 : 0.0};
  const double tm[2][2] = {{p.tm[0], p.tm[1]}, {p.tm[2], p.tm[3]}};
  if (p.W) p.W[snp * p.t + p.j] = (float)(bw[0] * c0 + bw[1] * c1);
  const double bR[2] = {tm[0][0] * bw[0] + tm[0][1] * bw[1], tm[1][0] * bw[0] + tm[1][1] * bw[1]};
  // reported Var_RR = tm Si tm^T
  double vr[2][2];
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      double x = 0.0;
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int z = 0; z < 2; ++z) x += tm[g][u] * si[u][z] * tm[h][z];
      vr[g][h] = x;
    }
  if (p.out_snp) {
    Bo[0] = (float)bR[0];
    Bo[1] = (float)bR[1];
    Bo[2] = (float)sqrt(vr[0][0]);
    Bo[3] = (float)sqrt(vr[1][1]);
    return;
  }
#pragma unroll
  for (int k = 0; k < QM; ++k)
    if (k < q) {
      double b = __ldg(&p.b0[k]) - v[0][k] * bw[0] - v[1][k] * bw[1];
      if (k == 0) b -= mu[0] * bw[0] + mu[1] * bw[1];
      Bo[k] = (float)b;
    }
  Bo[q] = (float)bR[0];
  Bo[q + 1] = (float)bR[1];
  if (!p.out_var) return;
  // Var_c (centred, working basis), entry (r, c) of [[P + V Si V^T, -V Si], [-Si V^T, Si]]
  auto vk = [&](int u, int k) { return v[u][k < QM ? k : QM - 1]; };
  auto vc = [&](int r, int c) -> double {
    if (r >= q && c >= q) return si[r - q][c - q];
    if (c >= q) return -(vk(0, r) * si[0][c - q] + vk(1, r) * si[1][c - q]);
    if (r >= q) return -(vk(0, c) * si[0][r - q] + vk(1, c) * si[1][r - q]);
    double x = __ldg(&p.P[r * q + c]);
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int z = 0; z < 2; ++z) x += vk(u, r) * si[u][z] * vk(z, c);
    return x;
  };
  // row r of R as up to three (index, coefficient) terms
  auto rterms = [&](int r, int* idx, double* cf) -> int {
    if (r >= q) {
      idx[0] = q; cf[0] = tm[r - q][0];
      idx[1] = q + 1; cf[1] = tm[r - q][1];
      return 2;
    }
    idx[0] = r; cf[0] = 1.0;
    if (r != 0) return 1;
    idx[1] = q; cf[1] = -mu[0];
    idx[2] = q + 1; cf[2] = -mu[1];
    return 3;
  };
  for (int r = 0; r < p2; ++r)
    for (int c = r; c < p2; ++c) {
      int ir[3], ic[3];
      double fr[3], fc[3];
      const int nr = rterms(r, ir, fr), nc = rterms(c, ic, fc);
      double x = 0.0;
      for (int u = 0; u < nr; ++u)
        for (int z = 0; z < nc; ++z) x += fr[u] * fc[z] * vc(ir[u], ic[z]);
      Bo[p2 + r * p2 - r * (r - 1) / 2 + (c - r)] = (float)x;
    }
}

// QM: compile-time bound on q (3 or 7), so the epilogue's per-column arrays stay in registers.
// GP: genetic columns per SNP (1, or 2 for a two-column genetic model).  NP: BF16 pieces of the
// split matrix (2, or 3 for a badly conditioned M; a compile-time bound keeps the issuer's and
// producer's piece loops unrolled).  F8: the FP16 hi + E4M3 lo split (NP = 2).
template <int QM, int GP, int NP, bool F8>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    chol_tc_kernel(const __grid_constant__ CholMaps lmaps, const __grid_constant__ CUtensorMap mapG,
                   const CholTcParams p) {
  static_assert(!F8 || NP == 2, "the FP8 split has two pieces");
  using L = Layout<F8>;
  using Bars = typename L::Bars;
  constexpr int SA = L::SA, SB = L::SB, PR = L::PR, A_SLOT = L::A_SLOT, B_SLOT = L::B_SLOT;
  constexpr int TS = BM / GP;        // SNPs per tile
  constexpr int PKB = TS * 16;       // bytes of one packed slice (64 genotypes of TS SNPs)
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA = smem;
  uint8_t* sB = sA + SA * A_SLOT;
  uint8_t* sP = sB + SB * B_SLOT;
  Bars* bars = (Bars*)(sP + PR * PK_BYTES);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int64_t tiles_run = (p.m + TS - 1) / TS;
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
    for (int i = 0; i < 2; ++i) {
      mbar_init(&bars->mu_full[i], 128);            // every epilogue thread stores its SNP's centre
      mbar_init(&bars->mu_empty[i], 32 * NCONV);    // every converter thread has read its row's
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
    for (int j = 0; j < 4; ++j) prefetch_tensormap(&lmaps.m[j]);
    if (F8)
      for (int j = 0; j < 4; ++j) prefetch_tensormap(&lmaps.m8[j]);
    prefetch_tensormap(&mapG);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = bars->tmem_base;
  volatile int* abort = &bars->abort;

  if (warp == TMA_WARP) {
    // ------------------------------------------------------------ L^-1 tiles via TMA
    if (lane == 0) {
      int bs = 0;
      uint32_t bph = 0;
      bool ok = true;
      for (Step st{blockIdx.x, nblocks - 1, 0}; st.tile < tiles_run && ok;
           advance(st, nblocks, p.kpad)) {
        const int j = diag_skip(st.nb, st.ks);  // rows 64 j .. 255 of the block
        if constexpr (F8) {
          // one slot: the FP16 hi tile, then the E4M3 lo tile (64-byte rows)
          ok = mbar_wait(&bars->b_empty[bs], bph ^ 1, abort, tflag, WAIT_NS);
          if (!ok) break;
          const int y = st.nb * BN + 64 * j;
          uint8_t* dst = sB + bs * B_SLOT;
          mbar_arrive_expect_tx(&bars->b_full[bs], (B_BYTES / 4 + B8_BYTES / 4) * (4 - j));
          tma_load_2d(dst + (B_BYTES / 4) * j, &lmaps.m[j], &bars->b_full[bs], st.ks * BK, y);
          tma_load_2d(dst + B_BYTES + (B8_BYTES / 4) * j, &lmaps.m8[j], &bars->b_full[bs],
                      st.ks * BK, y);
          if (++bs == SB) { bs = 0; bph ^= 1; }
        } else {
          for (int piece = 0; piece < NP; ++piece) {
            ok = mbar_wait(&bars->b_empty[bs], bph ^ 1, abort, tflag, WAIT_NS);
            if (!ok) break;
            const int y = piece * p.rpad + st.nb * BN + 64 * j;
            uint8_t* dst = sB + bs * B_BYTES + (B_BYTES / 4) * j;
            mbar_arrive_expect_tx(&bars->b_full[bs], (B_BYTES / 4) * (4 - j));
            tma_load_2d(dst, &lmaps.m[j], &bars->b_full[bs], st.ks * BK, y);
            if (++bs == SB) { bs = 0; bph ^= 1; }
          }
        }
      }
    } else if (lane == 1) {
      // packed genotype slices (64 genotypes x TS SNPs) via TMA, in the K-step order the
      // converters consume them; rows past m read as zero
      int ps = 0;
      uint32_t pph = 0;
      for (Step st{blockIdx.x, nblocks - 1, 0}; st.tile < tiles_run; advance(st, nblocks, p.kpad)) {
        if (st.nb == nblocks - 1 && st.ks == 0) {
          // two tiles ahead, the rows into L2: their slices, and the epilogue's reads of them
          // for the SNP centres, then hit L2 instead of waiting on DRAM
          const int64_t t2 = st.tile + 2 * (int64_t)gridDim.x;
          if (t2 < tiles_run) {
            const int64_t r0 = t2 * TS, r1 = r0 + TS < p.m ? r0 + TS : p.m;
            prefetch_l2_range(p.G + r0 * p.row_bytes, p.G + r1 * p.row_bytes);
          }
        }
        if (!mbar_wait(&bars->pk_empty[ps], pph ^ 1, abort, tflag, WAIT_NS)) break;
        mbar_arrive_expect_tx(&bars->pk_full[ps], PKB);
        tma_load_2d(sP + ps * PK_BYTES, &mapG, &bars->pk_full[ps], st.ks * 16,
                    (int32_t)(st.tile * TS));
        if (++ps == PR) { ps = 0; pph ^= 1; }
      }
    }
  } else if (warp == MMA_WARP) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int as = 0, bs = 0, buf = 0;
      uint32_t aph = 0, bph = 0, accph = 0;
      bool ok = true;
      for (int64_t tile = blockIdx.x; tile < tiles_run && ok; tile += gridDim.x) {
        for (int nb = nblocks - 1; nb >= 0 && ok; --nb) {
          ok = mbar_wait(&bars->acc_empty[buf], accph ^ 1, abort, tflag, WAIT_NS);
          if (!ok) break;
          tc_fence_after();
          const uint32_t dt = tmem + buf * BN;
          const int nk = ksteps(nb, p.kpad), ncols = block_cols(nb, p.n, p.naug);
          for (int ks = 0; ks < nk && ok; ++ks) {
            ok = mbar_wait(&bars->a_full[as], aph, abort, tflag, WAIT_NS);
            if (!ok) break;
            tc_fence_after();
            const uint64_t ad = sw128_desc(sA + as * A_SLOT);
            const int j = diag_skip(nb, ks);  // accumulator columns 64 j .. ncols - 1
            if constexpr (F8) {
              // (x - mu in FP16) x (hi in FP16), then (x in E4M3) x (lo in E4M3), one accumulator
              const uint32_t idesc = idesc_f16(BM, ncols - 64 * j);
              const uint64_t ad8 = sw64_desc(sA + as * A_SLOT + A_BYTES);
              ok = mbar_wait(&bars->b_full[bs], bph, abort, tflag, WAIT_NS);
              if (!ok) break;
              tc_fence_after();
              const uint64_t bd = sw128_desc(sB + bs * B_SLOT + (B_BYTES / 4) * j);
              const uint64_t bd8 = sw64_desc(sB + bs * B_SLOT + B_BYTES + (B8_BYTES / 4) * j);
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(dt + 64 * j, ad + 2 * kk, bd + 2 * kk, idesc, (ks | kk) != 0);
#pragma unroll
              for (int kk = 0; kk < BK / 32; ++kk)
                mma_fp8(dt + 64 * j, ad8 + 2 * kk, bd8 + 2 * kk, idesc, 1u);
              mma_commit(&bars->b_empty[bs]);
              if (++bs == SB) { bs = 0; bph ^= 1; }
              mma_commit(&bars->a_empty[as]);
              if (++as == SA) { as = 0; aph ^= 1; }
            } else {
              const uint32_t idesc = idesc_bf16(BM, ncols - 64 * j);
              for (int piece = 0; piece < NP; ++piece) {
                ok = mbar_wait(&bars->b_full[bs], bph, abort, tflag, WAIT_NS);
                if (!ok) break;
                tc_fence_after();
                const uint64_t bd = sw128_desc(sB + bs * B_SLOT + (B_BYTES / 4) * j);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                  mma_bf16(dt + 64 * j, ad + 2 * kk, bd + 2 * kk, idesc, (ks | piece | kk) != 0);
                mma_commit(&bars->b_empty[bs]);
                if (++bs == SB) { bs = 0; bph ^= 1; }
              }
              mma_commit(&bars->a_empty[as]);
              if (++as == SA) { as = 0; aph ^= 1; }
            }
          }
          if (ok) mma_commit(&bars->acc_full[buf]);
          if (++buf == 2) { buf = 0; accph ^= 1; }
        }
      }
      mma_commit(&bars->done);  // TMEM is released only after every issued MMA retired
      mbar_wait(&bars->done, 0, abort, tflag, WAIT_NS);
    }
  } else if (warp >= 4) {
    // ------------------------------------------------------------ genotype converters
    // Thread ct converts half hh of row r of each K step: packed bytes 8 hh .. 8 hh + 7 (32
    // genotypes) into BF16 (FP8 variant: FP16) chunks 4 hh .. 4 hh + 3 of the row's swizzled
    // 128-byte line, and in the FP8 variant into E4M3 chunks 2 hh, 2 hh + 1 of the row's
    // 64-byte line (chunk c at c ^ ((r >> 1) & 3)).
    const int ct = conv_index(warp) * 32 + lane;
    const int r = ct >> 1, hh = ct & 1;
    const int srow = row_snp<GP>(r);             // the row's SNP within the tile
    const uint32_t code = p.code[row_col<GP>(r)];  // the row's genetic column
    const uint32_t line = (r >> 3) * 1024 + (r & 7) * 128;
    const uint32_t line8 = r * 64;
    const uint32_t t8 = coded_e4m3_table(code);  // the uncentred codes in E4M3
    __half2 mu2 = __float2half2_rn(0.f);          // FP8 variant: the row's centre, twice
    int per_tile = 0;
    for (int nb = 0; nb < nblocks; ++nb) per_tile += ksteps(nb, p.kpad);
    int as = 0, ps = 0;
    uint32_t aph = 0, pph = 0;
    bool ok = true;
    int ti = 0;  // this CTA's tile counter (selects the centre buffer)
    for (int64_t tile = blockIdx.x; tile < tiles_run && ok; tile += gridDim.x, ++ti) {
      // byte tables of this row: cd(g) - mu (mu = 0 without centring)
      uint32_t lutlo, luthi;
      if (p.centre) {
        const int mb = ti & 1;
        ok = __all_sync(0xffffffffu,
                        mbar_wait(&bars->mu_full[mb], (ti >> 1) & 1, abort, tflag, WAIT_NS));
        if (!ok) break;
        if (F8)
          mu2 = __float2half2_rn(bars->mu[mb][r]);  // a multiple of 1/64: exact
        else
          coded_lut(bars->mu[mb][r], code, lutlo, luthi);
        mbar_arrive(&bars->mu_empty[mb]);
      } else {
        coded_lut(0.f, code, lutlo, luthi);
      }
      for (int g = 0; g < per_tile; ++g) {
        // warp-uniform exits: every lane leaves together if any wait gave up
        ok = __all_sync(0xffffffffu, mbar_wait(&bars->pk_full[ps], pph, abort, tflag, WAIT_NS));
        if (!ok) break;
        const uint2 w = *reinterpret_cast<const uint2*>(sP + ps * PK_BYTES + srow * 16 + hh * 8);
        // the slot is refilled by TMA (async proxy): order these generic reads before it
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->pk_empty[ps]);
        if (++ps == PR) { ps = 0; pph ^= 1; }
        uint4 o[4], e8[2];
        if constexpr (F8) {
          // E4M3 codes by byte permutes, then FP16 cd - mu from them, in the same K order
          e8[0] = packed16_to_e4m3x16(w.x, t8);
          e8[1] = packed16_to_e4m3x16(w.y, t8);
          e4m3x16_to_f16_centred(e8[0], mu2, o[0], o[1]);
          e4m3x16_to_f16_centred(e8[1], mu2, o[2], o[3]);
        } else {
          packed8_to_bf16x32(w, lutlo, luthi, o);
        }
        ok = __all_sync(0xffffffffu, mbar_wait(&bars->a_empty[as], aph ^ 1, abort, tflag, WAIT_NS));
        if (!ok) break;
        uint8_t* dst = sA + as * A_SLOT + line;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int j = 4 * hh + i;
          *reinterpret_cast<uint4*>(dst + ((j ^ (r & 7)) << 4)) = o[i];
        }
        if (F8) {
          uint8_t* dst8 = sA + as * A_SLOT + A_BYTES + line8;
#pragma unroll
          for (int i = 0; i < 2; ++i) {
            const int j = 2 * hh + i;
            *reinterpret_cast<uint4*>(dst8 + ((j ^ ((r >> 1) & 3)) << 4)) = e8[i];
          }
        }
        // every lane's writes are ordered before the async proxy, then one arrive per warp
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars->a_full[as]);
        if (++as == SA) { as = 0; aph ^= 1; }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 0-3)
    // Per block: s += sum of squares of the whitened genotype columns (rows < n); columns
    // n .. n+q of the last block hold a_k and c.  FP32 within a block, FP64 across blocks.
    const int q = p.q, n = p.n;
    int buf = 0;
    uint32_t accph = 0;
    bool ok = true;
    // This thread's row: genetic column gcol of SNP row_snp(row) of each tile (GP = 2: lanes
    // 0-15 hold the first column of the warp's 16 SNPs, lanes 16-31 the second).
    const int row = 32 * warp + lane;
    const int gcol = row_col<GP>(row);
    // With centring, this thread also finds the centre of its row one tile ahead (the
    // converters build the tile's byte tables from it): the nearest multiple of 1/64 to the
    // mean of the coded column, clamped to [0, 2] so that cd(g) - mu stays exact in BF16.  Rows
    // past m get 0.
    auto centre_of = [&](int64_t t) -> float {
      const int64_t snp = t * TS + row_snp<GP>(row);
      if (snp >= p.m) return 0.f;
      const uint4* rw = reinterpret_cast<const uint4*>(p.G + snp * p.row_bytes);
      int n1 = 0, n2 = 0;
      for (int i = 0; i < p.row_bytes / 16; ++i) {
        const uint4 v = __ldg(rw + i);
        count12(v.x, n1, n2);
        count12(v.y, n1, n2);
        count12(v.z, n1, n2);
        count12(v.w, n1, n2);
      }
      return coded_centre(n1, n2, n, p.code[gcol]);
    };
    auto publish_centre = [&](int ti, float c) -> bool {
      const int mb = ti & 1;
      // the converters have read this buffer's previous tile (two tiles back)
      if (!__all_sync(0xffffffffu, mbar_wait(&bars->mu_empty[mb], ((ti >> 1) & 1) ^ 1, abort,
                                             tflag, WAIT_NS)))
        return false;
      bars->mu[mb][32 * warp + lane] = c;
      mbar_arrive(&bars->mu_full[mb]);
      return true;
    };
    float mu_cur = 0.f;
    if (p.centre && blockIdx.x < tiles_run) {
      mu_cur = centre_of(blockIdx.x);
      ok = publish_centre(0, mu_cur);
    }
    int ti = 0;
    for (int64_t tile = blockIdx.x; tile < tiles_run; tile += gridDim.x, ++ti) {
      float mu_next = 0.f;
      if (p.centre && ok && tile + gridDim.x < tiles_run) {
        mu_next = centre_of(tile + gridDim.x);
        ok = publish_centre(ti + 1, mu_next);
      }
      double S = 0.0, X = 0.0;  // s of this row; with GP = 2, the cross product with its partner
      float A[QM], C = 0.f, Wd = 0.f;  // Wd (FP8 variant): w . (x - mu) + mu lsa[q + 1]
#pragma unroll
      for (int k = 0; k < QM; ++k) A[k] = 0.f;
      for (int nb = nblocks - 1; nb >= 0; --nb) {
        if (ok) ok = __all_sync(0xffffffffu, mbar_wait(&bars->acc_full[buf], accph, abort, tflag, WAIT_NS));
        if (ok) {
          tc_fence_after();
          const uint32_t base = tmem + ((uint32_t)(32 * warp) << 16) + buf * BN;
          const int c0 = nb * BN, ncols = block_cols(nb, n, p.naug);
          // four partial sums each (no serial FMA chain); chunks of 32 columns loaded one
          // ahead of the one being summed
          float ss[4] = {0.f, 0.f, 0.f, 0.f}, xs[4] = {0.f, 0.f, 0.f, 0.f};
          auto sum_chunk = [&](const uint32_t (&ra)[32], int c) {
            if (c0 + c + 32 <= n) {
#pragma unroll
              for (int i = 0; i < 32; ++i) {
                const float x = __uint_as_float(ra[i]);
                ss[i & 3] = fmaf(x, x, ss[i & 3]);
                // the partner row (the SNP's other genetic column) is 16 lanes away
                if (GP == 2) xs[i & 3] = fmaf(x, __shfl_xor_sync(0xffffffffu, x, 16), xs[i & 3]);
              }
            } else {
              // the chunk holding row n: genotype columns, then a_0 .. a_{q-1}, c (and w)
#pragma unroll
              for (int i = 0; i < 32; ++i) {
                const int col = c0 + c + i;
                const float x = __uint_as_float(ra[i]);
                if (GP == 2) {
                  const float xp = __shfl_xor_sync(0xffffffffu, x, 16);
                  if (col < n) xs[i & 3] = fmaf(x, xp, xs[i & 3]);
                }
                if (col < n) ss[i & 3] = fmaf(x, x, ss[i & 3]);
#pragma unroll
                for (int k = 0; k < QM; ++k)
                  if (k < q && col == n + k) A[k] = x;
                if (col == n + q) C = x;
                if (F8 && col == n + q + 1) Wd = x;
              }
            }
          };
          // every column of the block is in registers: hand the accumulator back to the issuer
          auto release = [&]() {
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars->acc_empty[buf]);
          };
          if constexpr (QM <= 3) {
            uint32_t ra[32], rb[32];
            tmem_ld32_async(base, ra);
#pragma unroll 1
            for (int c = 0; c < ncols; c += 64) {
              const bool second = c + 32 < ncols;
              tmem_wait32(ra);
              if (second)
                tmem_ld32_async(base + c + 32, rb);
              else
                release();
              sum_chunk(ra, c);
              if (second) {
                tmem_wait32(rb);
                if (c + 64 < ncols)
                  tmem_ld32_async(base + c + 64, ra);
                else
                  release();
                sum_chunk(rb, c + 32);
              }
            }
          } else {
            // q > 3: the registers of a second chunk are not to be had (the warps of an SMSP
            // share its 16 K registers: 128 per thread here), so one chunk at a time
            uint32_t ra[32];
#pragma unroll 1
            for (int c = 0; c < ncols; c += 32) {
              tmem_ld32_async(base + c, ra);
              tmem_wait32(ra);
              if (c + 32 >= ncols) release();
              sum_chunk(ra, c);
            }
          }
          S += (double)((ss[0] + ss[1]) + (ss[2] + ss[3]));
          X += (double)((xs[0] + xs[1]) + (xs[2] + xs[3]));
        }
        if (++buf == 2) { buf = 0; accph ^= 1; }
      }
      if constexpr (F8) {
        // remove the lo product's centring term mu lsum_r from every row, then the power-of-two
        // scales of the row groups (exact)
        const float mu = p.centre ? mu_cur : 0.f;
#pragma unroll
        for (int k = 0; k < QM; ++k)
          if (k < q) A[k] = (A[k] - mu * p.lsa[k]) * p.unscale[1 + k];
        C = (C - mu * p.lsa[q]) * p.unscale[1 + q];
        const double wx = (double)((Wd - mu * p.lsa[q + 1]) * p.unscale[2 + q]);
        const double u0 = (double)p.unscale[0];
        if (GP == 2) {
          // the partner row: the SNP's other working column (16 lanes away)
          const double wxp = __shfl_xor_sync(0xffffffffu, wx, 16);
          const double mup = (double)__shfl_xor_sync(0xffffffffu, mu, 16);
          X = (X - mup * wx - (double)mu * wxp - (double)mu * mup * p.k2) * u0 * u0;
        }
        S = (S - 2.0 * mu * wx - (double)mu * mu * p.k2) * u0 * u0;
      }
      const int64_t snp = tile * TS + row_snp<GP>(row);
      if (GP == 2) {
        // the SNP's first-column lane (lanes 0-15) solves with its partner's s, a, c and centre
        const double S1 = __shfl_down_sync(0xffffffffu, S, 16);
        const float C1 = __shfl_down_sync(0xffffffffu, C, 16);
        const float mu1 = __shfl_down_sync(0xffffffffu, mu_cur, 16);
        float A1[QM];
#pragma unroll
        for (int k = 0; k < QM; ++k) A1[k] = __shfl_down_sync(0xffffffffu, A[k], 16);
        if (ok && gcol == 0 && snp < p.m) solve_pair<QM>(p, A, A1, C, C1, S, X, S1, mu_cur, mu1, snp);
      } else if (ok && snp < p.m) {
        double v[QM], aPa = 0.0;
#pragma unroll
        for (int k = 0; k < QM; ++k) {
          double acc = 0.0;
          if (k < q) {
#pragma unroll
            for (int l = 0; l < QM; ++l)
              if (l < q) acc += __ldg(&p.P[k * q + l]) * (double)A[l];
            aPa += (double)A[k] * acc;
          }
          v[k] = acc;
        }
        const double sigma = S - aPa;
        const int pp = p.out_snp ? 2 : p.out_var ? (q + 1) + (q + 1) * (q + 2) / 2 : q + 1;
        float* Bo = p.B + (snp * p.t + p.j) * pp;
        if (sigma > 1e-5 * S && p.out_snp) {
          const double bs = (double)C / sigma;
          Bo[0] = (float)bs;
          Bo[1] = (float)(1.0 / sqrt(sigma));  // standard error: Var(b_snp) = 1 / sigma
          if (p.W) p.W[snp * p.t + p.j] = (float)(bs * (double)C);
        } else if (sigma > 1e-5 * S) {
          const double bs = (double)C / sigma;
          double bl[QM];
#pragma unroll
          for (int k = 0; k < QM; ++k) bl[k] = k < q ? __ldg(&p.b0[k]) - v[k] * bs : 0.0;
          // centred SNP x - mu: the intercept (column 0 of X_L) absorbs mu * b_snp
          if (p.centre) bl[0] -= (double)mu_cur * bs;
#pragma unroll
          for (int k = 0; k < QM; ++k)
            if (k < q) Bo[k] = (float)bl[k];
          Bo[q] = (float)bs;
          if (p.W) p.W[snp * p.t + p.j] = (float)(bs * (double)C);
          if (p.out_var) {
            // Var(b) of the centred design, [[P + v v^T / sigma, -v / sigma], [., 1 / sigma]],
            // mapped back to the SNP x = (x - mu) + mu 1: b = T b_c with T = I - mu e_0 e_q^T,
            // so Var(b) = T Var_c T^T changes only row and column 0 (the intercept).  Packed
            // upper triangle, row by row, after the q + 1 coefficients.
            const double inv = 1.0 / sigma, mu = p.centre ? (double)mu_cur : 0.0;
            auto vk = [&](int k) { return v[k < QM ? k : QM - 1]; };  // every index in bounds
            auto vc = [&](int r, int c) -> double {  // r <= c
              if (c < q) return __ldg(&p.P[r * q + c]) + vk(r) * vk(c) * inv;
              return r < q ? -vk(r) * inv : inv;
            };
#pragma unroll
            for (int r = 0; r <= QM; ++r)
#pragma unroll
              for (int c = r; c <= QM; ++c) {
                if (r > q || c > q) continue;
                double x = vc(r, c);
                if (r == 0) x -= mu * (c < q ? -vk(c) * inv : inv);  // - mu Var_c[q][c]
                if (r == 0 && c == 0) x -= mu * vc(0, q) - mu * mu * inv;
                Bo[(q + 1) + r * (q + 1) - r * (r - 1) / 2 + (c - r)] = (float)x;
              }
          }
        } else {
          for (int k = 0; k < pp; ++k) Bo[k] = __int_as_float(0x7fc00000);
          if (p.W) p.W[snp * p.t + p.j] = __int_as_float(0x7fc00000);
          atomicAdd(&p.flags[FLAG_SINGULAR], 1);
        }
      }
      mu_cur = mu_next;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == MMA_WARP) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

}  // namespace

namespace {
int g_max_ctas[64][2];  // per device: co-resident CTAs of each instantiation

template <int QM>
int max_resident_ctas() {
  int per_sm = 0, per_sm8 = 0, dev = 0, sms = 0;
  GW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chol_tc_kernel<QM, 1, 2, false>,
                                                        NUM_THREADS, Layout<false>::SMEM));
  GW_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm8, chol_tc_kernel<QM, 1, 2, true>,
                                                        NUM_THREADS, Layout<true>::SMEM));
  per_sm = per_sm8 < per_sm ? per_sm8 : per_sm;
  GW_REQUIRE(per_sm >= 1, GWAS_ERR_UNSUPPORTED, "the CHOL tensor-core kernel does not fit on an SM");
  GW_CUDA(cudaGetDevice(&dev));
  GW_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return per_sm * sms;
}

int current_device() {
  int dev = 0;
  GW_CUDA(cudaGetDevice(&dev));
  return dev & 63;
}
}  // namespace

template <int QM, int GP, int NP, bool F8 = false>
void set_smem() {
  GW_CUDA(cudaFuncSetAttribute(chol_tc_kernel<QM, GP, NP, F8>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Layout<F8>::SMEM));
}

template <int GP, int NP, bool F8 = false>
void launch_q(unsigned grid, cudaStream_t s, const CholMaps& lmaps, const CUtensorMap& mapG,
              const CholTcParams& p) {
  constexpr size_t SMEM = Layout<F8>::SMEM;
  if (p.q <= 3)
    chol_tc_kernel<3, GP, NP, F8><<<grid, NUM_THREADS, SMEM, s>>>(lmaps, mapG, p);
  else
    chol_tc_kernel<QMAX, GP, NP, F8><<<grid, NUM_THREADS, SMEM, s>>>(lmaps, mapG, p);
}

void chol_tc_prepare() {
  static std::mutex mu;  // setups may run on several host threads at once
  std::lock_guard<std::mutex> lock(mu);
  int* mx = g_max_ctas[current_device()];
  if (mx[0] && mx[1]) return;  // attributes and occupancy belong to the device: once per device
  set_smem<3, 1, 2>();
  set_smem<QMAX, 1, 2>();
  set_smem<3, 2, 2>();
  set_smem<QMAX, 2, 2>();
  set_smem<3, 1, 3>();
  set_smem<QMAX, 1, 3>();
  set_smem<3, 2, 3>();
  set_smem<QMAX, 2, 3>();
  set_smem<3, 1, 2, true>();
  set_smem<QMAX, 1, 2, true>();
  set_smem<3, 2, 2, true>();
  set_smem<QMAX, 2, 2, true>();
  mx[0] = max_resident_ctas<3>();
  mx[1] = max_resident_ctas<QMAX>();
}

int chol_tc_resident_ctas(int q) { return g_max_ctas[current_device()][q <= 3 ? 0 : 1]; }

void chol_tc_launch(cudaStream_t s, const CholMaps& lmaps, const CUtensorMap& mapG,
                    const CholTcParams& p, int num_sms) {
  if (p.m <= 0) return;
  GW_REQUIRE(p.q >= 1 && p.q <= QMAX, GWAS_ERR_ARG, "q=%d outside [1,%d]", p.q, QMAX);
  GW_REQUIRE(p.gp == 1 || p.gp == 2, GWAS_ERR_ARG, "genetic columns %d outside [1,2]", p.gp);
  GW_REQUIRE(p.pieces == 2 || p.pieces == 3, GWAS_ERR_ARG, "split pieces %d outside [2,3]",
             p.pieces);
  // persistent: no more CTAs than fit at once (and no more than the tiles need)
  const int64_t tiles = (p.m + BM / p.gp - 1) / (BM / p.gp);
  int64_t cap = chol_tc_resident_ctas(p.q);
  if (cap <= 0 || cap > num_sms) cap = num_sms;
  const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
  GW_REQUIRE(!p.fp8 || p.pieces == 2, GWAS_ERR_ARG, "the FP8 split has two pieces");
  if (p.fp8 && p.gp == 1)
    launch_q<1, 2, true>(grid, s, lmaps, mapG, p);
  else if (p.fp8)
    launch_q<2, 2, true>(grid, s, lmaps, mapG, p);
  else if (p.gp == 1 && p.pieces == 2)
    launch_q<1, 2>(grid, s, lmaps, mapG, p);
  else if (p.gp == 1)
    launch_q<1, 3>(grid, s, lmaps, mapG, p);
  else if (p.pieces == 2)
    launch_q<2, 2>(grid, s, lmaps, mapG, p);
  else
    launch_q<2, 3>(grid, s, lmaps, mapG, p);
  GW_CHECK_LAUNCH();
}

}  // namespace gw
