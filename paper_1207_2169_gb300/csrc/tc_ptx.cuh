// Inline-PTX building blocks for sm_103a: mbarriers, TMA tile loads, tcgen05 MMA / TMEM.
//
// Conventions used by every kernel of this library:
//   * operand tiles are K-major with the 128-byte swizzle (rows of 64 BF16 values, 8-row
//     atoms of 1024 bytes), the layout a TMA load with CU_TENSOR_MAP_SWIZZLE_128B produces;
//   * accumulators are FP32 in tensor memory, M = 128 rows on the 128 TMEM lanes;
//   * every wait is bounded in time: on expiry the kernel records FLAG_TIMEOUT and unwinds.
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <stdint.h>

namespace gw {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// As mbar_try_wait, letting the hardware suspend the thread for up to hint_ns while the phase is
// incomplete (it resumes as soon as the phase completes), so waiting warps do not spin.
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t* bar, uint32_t parity,
                                                      uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Waits for the phase with the given parity to complete.  Gives up after `limit_ns` or when
// *abort is set by another role; returns false then (and sets *abort / the global flag).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort,
                                          int* gflag, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait_suspend(bar, parity, 20000u)) return true;
    if ((it & 63) == 0) {
      if (*abort) return false;
      if (globaltimer_ns() - t0 > limit_ns) {
        *abort = 1;
        atomicExch(gflag, 1);
        return false;
      }
    }
  }
}

// ---------------------------------------------------------------------------- TMA
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int32_t x, int32_t y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// L2 prefetch hint for the bytes of [lo, hi) that lie on whole 16-byte units inside the range
// (bulk prefetch; no data is delivered to the SM).  Issued in pieces of at most 32 KB.
__device__ __forceinline__ void prefetch_l2_range(const void* lo, const void* hi) {
  uintptr_t a = ((uintptr_t)lo + 15) & ~(uintptr_t)15;
  const uintptr_t b = (uintptr_t)hi & ~(uintptr_t)15;
  while (a < b) {
    const uint32_t sz = (uint32_t)(b - a < 32768 ? b - a : 32768);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"(sz) : "memory");
    a += sz;
  }
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Generic-proxy shared-memory writes -> visible to the async proxy (tensor core, TMA).
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------------------- tcgen05
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(const void* tile) {
  const uint64_t addr = smem_u32(tile);
  uint64_t d = 0;
  d |= (addr & 0x3FFFFull) >> 4;        // start address
  d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;     // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;               // fixed 0b001 (descriptor version)
  d |= (uint64_t)2 << 61;               // 128-byte swizzle
  return d;
}

// Shared-memory matrix descriptor: K-major, 64-byte swizzle (rows of 64 bytes: 64 FP8 values),
// 8-row atoms 512 bytes apart.  Within an atom, 16-byte chunk c of row r sits at chunk
// c ^ ((r >> 1) & 3): address bits 4-5 are XORed with bits 7-8, the layout a TMA load with
// CU_TENSOR_MAP_SWIZZLE_64B produces.
__device__ __forceinline__ uint64_t sw64_desc(const void* tile) {
  const uint64_t addr = smem_u32(tile);
  uint64_t d = 0;
  d |= (addr & 0x3FFFFull) >> 4;        // start address
  d |= (uint64_t)1 << 16;               // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;      // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;               // fixed 0b001 (descriptor version)
  d |= (uint64_t)4 << 61;               // 64-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

// Instruction descriptor of kind::f16 with FP16 x FP16 -> FP32 (format code 0 for A and B), both
// K-major.  The same bits describe E4M3 x E4M3 -> FP32 under kind::f8f6f4 (E4M3 is code 0 there).
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// D (FP32, TMEM) (+)= A B^T with 8-bit operands (kind::f8f6f4; K = 32 per instruction, i.e. 32
// bytes of each operand row).  Accumulates into the same TMEM columns as kind::f16 products.
__device__ __forceinline__ void mma_fp8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                        uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// Arrive (once) on an mbarrier when every tcgen05 op issued so far by this thread completes.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// Asynchronous half of tmem_ld32: the registers are valid only after tmem_wait32 on them.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// Waits for every outstanding tcgen05.ld of the thread; the "+r" operands make each use of
// the 32 registers depend on the wait, so no use can be scheduled before it.
__device__ __forceinline__ void tmem_wait32(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                 "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                 "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                 "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes (lane i of the warp gets row i).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  tmem_ld32_async(taddr, r);
  tmem_wait32(r);
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Named barrier among `count` threads (ids 1..15; 0 is __syncthreads).
__device__ __forceinline__ void named_bar(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Four genotype bytes (each 0, 1 or 2) -> four BF16 values (0x0000, 0x3F80, 0x4000) in two
// words, by a byte-permute table lookup: for a pair of genotypes (g0, g1) the selector nibbles
// are (g0, g0+4, g1, g1+4), picking the low byte from {00,80,00} and the high byte from
// {00,3F,40}.  (t * 17 spreads the two genotype bytes of t into nibbles 0 and 2.)  Values
// outside {0,1,2} give unspecified BF16 values; validate_genotypes rejects them.
__device__ __forceinline__ uint2 geno4_to_bf16x4(uint32_t w) {
  constexpr uint32_t LO = 0x00008000u, HI = 0x00403F00u;
  const uint32_t s0 = (w & 0xFFFFu) * 17u + 0x4040u;
  const uint32_t s1 = (w >> 16) * 17u + 0x4040u;
  return make_uint2(__byte_perm(LO, HI, s0), __byte_perm(LO, HI, s1));
}

__device__ __forceinline__ uint4 geno8_to_bf16x8(uint2 w) {
  const uint2 a = geno4_to_bf16x4(w.x), b = geno4_to_bf16x4(w.y);
  return make_uint4(a.x, a.y, b.x, b.y);
}

// 2-bit packed genotypes -> BF16.  For a byte b holding codes c0..c3 (bits 0-1 .. 6-7), the
// pair (c0, c1) becomes the selector value c0 | c1 << 8 (then * 17 + 0x4040 as above), and
// likewise (c2, c3).  LO / HI are the byte tables of the three values (plain: 0x00/0x80/0x00 and
// 0x00/0x3F/0x40; centred: see centred_lut).  Eight bytes -> 32 BF16 values in out[0..3].
__device__ __forceinline__ void packed8_to_bf16x32(uint2 w, uint32_t LO, uint32_t HI,
                                                   uint4 (&out)[4]) {
  uint32_t o[16];
  const uint32_t wd[2] = {w.x, w.y};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int bi = 0; bi < 4; ++bi) {
      const uint32_t b = (wd[h] >> (8 * bi)) & 0xFFu;
      const uint32_t t0 = (b & 3u) | ((b << 6) & 0x300u);
      const uint32_t t1 = ((b >> 4) & 3u) | ((b << 2) & 0x300u);
      o[8 * h + 2 * bi] = __byte_perm(LO, HI, t0 * 17u + 0x4040u);
      o[8 * h + 2 * bi + 1] = __byte_perm(LO, HI, t1 * 17u + 0x4040u);
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) out[i] = make_uint4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
}

constexpr uint32_t GENO_LO = 0x00008000u, GENO_HI = 0x00403F00u;

// Byte tables for centred genotypes g - mu (g = 0, 1, 2): low bytes and high bytes of the
// three BF16 values.  Exact when mu is a multiple of 1/64 in [0, 2].
__device__ __forceinline__ void centred_lut(float mu, uint32_t& lo, uint32_t& hi) {
  lo = 0u;
  hi = 0u;
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn((float)g - mu));
    lo |= (b & 0xFFu) << (8 * g);
    hi |= (b >> 8) << (8 * g);
  }
}

// Byte tables for a coded, centred genotype cd(g) - mu (g = 0, 1, 2), cd(g) = byte g of `code`
// (the genetic model's value for hard call g: 0, 1 or 2).  Exact when mu is a multiple of 1/64 in
// [0, 2].  code = 0x020100 (the allele count) gives centred_lut.
__device__ __forceinline__ void coded_lut(float mu, uint32_t code, uint32_t& lo, uint32_t& hi) {
  lo = 0u;
  hi = 0u;
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const float v = (float)((code >> (8 * g)) & 0xFFu) - mu;
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    lo |= (b & 0xFFu) << (8 * g);
    hi |= (b >> 8) << (8 * g);
  }
}

// Byte table of the uncentred coded genotype cd(g) in E4M3 (g = 0, 1, 2; cd(g) in {0, 1, 2}:
// 0x00, 0x38 = 1.0, 0x40 = 2.0, all exact), byte g; byte 3 (the invalid code) is 0.
__device__ __forceinline__ uint32_t coded_e4m3_table(uint32_t code) {
  uint32_t t = 0u;
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    const uint32_t v = (code >> (8 * g)) & 0xFFu;
    t |= (v == 0u ? 0x00u : v == 1u ? 0x38u : 0x40u) << (8 * g);
  }
  return t;
}

// Sixteen 2-bit genotype codes (one 32-bit word of a packed row, call i in bits 2i..2i+1) ->
// sixteen E4M3 bytes by table lookup, in the order of calls 0 2 4 6 1 3 5 7 8 10 12 14 9 11 13 15:
// w & 0x33333333 holds the even calls one per nibble and (w >> 2) & 0x33333333 the odd ones, so
// each byte permute turns four nibbles into four table bytes.  The 8-bit operand it feeds has
// its K columns stored in the same order within every aligned group of 16 (e4m3_k_slot).
__device__ __forceinline__ uint4 packed16_to_e4m3x16(uint32_t w, uint32_t table) {
  const uint32_t ev = w & 0x33333333u, od = (w >> 2) & 0x33333333u;
  return make_uint4(__byte_perm(table, 0u, ev), __byte_perm(table, 0u, od),
                    __byte_perm(table, 0u, ev >> 16), __byte_perm(table, 0u, od >> 16));
}

// Sixteen E4M3 values (as from packed16_to_e4m3x16) -> sixteen FP16 values v - mu, in the same
// order: each pair of bytes is widened by one e4m3x2 -> f16x2 conversion and mu2 (mu in both
// halves) subtracted.  Exact for v in {0, 1, 2} and mu a multiple of 1/64 in [0, 2].
__device__ __forceinline__ void e4m3x16_to_f16_centred(uint4 e, __half2 mu2, uint4& lo8,
                                                       uint4& hi8) {
  const uint32_t w[4] = {e.x, e.y, e.z, e.w};
  uint32_t o[8];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const __half2_raw r = __nv_cvt_fp8x2_to_halfraw2(
          (__nv_fp8x2_storage_t)((w[i] >> (16 * h)) & 0xFFFFu), __NV_E4M3);
      const __half2 v = __hsub2(__half2(r), mu2);
      o[2 * i + h] = *reinterpret_cast<const uint32_t*>(&v);
    }
  }
  lo8 = make_uint4(o[0], o[1], o[2], o[3]);
  hi8 = make_uint4(o[4], o[5], o[6], o[7]);
}

// Position, within its aligned group of 16 K columns, at which packed16_to_e4m3x16 places call i.
__host__ __device__ constexpr int e4m3_k_slot(int i) {
  return (i & 8) | ((i & 1) << 2) | ((i >> 1) & 3);
}

// Counts of codes 1 and 2 in a word of sixteen 2-bit genotype codes (code 3 counts as neither).
__device__ __forceinline__ void count12(uint32_t w, int& n1, int& n2) {
  const uint32_t lo = w & 0x55555555u, hi = (w >> 1) & 0x55555555u;
  n1 += __popc(lo & ~hi);
  n2 += __popc(hi & ~lo);
}

// The centre of a SNP's coded column from its counts of genotypes 1 and 2 among n: the multiple
// of 1/64 nearest the column mean, clamped to [0, 2] (so that every cd(g) - mu is exact in BF16).
__device__ __forceinline__ float coded_centre(int n1, int n2, int n, uint32_t code) {
  const float c0 = (float)(code & 0xFFu), c1 = (float)((code >> 8) & 0xFFu),
              c2 = (float)((code >> 16) & 0xFFu);
  const float sum = c0 * (float)(n - n1 - n2) + c1 * (float)n1 + c2 * (float)n2;
  const float c = rintf(64.f * sum / (float)n) / 64.f;
  return fminf(fmaxf(c, 0.f), 2.f);
}

__device__ __forceinline__ uint4 geno8_to_bf16x8_lut(uint2 w, uint32_t LO, uint32_t HI) {
  const uint32_t s0 = (w.x & 0xFFFFu) * 17u + 0x4040u, s1 = (w.x >> 16) * 17u + 0x4040u;
  const uint32_t s2 = (w.y & 0xFFFFu) * 17u + 0x4040u, s3 = (w.y >> 16) * 17u + 0x4040u;
  return make_uint4(__byte_perm(LO, HI, s0), __byte_perm(LO, HI, s1), __byte_perm(LO, HI, s2),
                    __byte_perm(LO, HI, s3));
}

// Eight int8 values -> eight BF16 (exact for |v| <= 256) packed in a uint4.
__device__ __forceinline__ uint4 i8x8_to_bf16x8(uint2 w) {
  uint32_t o[4];
  const uint32_t src[2] = {w.x, w.y};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int pr = 0; pr < 2; ++pr) {
      const int b0 = (int)(int8_t)((src[h] >> (16 * pr)) & 0xFF);
      const int b1 = (int)(int8_t)((src[h] >> (16 * pr + 8)) & 0xFF);
      o[2 * h + pr] = (__float_as_uint((float)b0) >> 16) | (__float_as_uint((float)b1) & 0xFFFF0000u);
    }
  }
  return make_uint4(o[0], o[1], o[2], o[3]);
}

}  // namespace tc
}  // namespace gw
