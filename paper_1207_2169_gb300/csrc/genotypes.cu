// Genotype formats: int8 hard calls and 2-bit packed codes.
//
// Packed layout (GWAS_GENO_PACKED2): SNP i occupies row_bytes = ceil(n / 64) * 16 bytes at
// XR + i * row_bytes; genotype k sits in byte k / 4, bits 2 (k % 4) .. 2 (k % 4) + 1, holding the
// allele count 0, 1 or 2 (3 is invalid); codes for k >= n are 0.  Rows are whole 16-byte units,
// so the tensor-core kernels fetch 64-genotype slices of 128 SNPs as one TMA box.
#include "common.cuh"

namespace gw {
namespace {

// Four int8 calls (one 32-bit word) -> four 2-bit codes in the low byte; a byte outside
// {0, 1, 2} (including negative ones) becomes code 3 and sets *bad.
__device__ __forceinline__ uint32_t pack4(uint32_t x, bool& bad) {
  const uint32_t big = (x | ((x & 0x7F7F7F7Fu) + 0x7D7D7D7Du)) & 0x80808080u;  // byte >= 3
  bad |= big != 0u;
  const uint32_t v = (x & 0x03030303u) | (big >> 6) | (big >> 7);
  const uint32_t t = v | (v >> 6);  // codes 0,1 in bits 0-3, codes 2,3 in bits 16-19
  return (t & 0xFu) | ((t >> 12) & 0xF0u);
}

// One thread per 32-bit word of packed output (16 calls).  Rows whose start is 8-byte aligned
// (n a multiple of 8) are read as two 8-byte words per thread.
__global__ void pack2_kernel(const int8_t* __restrict__ x, int64_t m, int n, int row_bytes,
                             uint32_t* __restrict__ out, int* flags, int validate) {
  const int words = row_bytes / 4;
  const int64_t total = m * words;
  const bool vec = (n % 8 == 0) && ((reinterpret_cast<uintptr_t>(x) & 7) == 0);
  bool bad = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t snp = e / words;
    const int k0 = (int)(e % words) * 16;
    const int8_t* row = x + snp * n;
    uint32_t w = 0;
    if (vec && k0 + 16 <= n) {
      const uint2 a = __ldg(reinterpret_cast<const uint2*>(row + k0));
      const uint2 b = __ldg(reinterpret_cast<const uint2*>(row + k0 + 8));
      w = pack4(a.x, bad) | pack4(a.y, bad) << 8 | pack4(b.x, bad) << 16 | pack4(b.y, bad) << 24;
    } else if (vec && k0 + 8 <= n) {
      const uint2 a = __ldg(reinterpret_cast<const uint2*>(row + k0));
      w = pack4(a.x, bad) | pack4(a.y, bad) << 8;
    } else if (k0 < n) {
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int k = k0 + i;
        if (k < n) {
          const uint32_t g = (uint8_t)row[k];
          bad |= g > 2;
          w |= (g > 2 ? 3u : g) << (2 * i);  // invalid values become the invalid code 3
        }
      }
    }
    out[e] = w;
  }
  if (validate && __syncthreads_or(bad) && threadIdx.x == 0) atomicExch(&flags[FLAG_GENOTYPE], 1);
}

__global__ void unpack2_kernel(const uint8_t* __restrict__ in, int64_t m, int n, int row_bytes,
                               int8_t* __restrict__ out) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t snp = e / n;
    const int k = (int)(e % n);
    out[e] = (int8_t)((in[snp * row_bytes + k / 4] >> (2 * (k % 4))) & 3u);
  }
}

// Packed codes must be 0, 1 or 2, and 0 past the n-th genotype of a row.
__global__ void validate_packed_kernel(const uint32_t* __restrict__ in, int64_t m, int n,
                                       int row_bytes, int* flags) {
  const int words = row_bytes / 4;
  const int64_t total = m * words;
  bool bad = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t w = in[e];
    bad |= (w & (w >> 1) & 0x55555555u) != 0u;  // a code 3
    const int k0 = (int)(e % words) * 16;
    if (k0 + 16 > n) {
      const int keep = n - k0 > 0 ? n - k0 : 0;  // valid codes in this word
      const uint32_t mask = keep >= 16 ? 0u : ~0u << (2 * keep);
      bad |= (w & mask) != 0u;
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(&flags[FLAG_GENOTYPE], 1);
}

// mu[i pr + k] = nearest multiple of 1/64 to the mean of SNP i's coded column k (coding word
// code_k: the values of genotypes 0, 1, 2 in bytes 0, 1, 2), clamped to [0, 2], from packed
// codes (one warp per SNP).
__global__ void centres_packed_kernel(const uint32_t* __restrict__ in, int64_t m, int n,
                                      int row_bytes, float* __restrict__ mu, int pr,
                                      uint32_t code0, uint32_t code1) {
  const int64_t snp = blockIdx.x * (int64_t)(blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x % 32;
  if (snp >= m) return;
  const int words = row_bytes / 4;
  const uint32_t* row = in + snp * words;
  int n1 = 0, n2 = 0;  // genotypes 1 and 2 (padding codes past n are 0)
  for (int w = lane; w < words; w += 32) {
    const uint32_t v = row[w];
    const uint32_t lo = v & 0x55555555u, hi = (v >> 1) & 0x55555555u;
    n1 += __popc(lo & ~hi);
    n2 += __popc(hi & ~lo);
  }
  for (int o = 16; o > 0; o >>= 1) {
    n1 += __shfl_xor_sync(0xffffffffu, n1, o);
    n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  }
  if (lane < pr) {
    const uint32_t code = lane == 0 ? code0 : code1;
    const float sum = (float)(code & 0xFFu) * (float)(n - n1 - n2) +
                      (float)((code >> 8) & 0xFFu) * (float)n1 + (float)((code >> 16) & 0xFFu) * (float)n2;
    const float c = rintf(64.f * sum / (float)n) / 64.f;
    mu[snp * pr + lane] = fminf(fmaxf(c, 0.f), 2.f);
  }
}

}  // namespace

int packed_row_bytes(int n) { return ((n + 63) / 64) * 16; }

void pack_genotypes(cudaStream_t s, const int8_t* x, int64_t m, int n, uint8_t* out, int* flags,
                    bool validate) {
  if (m <= 0) return;
  pack2_kernel<<<2368, 256, 0, s>>>(x, m, n, packed_row_bytes(n), (uint32_t*)out, flags,
                                    validate ? 1 : 0);
  GW_CHECK_LAUNCH();
}

void unpack_genotypes(cudaStream_t s, const uint8_t* in, int64_t m, int n, int8_t* out) {
  if (m <= 0) return;
  unpack2_kernel<<<2368, 256, 0, s>>>(in, m, n, packed_row_bytes(n), out);
  GW_CHECK_LAUNCH();
}

void validate_packed(cudaStream_t s, const uint8_t* in, int64_t m, int n, int* flags) {
  if (m <= 0) return;
  validate_packed_kernel<<<1184, 256, 0, s>>>((const uint32_t*)in, m, n, packed_row_bytes(n),
                                              flags);
  GW_CHECK_LAUNCH();
}

void snp_centres_packed(cudaStream_t s, const uint8_t* in, int64_t m, int n, float* mu, int pr,
                        const uint32_t* code) {
  if (m <= 0) return;
  centres_packed_kernel<<<(unsigned)((m + 7) / 8), 256, 0, s>>>(
      (const uint32_t*)in, m, n, packed_row_bytes(n), mu, pr, code[0], pr > 1 ? code[1] : 0u);
  GW_CHECK_LAUNCH();
}

}  // namespace gw

// ------------------------------------------------------------------------------------------
// p-values of Wald statistics: the chi-square(1) upper tail erfc(sqrt(w / 2))
// ------------------------------------------------------------------------------------------
namespace gw {
namespace {
// chi-square upper tail: dof 1 -> erfc(sqrt(x / 2)), dof 2 -> exp(-x / 2)
__global__ void pvalue_kernel(const float* __restrict__ w, int64_t count, int dof,
                              float* __restrict__ pv) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float x = w[e];
    pv[e] = x >= 0.f ? (dof == 2 ? expf(-0.5f * x) : erfcf(sqrtf(0.5f * x))) : (x == x ? 1.f : x);
  }
}
}  // namespace

void wald_pvalues(cudaStream_t s, const float* w, int64_t count, int dof, float* pv) {
  if (count <= 0) return;
  pvalue_kernel<<<1184, 256, 0, s>>>(w, count, dof, pv);
  GW_CHECK_LAUNCH();
}
}  // namespace gw
