// Self-test of the bounded waits every tensor-core kernel uses: one thread waits on an mbarrier
// phase that nothing completes, with a short limit, and must give up, record FLAG_TIMEOUT and
// return -- the GPU context stays usable.  No fault, trap or endless loop is involved.
#include "common.cuh"
#include "tc_ptx.cuh"

namespace gw {
namespace {

__global__ void wait_timeout_kernel(int* flags, uint64_t limit_ns, int* result) {
  __shared__ uint64_t bar;
  __shared__ int abort_;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);  // one arrival would complete phase 0; none comes
    abort_ = 0;
    tc::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const bool completed = tc::mbar_wait(&bar, 0, &abort_, flags + FLAG_TIMEOUT, limit_ns);
    *result = completed ? 1 : 0;
  }
}

}  // namespace

gwas_status selftest_wait_timeout(int limit_ms) {
  int* d = nullptr;
  GW_CUDA(cudaMalloc(&d, sizeof(int) * (FLAG_COUNT + 1)));
  int h[FLAG_COUNT + 1] = {0};
  cudaError_t e = cudaMemset(d, 0, sizeof(int) * (FLAG_COUNT + 1));
  if (e == cudaSuccess) {
    wait_timeout_kernel<<<1, 32>>>(d, (uint64_t)limit_ms * 1000000ull, d + FLAG_COUNT);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) {
    set_error("self-test launch failed: %s", cudaGetErrorString(e));
    return GWAS_ERR_CUDA;
  }
  if (h[FLAG_COUNT] != 0 || h[FLAG_TIMEOUT] != 1) {
    set_error("self-test: the wait did not give up as designed (completed=%d flag=%d)",
              h[FLAG_COUNT], h[FLAG_TIMEOUT]);
    return GWAS_ERR_CUDA;
  }
  set_error("bounded wait gave up after %d ms (self-test)", limit_ms);
  return GWAS_ERR_TIMEOUT;
}

}  // namespace gw
