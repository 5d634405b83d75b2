// Tensor-core split-BF16 scan (tcgen05 / TMEM / TMA on sm_103a).
#include "tc.cuh"

namespace gw {

struct TcState {
  int algo, n, q, t;
};

void tc_check_supported(int algo, int n, int q, int t) {
  (void)algo; (void)n; (void)q; (void)t;
  GW_REQUIRE(false, GWAS_ERR_UNSUPPORTED, "the split-BF16 tensor-core path is not built yet");
}

TcState* tc_setup(cudaStream_t, const TcSetupArgs&) {
  GW_REQUIRE(false, GWAS_ERR_UNSUPPORTED, "the split-BF16 tensor-core path is not built yet");
  return nullptr;
}

void tc_scan(cudaStream_t, TcState*, const TcScanArgs&) {
  GW_REQUIRE(false, GWAS_ERR_UNSUPPORTED, "the split-BF16 tensor-core path is not built yet");
}

void tc_destroy(TcState* st) { delete st; }

}  // namespace gw
