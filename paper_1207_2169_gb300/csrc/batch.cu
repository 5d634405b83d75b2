// Batched scans of several cohorts (gwas_setup_batch / gwas_scan_batch): one CUDA graph per
// block shape, whose launch plan is chosen by timing the candidates on the first call.
//
// Each cohort keeps its own handle (its own n, q, t, kinship and traits); a batch scan runs the
// tensor-core scan of every cohort on its block of packed genotypes.  Small cohorts cannot fill
// the GPU on their own, so the plans differ in how the cohorts' persistent kernels share the SMs:
//   0  one after another on one stream, each with every SM;
//   1  all at once, one stream each, each kernel capped at an SM share proportional to its work;
//   2  all at once, one stream each, every kernel with every SM (the hardware interleaves CTAs);
//   3  two lanes of half the SMs each, cohorts assigned longest first to the less loaded lane.
// Each plan is timed with the EIG cohorts' internal SNP chunk (one ROT, SQ and AC launch per
// chunk) at its capacity, half and a quarter of it: shorter launches interleave better when the
// cohorts share the SMs, longer ones waste less at launch boundaries when they run alone.
#include <algorithm>
#include <atomic>
#include <thread>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

#define GW_API extern "C" __attribute__((visibility("default")))

namespace gw {
TcState* handle_tc(gwas_handle h);
int handle_device(gwas_handle h);
int* handle_flags(gwas_handle h);
int handle_n(gwas_handle h);
int handle_t(gwas_handle h);
int handle_p(gwas_handle h);
}  // namespace gw

using namespace gw;

namespace {
constexpr int NPLANS = 4;
constexpr int NCHUNK = 3;  // EIG chunk = capacity / 2^i, i < NCHUNK
}

struct gwas_batch_s {
  int dev = 0, num_sms = 0;
  std::vector<gwas_handle> h;
  std::vector<cudaStream_t> side;
  cudaStream_t cap = nullptr;  // graphs are captured here (the caller's stream may be the legacy one)
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
  // the graph of the current block shape
  std::vector<int64_t> shape;  // m per cohort
  int plan = -1, chunk_div = 0;  // chosen plan; chosen chunk = capacity >> chunk_div
  double plan_ms[NCHUNK][NPLANS] = {};
  cudaGraphExec_t exec = nullptr;
};

namespace {

void destroy_batch(gwas_batch b) {
  if (!b) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(b->dev);
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (cudaStream_t s : b->side) cudaStreamDestroy(s);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (cudaEvent_t e : b->ev_join) cudaEventDestroy(e);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->ev_t0) cudaEventDestroy(b->ev_t0);
  if (b->ev_t1) cudaEventDestroy(b->ev_t1);
  for (gwas_handle h : b->h) gwas_destroy(h);
  delete b;
  cudaSetDevice(cur);
}

// The scans of every cohort under plan `plan`, issued on `s` (the batch's capture stream) and on
// the batch's side streams forked from it.
void issue_plan(gwas_batch b, const gwas_cohort_block* blk, int plan, cudaStream_t s) {
  const int k = (int)b->h.size();
  std::vector<double> work(k);
  double total = 0.0;
  for (int i = 0; i < k; ++i) {
    work[i] = blk[i].m > 0 ? tc_scan_work(handle_tc(b->h[i]), blk[i].m) : 0.0;
    total += work[i];
  }
  auto scan = [&](int i, cudaStream_t st, int max_ctas) {
    if (blk[i].m <= 0) return;
    TcScanArgs a{};
    a.G = blk[i].G;
    a.m = blk[i].m;
    a.B = blk[i].B;
    a.wald = blk[i].wald;
    a.flags = handle_flags(b->h[i]);
    a.max_ctas = max_ctas;
    tc_scan(st, handle_tc(b->h[i]), a);
  };
  if (plan == 0) {
    for (int i = 0; i < k; ++i) scan(i, s, 0);
    return;
  }
  // lanes: plan 1 and 2 one per cohort, plan 3 two
  const int lanes = plan == 3 ? std::min(2, k) : k;
  GW_CUDA(cudaEventRecord(b->ev_fork, s));
  for (int l = 0; l < lanes; ++l) GW_CUDA(cudaStreamWaitEvent(b->side[l], b->ev_fork, 0));
  if (plan == 3) {
    std::vector<int> order(k);
    for (int i = 0; i < k; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int x, int y) { return work[x] > work[y]; });
    double load[2] = {0.0, 0.0};
    const int half = std::max(2, b->num_sms / 2 / 2 * 2);
    for (int i : order) {
      const int l = lanes == 2 && load[1] < load[0] ? 1 : 0;
      load[l] += work[i];
      scan(i, b->side[l], lanes == 2 ? half : 0);
    }
  } else {
    for (int i = 0; i < k; ++i) {
      int cap = 0;
      if (plan == 1 && total > 0.0) {
        cap = (int)(b->num_sms * work[i] / total + 0.5);
        cap = std::max(2, std::min(b->num_sms, cap / 2 * 2));
      }
      scan(i, b->side[i], cap);
    }
  }
  for (int l = 0; l < lanes; ++l) {
    GW_CUDA(cudaEventRecord(b->ev_join[l], b->side[l]));
    GW_CUDA(cudaStreamWaitEvent(s, b->ev_join[l], 0));
  }
}

cudaGraph_t capture_plan(gwas_batch b, const gwas_cohort_block* blk, int plan) {
  cudaStream_t s = b->cap;
  GW_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  try {
    issue_plan(b, blk, plan, s);
  } catch (...) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(s, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  cudaGraph_t g = nullptr;
  GW_CUDA(cudaStreamEndCapture(s, &g));
  return g;
}

cudaGraphExec_t instantiate(cudaGraph_t g) {
  cudaGraphExec_t e = nullptr;
  GW_CUDA(cudaGraphInstantiate(&e, g, 0));
  return e;
}

gwas_status scan_batch_impl(gwas_batch b, const gwas_cohort_block* blk, cudaStream_t s) {
  GW_REQUIRE(b != nullptr && blk != nullptr, GWAS_ERR_ARG, "null batch or blocks");
  const int k = (int)b->h.size();
  std::vector<int64_t> shape(k);
  for (int i = 0; i < k; ++i) {
    GW_REQUIRE(blk[i].m >= 0, GWAS_ERR_ARG, "cohort %d: m < 0", i);
    if (blk[i].m == 0) continue;
    GW_REQUIRE(blk[i].G != nullptr && blk[i].B != nullptr, GWAS_ERR_ARG,
               "cohort %d: null genotypes or B", i);
    GW_REQUIRE(((uintptr_t)blk[i].G & 15) == 0, GWAS_ERR_ARG,
               "cohort %d: packed genotypes must start on a 16-byte boundary", i);
    shape[i] = blk[i].m;
  }
  int cur = 0;
  GW_CUDA(cudaGetDevice(&cur));
  GW_CUDA(cudaSetDevice(b->dev));
  try {
    if (b->exec && shape == b->shape) {
      // same shape, possibly new buffers: re-capture the chosen plan and update the graph
      cudaGraph_t g = capture_plan(b, blk, b->plan);
      cudaGraphExecUpdateResultInfo info;
      const cudaError_t e = cudaGraphExecUpdate(b->exec, g, &info);
      if (e != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(b->exec);
        b->exec = instantiate(g);
      }
      cudaGraphDestroy(g);
      GW_CUDA(cudaGraphLaunch(b->exec, s));
    } else {
      // new shape: time every plan once (after one untimed replay) and keep the fastest
      if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
      }
      double best = 0.0;
      auto set_chunks = [&](int div) {
        for (gwas_handle h : b->h) {
          TcState* st = handle_tc(h);
          tc_set_eig_chunk(st, tc_eig_chunk_capacity(st) >> div);
        }
      };
      for (int div = 0; div < NCHUNK; ++div) {
        set_chunks(div);
        for (int plan = 0; plan < NPLANS; ++plan) {
          cudaGraph_t g = capture_plan(b, blk, plan);
          cudaGraphExec_t e = instantiate(g);
          cudaGraphDestroy(g);
          GW_CUDA(cudaGraphLaunch(e, s));
          GW_CUDA(cudaEventRecord(b->ev_t0, s));
          GW_CUDA(cudaGraphLaunch(e, s));
          GW_CUDA(cudaEventRecord(b->ev_t1, s));
          GW_CUDA(cudaEventSynchronize(b->ev_t1));
          float ms = 0.f;
          GW_CUDA(cudaEventElapsedTime(&ms, b->ev_t0, b->ev_t1));
          b->plan_ms[div][plan] = ms;
          if (!b->exec || ms < best) {
            if (b->exec) cudaGraphExecDestroy(b->exec);
            b->exec = e;
            b->plan = plan;
            b->chunk_div = div;
            best = ms;
          } else {
            cudaGraphExecDestroy(e);
          }
        }
      }
      set_chunks(b->chunk_div);  // later re-captures of this shape use the chosen chunks
      b->shape = shape;
    }
  } catch (...) {
    cudaSetDevice(cur);
    throw;
  }
  GW_CUDA(cudaSetDevice(cur));
  return GWAS_OK;
}

}  // namespace

GW_API gwas_status gwas_setup_batch(int n_cohorts, const gwas_cohort* cohorts,
                                    const gwas_options* opt, gwas_batch* out) {
  if (out) *out = nullptr;
  gwas_batch b = nullptr;
  try {
    GW_REQUIRE(out != nullptr && cohorts != nullptr, GWAS_ERR_ARG, "null cohorts or out");
    GW_REQUIRE(n_cohorts >= 1 && n_cohorts <= 256, GWAS_ERR_ARG, "n_cohorts=%d outside [1,256]",
               n_cohorts);
    gwas_options o;
    gwas_default_options(&o);
    if (opt) o = *opt;
    GW_REQUIRE(o.precision == GWAS_PREC_SPLIT_BF16 || o.precision == GWAS_PREC_SPLIT_FP8,
               GWAS_ERR_UNSUPPORTED,
               "batched scans run the tensor-core path (precision SPLIT_BF16 or SPLIT_FP8)");
    b = new gwas_batch_s();
    b->dev = o.device;
    // The cohorts' setups (FP64 eigendecompositions and per-trait packs, each on its handle's
    // own streams) run on up to 8 host threads at once: a small cohort alone leaves most of the
    // GPU idle.  The first failure (lowest cohort index) is reported.
    b->h.assign(n_cohorts, nullptr);
    std::vector<gwas_status> sts(n_cohorts, GWAS_OK);
    std::vector<std::string> msgs(n_cohorts);
    std::atomic<int> next{0};
    auto worker = [&]() {
      for (int i = next++; i < n_cohorts; i = next++) {
        const gwas_cohort& c = cohorts[i];
        gwas_handle h = nullptr;
        sts[i] = gwas_setup(c.Phi, c.n, c.XL, c.q, c.Y, c.t, c.h2, c.s2, &o, &h);
        if (sts[i] != GWAS_OK) msgs[i] = gwas_last_error();
        b->h[i] = h;
      }
    };
    const int nthreads = n_cohorts < 8 ? n_cohorts : 8;
    std::vector<std::thread> pool;
    for (int k = 1; k < nthreads; ++k) pool.emplace_back(worker);
    worker();
    for (auto& th : pool) th.join();
    for (int i = 0; i < n_cohorts; ++i)
      if (sts[i] != GWAS_OK) {
        set_error("cohort %d: %s", i, msgs[i].c_str());
        throw Fail{sts[i]};
      }
    int cur = 0;
    GW_CUDA(cudaGetDevice(&cur));
    GW_CUDA(cudaSetDevice(b->dev));
    GW_CUDA(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->dev));
    b->side.resize(n_cohorts);
    b->ev_join.resize(n_cohorts);
    for (int i = 0; i < n_cohorts; ++i) {
      GW_CUDA(cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking));
      GW_CUDA(cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming));
    }
    GW_CUDA(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    GW_CUDA(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming));
    GW_CUDA(cudaEventCreate(&b->ev_t0));
    GW_CUDA(cudaEventCreate(&b->ev_t1));
    GW_CUDA(cudaSetDevice(cur));
    *out = b;
    set_error("%s", "");
    return GWAS_OK;
  } catch (const Fail& f) {
    destroy_batch(b);
    return f.st;
  } catch (...) {
    destroy_batch(b);
    set_error("unexpected C++ exception in gwas_setup_batch");
    return GWAS_ERR_CUDA;
  }
}

GW_API gwas_status gwas_scan_batch(gwas_batch b, const gwas_cohort_block* blocks, void* stream) {
  try {
    return scan_batch_impl(b, blocks, (cudaStream_t)stream);
  } catch (const Fail& f) {
    return f.st;
  } catch (...) {
    set_error("unexpected C++ exception in gwas_scan_batch");
    return GWAS_ERR_CUDA;
  }
}

GW_API gwas_status gwas_batch_plan(gwas_batch b, int* plan, double* plan_ms) {
  if (!b) {
    set_error("null batch");
    return GWAS_ERR_ARG;
  }
  if (plan) *plan = b->plan;
  if (plan_ms)
    for (int i = 0; i < NPLANS; ++i) plan_ms[i] = b->plan_ms[b->chunk_div][i];
  return GWAS_OK;
}

GW_API gwas_status gwas_batch_tuning(gwas_batch b, int* plan, int* chunk_div, double* ms) {
  if (!b) {
    set_error("null batch");
    return GWAS_ERR_ARG;
  }
  if (plan) *plan = b->plan;
  if (chunk_div) *chunk_div = b->chunk_div;
  if (ms)
    for (int d = 0; d < NCHUNK; ++d)
      for (int i = 0; i < NPLANS; ++i) ms[d * NPLANS + i] = b->plan_ms[d][i];
  return GWAS_OK;
}

GW_API gwas_handle gwas_batch_handle(gwas_batch b, int i) {
  if (!b || i < 0 || i >= (int)b->h.size()) return nullptr;
  return b->h[i];
}

GW_API void gwas_destroy_batch(gwas_batch b) { destroy_batch(b); }
