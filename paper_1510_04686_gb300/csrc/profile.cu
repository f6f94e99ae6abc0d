// Launch accounting and event timing behind negf_profile_* (see include/negf.h).
#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "profile.cuh"
#include "tc_gemm.cuh"

namespace negf {
namespace {
std::atomic<long long> g_launches{0};
std::atomic<int> g_prof{0};
std::mutex g_mu;
struct Pending {
  cudaEvent_t a, b;
  int kind;
};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
cudaEvent_t g_open[PROF_KINDS] = {};
long long g_count[PROF_KINDS] = {};
double g_ms[PROF_KINDS] = {};
double g_alg[PROF_KINDS] = {};
double g_hw[PROF_KINDS] = {};

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}
}  // namespace

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

namespace {
std::atomic<int> g_last_err{0};
}
cudaError_t note_error(cudaError_t e) {
  if (e != cudaSuccess) g_last_err.store((int)e);
  return e;
}
bool profiling_on() { return g_prof.load(std::memory_order_relaxed) != 0; }

void prof_begin(cudaStream_t s, int kind) {
  if (!profiling_on()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t e = get_event();
  if (e && cudaEventRecord(e, s) == cudaSuccess) g_open[kind] = e;
}
void prof_flops(int kind, double alg, double hw) {
  if (!profiling_on()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  g_alg[kind] += alg;
  g_hw[kind] += hw;
}

void prof_end(cudaStream_t s, int kind) {
  if (!profiling_on()) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t a = g_open[kind];
  if (!a) return;
  g_open[kind] = nullptr;
  cudaEvent_t b = get_event();
  if (b && cudaEventRecord(b, s) == cudaSuccess) g_pending.push_back(Pending{a, b, kind});
}

}  // namespace negf

using namespace negf;

extern "C" {

void negf_profile_enable(int32_t on) { g_prof.store(on ? 1 : 0); }

const char* negf_last_cuda_error(void) {
  return cudaGetErrorName(static_cast<cudaError_t>(g_last_err.load()));
}

long long negf_launch_count(void) { return g_launches.load(); }

negf_status negf_profile_read(int32_t kind, long long* launches, double* total_ms) {
  if (kind < 0 || kind >= PROF_KINDS || !launches || !total_ms) return NEGF_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  std::vector<Pending> keep;
  for (const Pending& p : g_pending) {
    if (cudaEventSynchronize(p.b) != cudaSuccess) return NEGF_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) != cudaSuccess) return NEGF_ERR_CUDA;
    g_count[p.kind] += 1;
    g_ms[p.kind] += ms;
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
  *launches = g_count[kind];
  *total_ms = g_ms[kind];
  return NEGF_OK;
}

void negf_profile_reset(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  tc_prof_reset();
  for (int k = 0; k < PROF_KINDS; ++k) {
    g_count[k] = 0;
    g_ms[k] = 0.0;
    g_alg[k] = 0.0;
    g_hw[k] = 0.0;
  }
}

negf_status negf_profile_flops(int32_t kind, double* algorithmic, double* hardware) {
  if (kind < 0 || kind >= PROF_KINDS || !algorithmic || !hardware) return NEGF_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  if (kind == PROF_TC_GEMM) {  // counted on the device, for the batch items that ran
    if (tc_prof_flops(algorithmic, hardware) != cudaSuccess) return NEGF_ERR_CUDA;
    return NEGF_OK;
  }
  *algorithmic = g_alg[kind];
  *hardware = g_hw[kind];
  return NEGF_OK;
}

}  // extern "C"
