// Launch counting and optional per-kernel CUDA-event timing.  Every kernel
// launch site in the library opens a ProfScope; when timing is enabled the
// scope records an event pair on the launch stream, and the totals are read
// back per kernel name.  Off by default (counting only).
#include "common.cuh"

#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

namespace nexel {

namespace {
struct Rec {
  const char* name;
  cudaEvent_t a, b;
};
std::atomic<long long> g_launches{0};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

ProfScope::ProfScope(const char* name, cudaStream_t st) : name_(name), st_(st), a_(nullptr) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  a_ = get_event();
  cudaEventRecord((cudaEvent_t)a_, st_);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = get_event();
  cudaEventRecord(b, st_);
  g_recs.push_back({name_, (cudaEvent_t)a_, b});
}

}  // namespace nexel

using namespace nexel;

extern "C" {

long long nexel_launch_count(void) { return g_launches.load(); }

int nexel_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = on != 0;
  for (auto& r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  return NEXEL_OK;
}

int nexel_profile_read(int max_entries, char* names, float* total_ms, int* launches,
                       int* n_out) {
  if (max_entries < 0 || !n_out) return NEXEL_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_mu);
  std::vector<const char*> keys;
  std::vector<double> tot;
  std::vector<int> cnt;
  for (auto& r : g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return NEXEL_ERR_CUDA;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return NEXEL_ERR_CUDA;
    size_t k = 0;
    while (k < keys.size() && std::strcmp(keys[k], r.name) != 0) ++k;
    if (k == keys.size()) {
      keys.push_back(r.name);
      tot.push_back(0.0);
      cnt.push_back(0);
    }
    tot[k] += ms;
    cnt[k] += 1;
  }
  int n = (int)keys.size();
  *n_out = n;
  for (int k = 0; k < n && k < max_entries; ++k) {
    if (names) {
      std::strncpy(names + 32 * k, keys[k], 31);
      names[32 * k + 31] = 0;
    }
    if (total_ms) total_ms[k] = (float)tot[k];
    if (launches) launches[k] = cnt[k];
  }
  return NEXEL_OK;
}

}  // extern "C"
