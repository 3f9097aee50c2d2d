// Launch counting and optional per-kernel CUDA-event timing.  Every kernel
// launch site in the library opens a ProfScope; when timing is enabled the
// scope records an event pair on the launch stream, and the totals are read
// back per kernel name.  Off by default (counting only).
#include "common.cuh"

#include <algorithm>
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
// Random float2 reductions into an L2-resident table: the index of
// reduction i is a 32-bit integer hash of (i, salt) (xorshift-multiply
// rounds with odd multipliers) masked to the table size.
__device__ __forceinline__ uint32_t probe_hash(uint32_t x) {
  x ^= x >> 15;
  x *= 0x2c1b3c6dU;
  x ^= x >> 12;
  x *= 0x297a2d39U;
  x ^= x >> 15;
  return x;
}

__global__ void __launch_bounds__(256) k_peak_red(float2* __restrict__ tab, uint32_t mask,
                                                  long long n, uint32_t salt) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    atomicAdd(tab + (probe_hash((uint32_t)i ^ salt) & mask), make_float2(1.f, 1.f));
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

int nexel_peak_l2_reductions(void* buf, size_t buf_bytes, long long n_ops, int reps,
                             float* gops_out, nexel_stream_t stream) {
  if (!buf || !gops_out || n_ops < 1 || reps < 1 || reps > 100 || buf_bytes < 8 ||
      (reinterpret_cast<uintptr_t>(buf) & 7) != 0)
    return NEXEL_ERR_INVALID_ARG;
  // the largest power-of-two count of float2 entries that fits the buffer
  uint32_t entries = 1;
  while ((size_t)entries * 2 * 8 <= buf_bytes && entries < (1u << 31)) entries <<= 1;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return NEXEL_ERR_CUDA;
  }
  cudaError_t e = cudaMemsetAsync(buf, 0, (size_t)entries * 8, st);
  std::vector<float> ms;
  for (int r = 0; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(a, st);
    if (e != cudaSuccess) break;
    {
      ProfScope ps("peak_l2_reductions", st);
      k_peak_red<<<nsm * 8, 256, 0, st>>>((float2*)buf, entries - 1, n_ops, (uint32_t)r * 0x9e3779b9u);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float x = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&x, a, b);
    ms.push_back(x);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e != cudaSuccess) return NEXEL_ERR_CUDA;
  std::sort(ms.begin(), ms.end());
  const float med = ms[ms.size() / 2];
  *gops_out = med > 0.f ? (float)((double)n_ops / (med * 1e-3) / 1e9) : 0.f;
  return NEXEL_OK;
}

}  // extern "C"
