// Batched multi-view entry points: one training step over several views of
// the same scene (uneven resolutions), issued without a host
// synchronisation, so that a caller can capture the whole step in one CUDA
// graph and replay it.
//
// Each view keeps its own workspaces; its preprocess uses the device-count
// form (the instance count never leaves the device; the workspace capacity
// bounds it and an overflow is flagged in the view's status word).  The
// views run as parallel branches forked from the caller's stream onto a
// per-device pool of streams and joined back into it, so that small views
// and latency-bound kernels of different views overlap on the GPU.  The
// surfel, table and MLP gradients of all views are summed with atomics.
#include "common.cuh"

#include <mutex>

namespace nexel {
namespace {

constexpr int kMaxDevices = 64;
constexpr int kBranches = 8;

struct Pool {
  bool ready = false;
  cudaStream_t s[kBranches] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kBranches] = {};
};

std::mutex g_pool_mu;
Pool g_pool[kMaxDevices];

// The current device's branch streams and events, created on first use.
// Creating them is not a stream operation, so it is also legal while the
// caller's stream is being captured.
int get_pool(Pool** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return NEXEL_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return NEXEL_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  Pool& p = g_pool[dev];
  if (!p.ready) {
    for (int b = 0; b < kBranches; ++b) {
      if (!p.s[b] && cudaStreamCreateWithFlags(&p.s[b], cudaStreamNonBlocking) != cudaSuccess)
        return NEXEL_ERR_CUDA;
      if (!p.join[b] && cudaEventCreateWithFlags(&p.join[b], cudaEventDisableTiming) != cudaSuccess)
        return NEXEL_ERR_CUDA;
    }
    if (!p.fork && cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming) != cudaSuccess)
      return NEXEL_ERR_CUDA;
    p.ready = true;
  }
  *out = &p;
  return NEXEL_OK;
}

// Fork: every branch used waits for what the caller's stream has queued.
int fork_branches(Pool* p, int n_branches, cudaStream_t st) {
  if (cudaEventRecord(p->fork, st) != cudaSuccess) return NEXEL_ERR_CUDA;
  for (int b = 0; b < n_branches; ++b)
    if (cudaStreamWaitEvent(p->s[b], p->fork, 0) != cudaSuccess) return NEXEL_ERR_CUDA;
  return NEXEL_OK;
}

// Join: the caller's stream waits for every branch used (always called
// after a fork, also on an error path, so that a capture stays joined).
int join_branches(Pool* p, int n_branches, cudaStream_t st) {
  int rc = NEXEL_OK;
  for (int b = 0; b < n_branches; ++b) {
    if (cudaEventRecord(p->join[b], p->s[b]) != cudaSuccess ||
        cudaStreamWaitEvent(st, p->join[b], 0) != cudaSuccess)
      rc = NEXEL_ERR_CUDA;
  }
  return rc;
}

template <typename T>
T at(T const* arr, int v) {
  return arr ? arr[v] : nullptr;
}

}  // namespace
}  // namespace nexel

using namespace nexel;

extern "C" {

int nexel_render_batch_fwd(int n_views, const nexel_camera* cams, const nexel_settings* settings,
                           const nexel_field* field, int N, const float* mu, const float* quat,
                           const float* scale, const float* opacity, const float* gamma,
                           const float* color, void* const* ws, const size_t* ws_bytes,
                           void* const* bwd_ws, const size_t* bwd_ws_bytes, float* const* image,
                           float* const* notex, float* const* weights, int* const* ids,
                           float* const* depths, float* const* textures, float* const* T_final,
                           nexel_stream_t stream) {
  if (n_views <= 0 || !cams || !settings || !ws || !ws_bytes || !image || !notex || !T_final)
    return NEXEL_ERR_INVALID_ARG;
  if (N < 0 || (N > 0 && (!mu || !quat || !scale || !opacity || !gamma || !color)))
    return NEXEL_ERR_INVALID_ARG;
  for (int v = 0; v < n_views; ++v) {
    int rc = check_fwd(&cams[v], settings, field, N, ws[v], ws_bytes[v], at(bwd_ws, v),
                       bwd_ws_bytes ? bwd_ws_bytes[v] : 0, image[v], notex[v], at(weights, v),
                       at(ids, v), at(depths, v), at(textures, v), T_final[v]);
    if (rc != NEXEL_OK) return rc;
  }
  Pool* p = nullptr;
  int rc = get_pool(&p);
  if (rc != NEXEL_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = n_views < kBranches ? n_views : kBranches;
  rc = fork_branches(p, nb, st);
  if (rc != NEXEL_OK) return rc;
  for (int v = 0; v < n_views && rc == NEXEL_OK; ++v) {
    cudaStream_t sv = p->s[v % kBranches];
    rc = preprocess_impl(&cams[v], settings, N, mu, quat, scale, opacity, gamma, color, ws[v],
                         ws_bytes[v], nullptr, sv);
    if (rc == NEXEL_OK)
      rc = render_fwd_impl(&cams[v], settings, field, N, ws[v], ws_bytes[v], at(bwd_ws, v),
                           image[v], notex[v], at(weights, v), at(ids, v), at(depths, v),
                           at(textures, v), T_final[v], sv);
  }
  const int jr = join_branches(p, nb, st);
  return rc != NEXEL_OK ? rc : jr;
}

int nexel_render_batch_bwd(int n_views, const nexel_camera* cams, const nexel_settings* settings,
                           const nexel_field* field, int N, const float* mu, const float* quat,
                           const float* scale, const float* opacity, const float* gamma,
                           void* const* ws, const size_t* ws_bytes, void* const* bwd_ws,
                           const size_t* bwd_ws_bytes, const float* const* weights,
                           const int* const* ids, const float* const* depths,
                           const float* const* T_final, const float* const* d_image,
                           const float* const* d_weights, const float* const* d_textures,
                           int accumulate, float* d_mu, float* d_quat, float* d_scale,
                           float* d_opacity, float* d_gamma, float* d_color, float* d_table,
                           float* d_mlp, nexel_stream_t stream) {
  if (n_views <= 0 || !cams || !settings || !ws || !ws_bytes || !d_image)
    return NEXEL_ERR_INVALID_ARG;
  if (settings->sh_degree == 3 && ((uintptr_t)d_color & 15)) return NEXEL_ERR_INVALID_ARG;
  for (int v = 0; v < n_views; ++v) {
    int rc = check_bwd(&cams[v], settings, field, N, mu, quat, scale, opacity, gamma, ws[v],
                       ws_bytes[v], at(bwd_ws, v), bwd_ws_bytes ? bwd_ws_bytes[v] : 0,
                       at(weights, v), at(ids, v), at(depths, v), at(T_final, v), d_image[v]);
    if (rc != NEXEL_OK) return rc;
  }
  Pool* p = nullptr;
  int rc = get_pool(&p);
  if (rc != NEXEL_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (!accumulate) {
    rc = zero_grads(settings, field, N, d_mu, d_quat, d_scale, d_opacity, d_gamma, d_color,
                    d_table, d_mlp, st);
    if (rc != NEXEL_OK) return rc;
  }
  const int nb = n_views < kBranches ? n_views : kBranches;
  rc = fork_branches(p, nb, st);
  if (rc != NEXEL_OK) return rc;
  for (int v = 0; v < n_views && rc == NEXEL_OK; ++v) {
    cudaStream_t sv = p->s[v % kBranches];
    rc = render_bwd_impl(&cams[v], settings, field, N, mu, quat, scale, opacity, gamma, ws[v],
                         ws_bytes[v], at(bwd_ws, v), at(weights, v), at(ids, v), at(depths, v),
                         at(T_final, v), d_image[v], at(d_weights, v), at(d_textures, v), d_mu,
                         d_quat, d_scale, d_opacity, d_gamma, d_color, d_table, d_mlp, true, sv);
  }
  const int jr = join_branches(p, nb, st);
  return rc != NEXEL_OK ? rc : jr;
}

}  // extern "C"
