// Batched multi-view entry points: one training step over several views of
// the same scene (uneven resolutions), issued without a host
// synchronisation, so that a caller can capture the whole step in one CUDA
// graph and replay it.
//
// Each view keeps its own workspaces; its preprocess uses the device-count
// form (the instance count never leaves the device; the workspace capacity
// bounds it and an overflow is flagged in the view's status word).  The
// per-view preprocess and binning run as parallel branches forked from the
// caller's stream onto a per-device pool of streams and joined back into
// it.  The per-tile phases then run as ONE launch each over the work of
// every view (up to kMaxBatchViews per launch): the collection forward and
// backward as persistent CTAs pulling (view, tile) items from a device
// queue, the tcgen05 texturing forward and backward and the hash-grid
// backward as persistent or flat grids over the views' concatenated tiles
// and rows.  (A step with recomputed buffers, without the feature cache or
// with the FP32 MLP keeps the per-view branches for every phase.)  The
// surfel, table and MLP gradients of all views are summed with atomics.
#include "common.cuh"
#include "texture_common.cuh"

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

bool fused_fwd_ok(const nexel_settings& s, const nexel_field* f) {
  return s.K > 0 && s.recompute_buffers == 0 && f &&
         (s.mlp_dtype == NEXEL_BF16 || s.mlp_dtype == NEXEL_F16);
}

bool fused_bwd_ok(const nexel_settings& s, const nexel_field* f) {
  return fused_fwd_ok(s, f) && s.cache_features != 0;
}

// Forward of every view after their preprocess: one collection launch and
// one texturing launch per chunk of kMaxBatchViews views.
int fused_fwd(int n_views, const nexel_camera* cams, const nexel_settings& s,
              const nexel_field& f, int N, void* const* ws, const size_t* ws_bytes,
              void* const* bwd_ws, float* const* image, float* const* notex,
              float* const* weights, int* const* ids, float* const* depths,
              float* const* textures, float* const* T_final, cudaStream_t st) {
  int log2KP = 0;
  while ((1 << log2KP) < s.K) ++log2KP;
  unsigned* queue = (unsigned*)((char*)ws[0] +
                                ws_layout_for_bytes(cams[0], s.K, N, ws_bytes[0]).counters +
                                kCountersBatchQueue);
  FieldDev fd = make_fielddev(make_devcam(cams[0]), f);
  for (int v0 = 0; v0 < n_views; v0 += kMaxBatchViews) {
    const int nv = std::min(kMaxBatchViews, n_views - v0);
    ViewBatch<CollectFwdView> cb;
    ViewBatch<TexFwdView> tb;
    cb.n = tb.n = nv;
    cb.item0[0] = tb.item0[0] = 0;
    for (int i = 0; i < nv; ++i) {
      const int v = v0 + i;
      const WsLayout L = ws_layout_for_bytes(cams[v], s.K, N, ws_bytes[v]);
      const DevCam c = make_devcam(cams[v]);
      char* w = (char*)ws[v];
      cb.v[i] = collect_fwd_view(c, w, L, notex[v], weights[v], ids[v], depths[v], T_final[v]);
      cb.item0[i + 1] = cb.item0[i] + L.n_tiles;
      uint32_t* cache = nullptr;
      if (s.cache_features) {
        const BwdLayout B = bwd_layout(cams[v], s.K, f.L * f.F, false);
        cache = (uint32_t*)((char*)bwd_ws[v] + B.feat);
      }
      tb.v[i] = TexFwdView{c, notex[v], weights[v], ids[v], depths[v], T_final[v], image[v],
                           textures[v], cache, (int*)(w + L.counters + kStatusOffset)};
      const long long rows = (long long)c.W * c.H << log2KP;
      tb.item0[i + 1] = tb.item0[i] + (int)((rows + 127) / 128);
    }
    cudaError_t e = launch_collect_fwd_batch(s, cb, queue, st);
    if (e == cudaSuccess) e = launch_texture_fwd_tc_batch(s, f, fd, tb, st);
    if (e != cudaSuccess) return NEXEL_ERR_CUDA;
  }
  return NEXEL_OK;
}

// Backward of every view: one tcgen05 texture-backward launch, one
// hash-grid backward launch and one collection-backward launch per chunk of
// kMaxBatchViews views, then each view's preprocess backward (atomics into
// the shared gradients).
int fused_bwd(int n_views, const nexel_camera* cams, const nexel_settings& s,
              const nexel_field& f, int N, const float* mu, const float* quat,
              const float* scale, const float* opacity, const float* gamma, void* const* ws,
              const size_t* ws_bytes, void* const* bwd_ws, const float* const* weights,
              const int* const* ids, const float* const* depths, const float* const* T_final,
              const float* const* d_image, const float* const* d_weights,
              const float* const* d_textures, float* d_mu, float* d_quat, float* d_scale,
              float* d_opacity, float* d_gamma, float* d_color, float* d_table, float* d_mlp,
              bool zeroed, cudaStream_t st) {
  int KP = 1;
  while (KP < s.K) KP <<= 1;
  unsigned* queue = (unsigned*)((char*)ws[0] +
                                ws_layout_for_bytes(cams[0], s.K, N, ws_bytes[0]).counters +
                                kCountersBatchQueue);
  FieldDev fd = make_fielddev(make_devcam(cams[0]), f);
  // the hash backward launches run one after another on this stream; the
  // first finds the table gradient zero unless the call accumulates
  fd.grad_mode = zeroed ? kGradZeroed : kGradExclusive;
  const int h2 = f.n_layers == 3 ? f.widths[2] : 0;
  cudaError_t e = cudaSuccess;
  for (int v0 = 0; v0 < n_views && e == cudaSuccess; v0 += kMaxBatchViews) {
    const int nv = std::min(kMaxBatchViews, n_views - v0);
    ViewBatch<TexBwdView> tb;
    ViewBatch<HashBwdView> hb;
    ViewBatch<CollectBwdView> cb;
    tb.n = hb.n = cb.n = nv;
    tb.item0[0] = hb.item0[0] = cb.item0[0] = 0;
    for (int i = 0; i < nv && e == cudaSuccess; ++i) {
      const int v = v0 + i;
      const WsLayout L = ws_layout_for_bytes(cams[v], s.K, N, ws_bytes[v]);
      const BwdLayout B = bwd_layout(cams[v], s.K, f.L * f.F, false);
      const DevCam c = make_devcam(cams[v]);
      char* w = (char*)ws[v];
      char* bw = (char*)bwd_ws[v];
      const long long n_rows = ((long long)c.W * c.H * KP + 15) / 16 * 16;
      if (gin_stride(n_rows) >= (1LL << 32)) e = cudaErrorInvalidValue;
      // the scratch is the caller's uninitialised memory: the status word
      // the kernels may set starts at zero, the gradient records too
      if (e == cudaSuccess) e = cudaMemsetAsync(bw + B.status, 0, 4, st);
      if (e == cudaSuccess)
        e = cudaMemsetAsync(w + L.grad_sorted, 0, sizeof(float) * kGradStride * (size_t)L.N, st);
      tb.v[i] = TexBwdView{c, (const uint32_t*)(bw + B.feat), weights[v], ids[v], d_image[v],
                           at(d_weights, v), at(d_textures, v), (float*)(bw + B.dweff),
                           (float2*)(bw + B.gin), n_rows, (int*)(bw + B.status)};
      tb.item0[i + 1] = tb.item0[i] + (int)((n_rows + 127) / 128);
      hb.v[i] = HashBwdView{c, ids[v], depths[v], (const float2*)(bw + B.gin),
                            (float*)(bw + B.ddepth), (uint32_t)n_rows,
                            (uint32_t)gin_stride(n_rows)};
      hb.item0[i + 1] = hb.item0[i] + hash_bwd_items(n_rows, KP);
      cb.v[i] = collect_bwd_view(c, w, L, bw, B, ids[v], T_final[v], d_image[v]);
      cb.item0[i + 1] = cb.item0[i] + L.n_tiles;
    }
    if (e == cudaSuccess)
      e = launch_texture_bwd_tc_batch(s.K, KP, f.widths[0], f.widths[1], h2,
                                      f.widths[f.n_layers], s.mlp_dtype == NEXEL_F16, f.weights,
                                      tb, d_mlp, st);
    if (e == cudaSuccess)
      e = launch_hash_bwd_batch(fd, s.K, KP, s.grid_dtype == NEXEL_F16, hb, d_table, st);
    fd.grad_mode = kGradExclusive;  // later view groups add to what this one left
    if (e == cudaSuccess) e = launch_collect_bwd_batch(s, cb, queue, st);
  }
  for (int v = 0; v < n_views && e == cudaSuccess; ++v) {
    const WsLayout L = ws_layout_for_bytes(cams[v], s.K, N, ws_bytes[v]);
    e = launch_preprocess_bwd(make_devcam(cams[v]), s, N, mu, quat, scale, opacity, gamma,
                              (char*)ws[v], L, 1, d_mu, d_quat, d_scale, d_opacity, d_gamma,
                              d_color, true, st);
  }
  return e == cudaSuccess ? NEXEL_OK : NEXEL_ERR_CUDA;
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
  const bool fused = fused_fwd_ok(*settings, field);
  for (int v = 0; v < n_views && rc == NEXEL_OK; ++v) {
    cudaStream_t sv = p->s[v % kBranches];
    rc = preprocess_impl(&cams[v], settings, N, mu, quat, scale, opacity, gamma, color, ws[v],
                         ws_bytes[v], nullptr, sv);
    if (rc == NEXEL_OK && !fused)
      rc = render_fwd_impl(&cams[v], settings, field, N, ws[v], ws_bytes[v], at(bwd_ws, v),
                           image[v], notex[v], at(weights, v), at(ids, v), at(depths, v),
                           at(textures, v), T_final[v], sv);
  }
  const int jr = join_branches(p, nb, st);
  if (rc != NEXEL_OK) return rc;
  if (jr != NEXEL_OK || !fused) return jr;
  return fused_fwd(n_views, cams, *settings, *field, N, ws, ws_bytes, bwd_ws, image, notex,
                   weights, ids, depths, textures, T_final, st);
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
  if (fused_bwd_ok(*settings, field))
    return fused_bwd(n_views, cams, *settings, *field, N, mu, quat, scale, opacity, gamma, ws,
                     ws_bytes, bwd_ws, weights, ids, depths, T_final, d_image, d_weights,
                     d_textures, d_mu, d_quat, d_scale, d_opacity, d_gamma, d_color, d_table,
                     d_mlp, !accumulate, st);
  const int nb = n_views < kBranches ? n_views : kBranches;
  rc = fork_branches(p, nb, st);
  if (rc != NEXEL_OK) return rc;
  for (int v = 0; v < n_views && rc == NEXEL_OK; ++v) {
    cudaStream_t sv = p->s[v % kBranches];
    rc = render_bwd_impl(&cams[v], settings, field, N, mu, quat, scale, opacity, gamma, ws[v],
                         ws_bytes[v], at(bwd_ws, v), at(weights, v), at(ids, v), at(depths, v),
                         at(T_final, v), d_image[v], at(d_weights, v), at(d_textures, v), d_mu,
                         d_quat, d_scale, d_opacity, d_gamma, d_color, d_table, d_mlp,
                         kGradShared, sv);
  }
  const int jr = join_branches(p, nb, st);
  return rc != NEXEL_OK ? rc : jr;
}

}  // extern "C"
