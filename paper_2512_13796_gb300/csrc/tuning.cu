// Launch-shape tuning: how many CTAs per SM the persistent texturing kernels
// keep in flight (the tile pipeline depth of the MLP kernels), the CTA size
// of the hash backward, the surfel staging batch of the collection kernels
// and the depth of the texturing forward's operand ring.  The choice is process-wide; nexel_autotune
// measures the candidates on the caller's own workload (one training step:
// forward + backward, timed with CUDA events on the caller's stream) and
// keeps the fastest, one knob after another (a change must gain 1 %).
#include "common.cuh"

#include <algorithm>
#include <atomic>
#include <vector>

namespace nexel {
namespace {

std::atomic<int> g_fwd{2}, g_bwd{3}, g_f32{2}, g_hash{256}, g_batch{256}, g_stages{4};
std::atomic<int> g_tc_wait_fault{0};

bool valid(const nexel_tuning& t) {
  return t.tex_fwd_ctas_per_sm >= 1 && t.tex_fwd_ctas_per_sm <= 2 &&
         t.tex_bwd_ctas_per_sm >= 1 && t.tex_bwd_ctas_per_sm <= 3 && t.f32_ctas_per_sm >= 1 &&
         t.f32_ctas_per_sm <= 2 && (t.hash_block == 128 || t.hash_block == 256) &&
         (t.collect_batch == 128 || t.collect_batch == 256 || t.collect_batch == 512) &&
         t.tex_fwd_stages >= 2 && t.tex_fwd_stages <= 4;
}

void put(const nexel_tuning& t) {
  g_fwd = t.tex_fwd_ctas_per_sm;
  g_bwd = t.tex_bwd_ctas_per_sm;
  g_f32 = t.f32_ctas_per_sm;
  g_hash = t.hash_block;
  g_batch = t.collect_batch;
  g_stages = t.tex_fwd_stages;
}

nexel_tuning get() {
  nexel_tuning t;
  t.tex_fwd_ctas_per_sm = g_fwd;
  t.tex_bwd_ctas_per_sm = g_bwd;
  t.f32_ctas_per_sm = g_f32;
  t.hash_block = g_hash;
  t.collect_batch = g_batch;
  t.tex_fwd_stages = g_stages;
  return t;
}

}  // namespace

int tc_wait_fault() { return g_tc_wait_fault; }

Tuning current_tuning() {
  Tuning t;
  t.tex_fwd_ctas = g_fwd;
  t.tex_bwd_ctas = g_bwd;
  t.f32_ctas = g_f32;
  t.hash_block = g_hash;
  t.collect_batch = g_batch;
  t.tex_fwd_stages = g_stages;
  return t;
}

}  // namespace nexel

using namespace nexel;

extern "C" {

int nexel_test_tc_wait_timeout(int polls) {
  if (polls < 0 || polls > (1 << 16)) return NEXEL_ERR_INVALID_ARG;
  g_tc_wait_fault = polls;
  return NEXEL_OK;
}

int nexel_get_tuning(nexel_tuning* out) {
  if (!out) return NEXEL_ERR_INVALID_ARG;
  *out = get();
  return NEXEL_OK;
}

int nexel_set_tuning(const nexel_tuning* t) {
  if (!t || !valid(*t)) return NEXEL_ERR_INVALID_ARG;
  put(*t);
  return NEXEL_OK;
}

int nexel_autotune(const nexel_camera* cam, const nexel_settings* settings,
                   const nexel_field* field, int N, const float* mu, const float* quat,
                   const float* scale, const float* opacity, const float* gamma,
                   const float* color, void* ws, size_t ws_bytes, void* bwd_ws,
                   size_t bwd_ws_bytes, float* image, float* notex, float* weights, int* ids,
                   float* depths, float* textures, float* T_final, const float* d_image,
                   float* d_mu, float* d_quat, float* d_scale, float* d_opacity, float* d_gamma,
                   float* d_color, float* d_table, float* d_mlp, int reps, void* flush,
                   size_t flush_bytes, nexel_tuning* best, float* best_ms,
                   nexel_stream_t stream) {
  if (reps < 1 || reps > 100 || !best || (flush_bytes > 0 && !flush)) return NEXEL_ERR_INVALID_ARG;
  int rc = check_fwd(cam, settings, field, N, ws, ws_bytes, bwd_ws, bwd_ws_bytes, image, notex,
                     weights, ids, depths, textures, T_final);
  if (rc != NEXEL_OK) return rc;
  rc = check_bwd(cam, settings, field, N, mu, quat, scale, opacity, gamma, ws, ws_bytes, bwd_ws,
                 bwd_ws_bytes, weights, ids, depths, T_final, d_image);
  if (rc != NEXEL_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  long long n_inst = 0;
  rc = preprocess_impl(cam, settings, N, mu, quat, scale, opacity, gamma, color, ws, ws_bytes,
                       &n_inst, st);
  if (rc != NEXEL_OK) return rc;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
    if (a) cudaEventDestroy(a);
    return NEXEL_ERR_CUDA;
  }
  auto step = [&]() {
    int r = render_fwd_impl(cam, settings, field, N, ws, ws_bytes, bwd_ws, image, notex, weights,
                            ids, depths, textures, T_final, st);
    if (r == NEXEL_OK)
      r = zero_grads(settings, field, N, d_mu, d_quat, d_scale, d_opacity, d_gamma, d_color,
                     d_table, d_mlp, st);
    if (r == NEXEL_OK)
      r = render_bwd_impl(cam, settings, field, N, mu, quat, scale, opacity, gamma, ws, ws_bytes,
                          bwd_ws, weights, ids, depths, T_final, d_image, nullptr, nullptr, d_mu,
                          d_quat, d_scale, d_opacity, d_gamma, d_color, d_table, d_mlp,
                          kGradZeroed, st);
    return r;
  };
  // median time of reps steps after one untimed step
  auto measure = [&](const nexel_tuning& t, float* ms) {
    put(t);
    int r = step();
    std::vector<float> v;
    for (int i = 0; i < reps && r == NEXEL_OK; ++i) {
      // the caller's buffer (larger than L2) written before each timed step
      if (flush_bytes > 0 && cudaMemsetAsync(flush, i & 0xff, flush_bytes, st) != cudaSuccess)
        return NEXEL_ERR_CUDA;
      if (cudaEventRecord(a, st) != cudaSuccess) return NEXEL_ERR_CUDA;
      r = step();
      if (cudaEventRecord(b, st) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess)
        return NEXEL_ERR_CUDA;
      float x = 0.f;
      cudaEventElapsedTime(&x, a, b);
      v.push_back(x);
    }
    if (r != NEXEL_OK) return r;
    std::sort(v.begin(), v.end());
    *ms = v[v.size() / 2];
    return NEXEL_OK;
  };
  nexel_tuning cur = get();
  float cur_ms = 0.f;
  rc = measure(cur, &cur_ms);
  // one knob after another, keeping the best value of each
  for (int knob = 0; knob < 6 && rc == NEXEL_OK; ++knob) {
    std::vector<int> vals;
    if (knob == 0) vals = {1, 2};
    else if (knob == 1) vals = {1, 2, 3};
    else if (knob == 2) vals = {1, 2};
    else if (knob == 3) vals = {128, 256};
    else if (knob == 4) vals = {128, 256, 512};
    else vals = {2, 3, 4};
    for (int v : vals) {
      nexel_tuning t = cur;
      int* field_of[6] = {&t.tex_fwd_ctas_per_sm, &t.tex_bwd_ctas_per_sm, &t.f32_ctas_per_sm,
                          &t.hash_block, &t.collect_batch, &t.tex_fwd_stages};
      if (*field_of[knob] == v) continue;
      *field_of[knob] = v;
      float ms = 0.f;
      rc = measure(t, &ms);
      if (rc != NEXEL_OK) break;
      // a candidate replaces the current value only when it is at least 1 %
      // faster (run-to-run noise of the median is below that)
      if (ms < 0.99f * cur_ms) {
        cur = t;
        cur_ms = ms;
      }
    }
  }
  put(cur);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc != NEXEL_OK) return rc;
  *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return NEXEL_OK;
}

}  // extern "C"
