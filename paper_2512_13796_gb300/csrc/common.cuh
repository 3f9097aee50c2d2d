// Internal declarations shared by the CUDA translation units of libnexel.
// Device helpers here are the single definition of the per-pixel surfel
// evaluation used by both the forward and the backward collection kernels,
// so that both take bit-identical discrete decisions.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/nexel.h"

namespace nexel {

constexpr int kTile = NEXEL_TILE;            // 16 x 16 pixel tiles
constexpr int kTilePix = kTile * kTile;      // one thread per pixel
constexpr int kRecF4 = 5;                    // packed surfel record: 5 float4
constexpr int kAuxF4 = 4;                    // camera-space frame for the backward
constexpr int kGradStride = 20;              // per-surfel gradient record (floats)
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;                        // instance (tile) sort
constexpr int kSortItemsDepth = 4;                    // depth sort of the surfels
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per sort block
constexpr int kScanItems = 8;
constexpr int kScanTile = 256 * kScanItems;

// Camera as the kernels see it (float32, with derived fields).
struct DevCam {
  int W, H, tiles_x, tiles_y;
  float fx, fy, cx, cy;
  float R[9];   // world -> camera rotation, row-major
  float t[3];
  float o[3];   // camera centre in world space
  float near_;
};

// Packed per-surfel record (rank order), see the preprocess kernel:
//  q0 = (cpx_hi, cpy_hi, cpx_lo, cpy_lo)  projected centre, pixels, as a
//        float-float pair (hi + lo)
//  q1 = (z, o, gamma1, gamma2)             centre view depth, opacity, gamma
//  q2 = (nx, ny, Cux, Cuy)                 normal and u-numerator per pixel
//  q3 = (Cvx, Cvy, dn0, 0)                 v-numerator, d_mu . n
//  q4 = (c0, c1, c2, id)                   colour and original index (bits)
// With d_mu = mu_c / z the ray through the centre and delta = d - d_mu the
// offset of a pixel's ray (z component 0), the hit of the ray o + t d with
// the surfel plane is t* = (mu_c . n) / (d . n) = z dn0 / (d . n) and, by
// a (d_mu . n) - n (d_mu . a) = d_mu x (a x n),
//   u = delta . Cu / (d . n),  Cu = -z (d_mu x v2) / sigma1,
//   v = delta . Cv / (d . n),  Cv =  z (d_mu x v1) / sigma2,
// with d . n = dn0 + delta . n.  No per-surfel constant divides by
// d_mu . n, so nearly edge-on surfels keep FP32 accuracy.  The x and y
// components are stored divided by fx and fy, so delta is in pixels.
//
// Auxiliary camera-space record for the backward (rank order):
//  a0 = (mu_c, sigma1), a1 = (v1_c, sigma2), a2 = (v2_c, 0), a3 = (n_c, 0).

struct Hit {
  float dx, dy, den, t, u, v, pu, pv, alpha;  // alpha before clamping
};

// |a|^(2 g); exact square for g == 1.
__device__ __forceinline__ float pow2g(float a, float g) {
  if (g == 1.0f) return a * a;
  return exp2f(2.0f * g * __log2f(fabsf(a)));
}

// Ray-surfel intersection and the generalised-Gaussian opacity (Sec. 4.1).
// Returns false when the surfel does not contribute (behind the near plane,
// alpha below alpha_min, or non-finite).
__device__ __forceinline__ bool eval_surfel(const float4& q0, const float4& q1, const float4& q2,
                                            const float4& q3, float fpx, float fpy, float near_,
                                            float alpha_min, Hit& h) {
  h.dx = (fpx - q0.x) - q0.z;
  h.dy = (fpy - q0.y) - q0.w;
  h.den = fmaf(h.dx, q2.x, fmaf(h.dy, q2.y, q3.z));
  const float inv = 1.0f / h.den;
  h.t = q1.x * q3.z * inv;  // z dn0 / den: exactly z on the centre ray
  if (!(h.t > near_)) return false;
  h.u = fmaf(h.dx, q2.z, h.dy * q2.w) * inv;
  h.v = fmaf(h.dx, q3.x, h.dy * q3.y) * inv;
  h.pu = pow2g(h.u, q1.z);
  h.pv = pow2g(h.v, q1.w);
  h.alpha = q1.y * expf(-0.5f * (h.pu + h.pv));
  if (!(h.alpha >= alpha_min) || h.alpha == 0.0f) return false;
  return true;
}

// ---------------------------------------------------------------- hash grid
// MapPositive of the supplementary material (x > 0 -> 2x - 1, else -2x) on
// the integer lattice coordinate, then the Instant-NGP spatial hash.
__device__ __forceinline__ uint32_t map_pos(int k) {
  return k > 0 ? (uint32_t)(2 * k - 1) : (uint32_t)(-2 * k);
}
__device__ __forceinline__ uint32_t hash3(int kx, int ky, int kz, uint32_t mask) {
  return (map_pos(kx) ^ (map_pos(ky) * 2654435761u) ^ (map_pos(kz) * 805459861u)) & mask;
}

template <typename TT>
__device__ __forceinline__ float2 load_entry(const TT* tab, uint32_t idx);
template <>
__device__ __forceinline__ float2 load_entry<float>(const float* tab, uint32_t idx) {
  return __ldg(reinterpret_cast<const float2*>(tab) + idx);
}
template <>
__device__ __forceinline__ float2 load_entry<__half>(const __half* tab, uint32_t idx) {
  __half2 h = __ldg(reinterpret_cast<const __half2*>(tab) + idx);
  return __half22float2(h);
}

// Eq. 3: Delta = 1 - exp(-(f / (s t))^2 / (2 pi)).
__device__ __forceinline__ float downweight(float focal, float s, float t) {
  float r = focal / (s * t);
  return -expm1f(-r * r * 0.15915494309189535f);
}

// Device status word bits (the word at kStatusOffset in the counters region
// of the main workspace, and BwdLayout::status): a bounded device wait that
// ran out, and instances dropped because the key buffers were full.
constexpr int kStatusTimeout = 1;
constexpr int kStatusCapacity = 2;
// counters region: [0] unused, [1] instance count, [8] status word
constexpr size_t kCountersInst = 4;
constexpr size_t kStatusOffset = 32;

// ------------------------------------------------------------ workspace
// Main workspace (binning results and per-pixel replay data).  Regions that
// depend only on (camera, K, N) come first; the instance buffers and the
// sort scratch, whose size follows the instance capacity, come last, so
// every call re-derives the same layout from (camera, K, N, ws_bytes).
struct WsLayout {
  size_t geom_orig, geom_sorted, aux_orig, aux_sorted, dkey0, dkey1, did0, did1, rect, conic, tmask, count,
      offs,
      ranges, n_contrib,
      grad_sorted, counters, fixed_end, inst0, inst1, hist, scan_sums, total;
  int N, P, K, n_tiles, tile_bits, rank_bits, key64, tile_passes;
  long long cap;
};
// Backward scratch (per sample): dL/dW_j, dL/dD_j, the field features and
// the texture gradient.
struct BwdLayout {
  size_t dweff, ddepth, feat, gtex, gin, rc_notex, rc_weights, rc_ids, rc_depths, rc_T,
      status,  // kernel status words (a bounded wait that ran out sets one)
      total;
};

WsLayout ws_layout(const nexel_camera& cam, int K, int N, long long cap);
// Largest capacity whose layout fits in ws_bytes (cap < 0 if none).
WsLayout ws_layout_for_bytes(const nexel_camera& cam, int K, int N, size_t ws_bytes);
BwdLayout bwd_layout(const nexel_camera& cam, int K, int feat_dim, bool recompute);
DevCam make_devcam(const nexel_camera& cam);

// Launch accounting: construct one before each kernel launch (see prof.cu).
class ProfScope {
 public:
  ProfScope(const char* name, cudaStream_t st);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  const char* name_;
  cudaStream_t st_;
  void* a_;
};
#define NEXEL_PROF(name, st) ::nexel::ProfScope _nexel_prof_scope_(name, st)

// Launchers (host side).  They return a cudaError_t.
cudaError_t launch_preprocess(const DevCam& c, const nexel_settings& s, int N, const float* mu,
                              const float* quat, const float* scale, const float* opacity,
                              const float* gamma, const float* color, char* ws,
                              const WsLayout& L, cudaStream_t st);
cudaError_t launch_depth_sort(int N, char* ws, const WsLayout& L, cudaStream_t st);
cudaError_t launch_count_scan(int N, char* ws, const WsLayout& L, cudaStream_t st);
// n_inst: the instance count read back on the host, or < 0 for the
// device-count form (capacity-sized launches that read the count written by
// launch_count_scan and flag an overflow in the status word).
cudaError_t launch_binning(const DevCam& c, int N, long long n_inst, char* ws, const WsLayout& L,
                           cudaStream_t st);
cudaError_t launch_collect_fwd(const DevCam& c, const nexel_settings& s, char* ws,
                               const WsLayout& L, float* notex, float* weights, int* ids,
                               float* depths, float* T_final, cudaStream_t st);
cudaError_t launch_collect_bwd(const DevCam& c, const nexel_settings& s, char* ws,
                               const WsLayout& L, const char* bws, const BwdLayout& B,
                               const int* ids, const float* T_final, const float* d_image,
                               cudaStream_t st);
cudaError_t launch_preprocess_bwd(const DevCam& c, const nexel_settings& s, int N, const float* mu,
                                  const float* quat, const float* scale, const float* opacity,
                                  const float* gamma, char* ws, const WsLayout& L, int accumulate,
                                  float* d_mu, float* d_quat, float* d_scale, float* d_opacity,
                                  float* d_gamma, float* d_color, bool atomic, cudaStream_t st);
// feat_cache (may be null): where a training forward leaves the per-sample
// field features for the backward (the backward's feature buffer).
cudaError_t launch_texture_fwd(const DevCam& c, const nexel_settings& s, const nexel_field& f,
                               const float* notex, const float* weights, const int* ids,
                               const float* depths, const float* T_final, float* image,
                               float* textures, void* feat_cache, int* status, cudaStream_t st);
// feat_cached: the forward left the features in bws (no gather here).
cudaError_t launch_texture_bwd(const DevCam& c, const nexel_settings& s, const nexel_field& f,
                               char* bws, const BwdLayout& B, const float* weights, const int* ids,
                               const float* depths, const float* d_image, const float* d_weights,
                               const float* d_textures, float* d_table, float* d_mlp,
                               bool feat_cached, cudaStream_t st);
bool texture_arch_supported(const nexel_settings& s, const nexel_field& f);

// Per-view bodies of the C entry points (api.cu), shared with the batched
// entry points (batch.cu).  check_* validate one view's arguments and launch
// nothing; the *_impl functions assume a passed check.  preprocess_impl with
// n_instances_out == nullptr is the device-count form.  render_bwd_impl
// always adds into the gradients (zero_grads clears them first);
// atomic_params makes the per-surfel additions atomic, for views that run
// concurrently.
int check_fwd(const nexel_camera* cam, const nexel_settings* settings, const nexel_field* field,
              int N, const void* ws, size_t ws_bytes, const void* bwd_ws, size_t bwd_ws_bytes,
              const float* image, const float* notex, const float* weights, const int* ids,
              const float* depths, const float* textures, const float* T_final);
int check_bwd(const nexel_camera* cam, const nexel_settings* settings, const nexel_field* field,
              int N, const float* mu, const float* quat, const float* scale, const float* opacity,
              const float* gamma, const void* ws, size_t ws_bytes, const void* bwd_ws,
              size_t bwd_ws_bytes, const float* weights, const int* ids, const float* depths,
              const float* T_final, const float* d_image);
int preprocess_impl(const nexel_camera* cam, const nexel_settings* settings, int N,
                    const float* mu, const float* quat, const float* scale, const float* opacity,
                    const float* gamma, const float* color, void* ws, size_t ws_bytes,
                    long long* n_instances_out, cudaStream_t st);
int render_fwd_impl(const nexel_camera* cam, const nexel_settings* settings,
                    const nexel_field* field, int N, void* ws, size_t ws_bytes, void* bwd_ws,
                    float* image, float* notex, float* weights, int* ids, float* depths,
                    float* textures, float* T_final, cudaStream_t st);
int zero_grads(const nexel_settings* settings, const nexel_field* field, int N, float* d_mu,
               float* d_quat, float* d_scale, float* d_opacity, float* d_gamma, float* d_color,
               float* d_table, float* d_mlp, cudaStream_t st);
int render_bwd_impl(const nexel_camera* cam, const nexel_settings* settings,
                    const nexel_field* field, int N, const float* mu, const float* quat,
                    const float* scale, const float* opacity, const float* gamma, void* ws,
                    size_t ws_bytes, void* bwd_ws, const float* weights, const int* ids,
                    const float* depths, const float* T_final, const float* d_image,
                    const float* d_weights, const float* d_textures, float* d_mu, float* d_quat,
                    float* d_scale, float* d_opacity, float* d_gamma, float* d_color,
                    float* d_table, float* d_mlp, bool atomic_params, cudaStream_t st);

}  // namespace nexel
