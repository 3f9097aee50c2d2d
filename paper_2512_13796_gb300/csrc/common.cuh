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
constexpr int kGradStride = 16;              // per-surfel gradient record (floats)
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;                        // instance (tile) sort
constexpr int kSortItemsDepth = 4;                    // depth sort of the surfels
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per sort block
// direct placement of the instances by tile (32-bit keys only): ranks per
// block, and the largest tile count (two shared-memory words per tile)
constexpr int kPlaceRanks = 1024;
constexpr int kPlaceThreads = 1024;  // one rank per thread when staging
constexpr int kPlaceMaxTiles = 8192;
// stored tile decisions: room for this many words (32 rectangle tiles each)
// per surfel on average; surfels past the room are tested again
constexpr int kMaskWordsPerSurfel = 8;
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

// Rotation of a (normalised) quaternion (w, x, y, z): columns v1, v2, n.
__device__ __forceinline__ void quat_cols(float w, float x, float y, float z, float3& v1, float3& v2,
                                          float3& n) {
  v1 = make_float3(1.f - 2.f * (y * y + z * z), 2.f * (x * y + w * z), 2.f * (x * z - w * y));
  v2 = make_float3(2.f * (x * y - w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z + w * x));
  n = make_float3(2.f * (x * z + w * y), 2.f * (y * z - w * x), 1.f - 2.f * (x * x + y * y));
}

// Real spherical harmonics of degree <= 3 at the unit direction (x, y, z)
// (orthonormal on the sphere; ordered by degree l, then m = -l .. l; with
// the Condon-Shortley phase): the per-primitive colour mode of Sec. 3 with
// the degree of Sec. 5 (S = 16).
struct Sh3 {
  float y[16];
};
__host__ __device__ inline Sh3 sh3_eval(float x, float y, float z) {
  // normalisation constants: sqrt((2l + 1) / (4 pi) (l - |m|)! / (l + |m|)!)
  // times the factors of the Cartesian forms
  const float k0 = 0.28209479177387814f, k1 = 0.48860251190291992f;
  const float k2a = 1.0925484305920792f, k2b = 0.31539156525252005f, k2c = 0.54627421529603959f;
  const float k3a = 0.59004358992664352f, k3b = 2.8906114426405538f, k3c = 0.45704579946446572f,
              k3d = 0.37317633259011540f, k3e = 1.4453057213202769f;
  const float xx = x * x, yy = y * y, zz = z * z;
  Sh3 r;
  r.y[0] = k0;
  r.y[1] = -k1 * y; r.y[2] = k1 * z; r.y[3] = -k1 * x;
  r.y[4] = k2a * x * y; r.y[5] = -k2a * y * z; r.y[6] = k2b * (2.f * zz - xx - yy);
  r.y[7] = -k2a * x * z; r.y[8] = k2c * (xx - yy);
  r.y[9] = -k3a * y * (3.f * xx - yy); r.y[10] = k3b * x * y * z;
  r.y[11] = -k3c * y * (4.f * zz - xx - yy); r.y[12] = k3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  r.y[13] = -k3c * x * (4.f * zz - xx - yy); r.y[14] = k3e * z * (xx - yy);
  r.y[15] = -k3a * x * (xx - 3.f * yy);
  return r;
}
// sum_k w[k] dY_k/d(x, y, z) of the polynomials above
__host__ __device__ inline float3 sh3_grad_dot(float x, float y, float z, const float* w) {
  const float k1 = 0.48860251190291992f;
  const float k2a = 1.0925484305920792f, k2b = 0.31539156525252005f, k2c = 0.54627421529603959f;
  const float k3a = 0.59004358992664352f, k3b = 2.8906114426405538f, k3c = 0.45704579946446572f,
              k3d = 0.37317633259011540f, k3e = 1.4453057213202769f;
  const float xx = x * x, yy = y * y, zz = z * z;
  float gx = 0.f, gy = 0.f, gz = 0.f;
  gy += -k1 * w[1]; gz += k1 * w[2]; gx += -k1 * w[3];
  gx += k2a * y * w[4]; gy += k2a * x * w[4];
  gy += -k2a * z * w[5]; gz += -k2a * y * w[5];
  gx += -2.f * k2b * x * w[6]; gy += -2.f * k2b * y * w[6]; gz += 4.f * k2b * z * w[6];
  gx += -k2a * z * w[7]; gz += -k2a * x * w[7];
  gx += 2.f * k2c * x * w[8]; gy += -2.f * k2c * y * w[8];
  gx += -6.f * k3a * x * y * w[9]; gy += -3.f * k3a * (xx - yy) * w[9];
  gx += k3b * y * z * w[10]; gy += k3b * x * z * w[10]; gz += k3b * x * y * w[10];
  gx += 2.f * k3c * x * y * w[11]; gy += -k3c * (4.f * zz - xx - 3.f * yy) * w[11];
  gz += -8.f * k3c * y * z * w[11];
  gx += -6.f * k3d * x * z * w[12]; gy += -6.f * k3d * y * z * w[12];
  gz += k3d * (6.f * zz - 3.f * xx - 3.f * yy) * w[12];
  gx += -k3c * (4.f * zz - 3.f * xx - yy) * w[13]; gy += 2.f * k3c * x * y * w[13];
  gz += -8.f * k3c * x * z * w[13];
  gx += 2.f * k3e * x * z * w[14]; gy += -2.f * k3e * y * z * w[14]; gz += k3e * (xx - yy) * w[14];
  gx += -3.f * k3a * (xx - yy) * w[15]; gy += 6.f * k3a * x * y * w[15];
  return make_float3(gx, gy, gz);
}

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
//  a0 = (mu_c, sigma1), a1 = (v1_c, sigma2), a2 = (v2_c, 1 / sigma1),
//  a3 = (n_c, 1 / sigma2).

struct Hit {
  float dx, dy, inv, t, u, v, pu, pv, e, alpha;  // inv = 1 / den; alpha = opacity e, unclamped
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
  const float den = fmaf(h.dx, q2.x, fmaf(h.dy, q2.y, q3.z));
  const float inv = 1.0f / den;
  h.inv = inv;
  h.t = q1.x * q3.z * inv;  // z dn0 / den: exactly z on the centre ray
  if (!(h.t > near_)) return false;
  h.u = fmaf(h.dx, q2.z, h.dy * q2.w) * inv;
  h.v = fmaf(h.dx, q3.x, h.dy * q3.y) * inv;
  h.pu = pow2g(h.u, q1.z);
  h.pv = pow2g(h.v, q1.w);
  h.e = expf(-0.5f * (h.pu + h.pv));
  h.alpha = q1.y * h.e;
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

// 1 - exp(-a) for a >= 0 without cancellation and without branches: the
// alternating Taylor series a - a^2/2! + ... + a^7/7! where a <= 1/2 (its
// truncation error, a^8/8!, is < 2.5e-7 of the result there), and 1 - e^-a
// beyond (the result is >= 0.39, so the exponential's rounding stays
// relative).
__device__ __forceinline__ float one_minus_exp_neg(float a) {
  float p = fmaf(a, -1.f / 5040.f, 1.f / 720.f);
  p = fmaf(a, p, -1.f / 120.f);
  p = fmaf(a, p, 1.f / 24.f);
  p = fmaf(a, p, -1.f / 6.f);
  p = fmaf(a, p, 0.5f);
  p = fmaf(a, -p, 1.f);
  const float small = a * p;
  const float big = 1.f - __expf(-a);
  return a <= 0.5f ? small : big;
}

// Eq. 3: Delta = 1 - exp(-(f / (s t))^2 / (2 pi)).
__device__ __forceinline__ float downweight(float focal, float s, float t) {
  float r = focal / (s * t);
  return one_minus_exp_neg(r * r * 0.15915494309189535f);
}

// Device status word bits (the word at kStatusOffset in the counters region
// of the main workspace, and BwdLayout::status): a bounded device wait that
// ran out, instances dropped because the key buffers were full, and surfels
// culled for a non-finite parameter.
constexpr int kStatusTimeout = 1;
constexpr int kStatusCapacity = 2;
constexpr int kStatusNumeric = 4;
// counters region (byte offsets): instance count, placed instances, stored
// tile-decision words, non-finite surfels, the status word, the statistics
constexpr size_t kCountersInst = 4;
constexpr size_t kCountersPlaced = 8;  // instances placed by the direct tile placement
constexpr size_t kCountersMaskWords = 12;  // stored tile-decision words wanted
constexpr size_t kCountersNonFinite = 16;  // surfels culled for a NaN / infinite parameter
constexpr size_t kCountersBatchQueue = 20;  // work queue of a batched launch (first view's block)
constexpr size_t kStatusOffset = 32;
constexpr size_t kStatsOffset = 64;  // 5 x u64 of nexel_render_stats

// ------------------------------------------------------------ workspace
// Main workspace (binning results and per-pixel replay data).  Regions that
// depend only on (camera, K, N) come first; the instance buffers and the
// sort scratch, whose size follows the instance capacity, come last, so
// every call re-derives the same layout from (camera, K, N, ws_bytes).
struct WsLayout {
  size_t geom_orig, geom_sorted, aux_orig, aux_sorted, dkey0, dkey1, did0, did1, rect, conic, tmask, count,
      shj,
      offs,
      ranges, n_contrib,
      grad_sorted, counters, place, place_tiles, mword_off, mwords, fixed_end, inst0, inst1, hist,
      scan_sums, total;
  long long mword_cap;  // words of room in mwords
  int N, P, K, n_tiles, tile_bits, rank_bits, key64, tile_passes;
  int place_ok;   // the instances are placed by tile directly (no tile sort)
  int rank_only;  // placed keys hold the depth rank alone (tile + rank bits > 32)
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
// ----------------------------------------------- views of one batched launch
// A batched launch covers the work items of up to kMaxBatchViews views: item
// i belongs to the view v with item0[v] <= i < item0[v + 1] (the views'
// items one after another).
constexpr int kMaxBatchViews = 16;
template <typename V>
struct ViewBatch {
  int n;
  int item0[kMaxBatchViews + 1];
  V v[kMaxBatchViews];
};

// A view's binned instances: 32-bit (tile << rank_bits | rank) keys or
// 64-bit keys whose low 32 bits are the depth rank.
struct KeySrc {
  const void* keys;
  uint32_t rmask;
  int key64;
};

// The view of work item `item` (the views' items lie one after another).
template <typename V>
__device__ __forceinline__ int view_of(const ViewBatch<V>& b, int item) {
  int v = 0;
  while (v + 1 < b.n && item >= b.item0[v + 1]) ++v;
  return v;
}

// Per-view arguments of the collection forward and backward (items: tiles).
struct CollectFwdView {
  DevCam c;
  const uint2* ranges;
  KeySrc keys;
  const float4* recs;
  float *notex, *weights;
  int* ids;
  float *depths, *T_final;
  int* n_contrib;
};
struct CollectBwdView {
  DevCam c;
  const uint2* ranges;
  KeySrc keys;
  const float4 *recs, *aux;
  const int* ids;
  const float* T_final;
  const int* n_contrib;
  const float *d_image, *dweff, *ddepth;
  float* grad;
};

CollectFwdView collect_fwd_view(const DevCam& c, char* ws, const WsLayout& L, float* notex,
                                float* weights, int* ids, float* depths, float* T_final);
CollectBwdView collect_bwd_view(const DevCam& c, char* ws, const WsLayout& L, const char* bws,
                                const BwdLayout& B, const int* ids, const float* T_final,
                                const float* d_image);
// queue: a device counter (reset by the launch) for persistent CTAs pulling
// the items of every view; nullptr: one CTA per item.  The backward's
// gradient records (grad of each view) must be zeroed by the caller.
cudaError_t launch_collect_fwd_batch(const nexel_settings& s, const ViewBatch<CollectFwdView>& b,
                                     unsigned* queue, cudaStream_t st);
cudaError_t launch_collect_bwd_batch(const nexel_settings& s, const ViewBatch<CollectBwdView>& b,
                                     unsigned* queue, cudaStream_t st);

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
// Blended error of every surfel (adds into err[N], original order).
cudaError_t launch_blend_error(const DevCam& c, const nexel_settings& s, char* ws,
                               const WsLayout& L, const float* image, const float* target,
                               float* err, cudaStream_t st);
// feat_cache (may be null): where a training forward leaves the per-sample
// field features for the backward (the backward's feature buffer).
cudaError_t launch_texture_fwd(const DevCam& c, const nexel_settings& s, const nexel_field& f,
                               const float* notex, const float* weights, const int* ids,
                               const float* depths, const float* T_final, float* image,
                               float* textures, void* feat_cache, int* status, cudaStream_t st);
// feat_cached: the forward left the features in bws (no gather here).
// grad_mode: kGradShared / kGradExclusive / kGradZeroed (d_table)
cudaError_t launch_texture_bwd(const DevCam& c, const nexel_settings& s, const nexel_field& f,
                               char* bws, const BwdLayout& B, const float* weights, const int* ids,
                               const float* depths, const float* d_image, const float* d_weights,
                               const float* d_textures, float* d_table, float* d_mlp,
                               bool feat_cached, int grad_mode, cudaStream_t st);
bool texture_arch_supported(const nexel_settings& s, const nexel_field& f);

// Stable LSD radix sort of n (uint32 key, uint32 value) pairs on all 32 key
// bits (result in buffer pair *which), and an in-place exclusive scan with
// the total; scratch: hist >= 256 ceil(n / 1024) words, sums >= that / 2048
// + 2 words (binning.cu).
cudaError_t sort_pairs_u32(uint32_t* k0, uint32_t* k1, uint32_t* v0, uint32_t* v1, long long n,
                           uint32_t* hist, uint32_t* sums, cudaStream_t st, int* which);
cudaError_t exclusive_scan_u32(uint32_t* a, long long n, uint32_t* sums, uint32_t* total,
                               cudaStream_t st);

// Launch shapes chosen by nexel_autotune / nexel_set_tuning (tuning.cu),
// process-wide: CTAs per SM of the persistent texturing kernels, the CTA
// size of the hash backward, the surfel staging batch of the collection
// kernels and the depth of the texturing forward's operand ring.
struct Tuning {
  int tex_fwd_ctas = 2, tex_bwd_ctas = 3, f32_ctas = 2, hash_block = 256;
  int collect_batch = 256, tex_fwd_stages = 4;
};
Tuning current_tuning();
// Test hook of the bounded waits (nexel_test_tc_wait_timeout): 0, or the
// poll limit with which the tensor-core kernels wait for MMAs they do not
// issue.
int tc_wait_fault();

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
// How a backward call holds its gradient outputs
constexpr int kGradShared = 0;     // other calls accumulate into them concurrently (atomics)
constexpr int kGradExclusive = 1;  // this call alone writes them until it completes
constexpr int kGradZeroed = 2;     // ... and they were zeroed just before it
int render_bwd_impl(const nexel_camera* cam, const nexel_settings* settings,
                    const nexel_field* field, int N, const float* mu, const float* quat,
                    const float* scale, const float* opacity, const float* gamma, void* ws,
                    size_t ws_bytes, void* bwd_ws, const float* weights, const int* ids,
                    const float* depths, const float* T_final, const float* d_image,
                    const float* d_weights, const float* d_textures, float* d_mu, float* d_quat,
                    float* d_scale, float* d_opacity, float* d_gamma, float* d_color,
                    float* d_table, float* d_mlp, int grad_mode, cudaStream_t st);

}  // namespace nexel
