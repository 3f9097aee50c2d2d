// Device helpers of the texturing pass shared by its FP32 and BF16 kernels:
// the neural-field description, the hashed trilinear gather (forward and
// backward) and the FP32 MLP.
#pragma once

#include "common.cuh"

#include <algorithm>

namespace nexel {

struct FieldDev {
  int L;
  uint32_t mask;  // T - 1
  float focal;    // f of Eq. 3 (fx)
  float s[NEXEL_MAX_LEVELS];
  float inv_s[NEXEL_MAX_LEVELS];  // 1 / s
  const void* table;
  const float* w;
  // per-sample feature buffer of a training step: feat_mode 1 = the forward
  // writes the features there, 2 = the backward reads them instead of
  // gathering, 0 = unused
  void* feat;
  int feat_mode;
  // how the call holds the table gradient (kGradShared: other streams may
  // accumulate into it concurrently; kGradExclusive: no other work writes it
  // while the hash backward runs, which may then reorder it temporarily, see
  // hash_bwd.cu; kGradZeroed: exclusive and all zero on entry)
  int grad_mode;
};

inline FieldDev make_fielddev(const DevCam& c, const nexel_field& f) {
  FieldDev d;
  d.feat = nullptr;
  d.feat_mode = 0;
  d.grad_mode = 0;
  d.L = f.L;
  d.mask = (uint32_t)f.T - 1u;
  d.focal = c.fx;
  for (int l = 0; l < NEXEL_MAX_LEVELS; ++l) {
    d.s[l] = l < f.L ? f.level_scale[l] : 0.f;
    d.inv_s[l] = l < f.L ? 1.f / f.level_scale[l] : 0.f;
  }
  d.table = f.table;
  d.w = f.weights;
  return d;
}

// OUT = 3: RGB texture; OUT = 48: degree-3 SH coefficients of the texture
// (o[3k + ch]), evaluated in the ray direction.
template <int IN, int H1, int H2, int OUT = 3>
struct MlpArch {
  static constexpr int HL = H2 > 0 ? H2 : H1;
  static constexpr int kOffLast = IN * H1 + (H2 > 0 ? H1 * H2 : 0);
  static constexpr int kWeights = kOffLast + OUT * HL;
};


// World-space direction of pixel (px, py), not normalised (z_cam = 1).
__device__ __forceinline__ float3 pixel_dir(const DevCam& c, int px, int py) {
  float dx = (px + 0.5f - c.cx) / c.fx, dy = (py + 0.5f - c.cy) / c.fy;
  return make_float3(c.R[0] * dx + c.R[3] * dy + c.R[6], c.R[1] * dx + c.R[4] * dy + c.R[7],
                     c.R[2] * dx + c.R[5] * dy + c.R[8]);
}

// SH basis of degree <= 3 in the normalised ray direction of pixel p.
__device__ __forceinline__ Sh3 pixel_sh3(const DevCam& c, long long p) {
  const float3 d = pixel_dir(c, (int)(p % c.W), (int)(p / c.W));
  const float inv = rsqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
  return sh3_eval(d.x * inv, d.y * inv, d.z * inv);
}

// Raw table entry (the FP16 pair as its 32-bit pattern, or the FP32 pair)
// and its conversion, so that many gathers can be in flight at once.
template <typename TT>
struct RawEntry;
template <>
struct RawEntry<__half> {
  using T = uint32_t;
  __device__ static T load(const __half* tl, uint32_t idx) {
    return __ldg(reinterpret_cast<const unsigned int*>(tl) + idx);
  }
  __device__ static float2 to2(T v) {
    return __half22float2(*reinterpret_cast<const __half2*>(&v));
  }
  __device__ static T zero() { return 0u; }
};
template <>
struct RawEntry<float> {
  using T = float2;
  __device__ static T load(const float* tl, uint32_t idx) {
    return __ldg(reinterpret_cast<const float2*>(tl) + idx);
  }
  __device__ static float2 to2(T v) { return v; }
  __device__ static T zero() { return make_float2(0.f, 0.f); }
};

// Down-weighted hashed trilinear features of one point (level-major, F = 2).
template <int IN, typename TT>
__device__ __forceinline__ void hash_features(const FieldDev& f, float3 x, float t, float* feat) {
  const TT* tab = reinterpret_cast<const TT*>(f.table);
  const size_t T = (size_t)f.mask + 1;
#pragma unroll
  for (int l = 0; l < IN / 2; ++l) {
    const float s = f.s[l];
    const float gx = s * x.x, gy = s * x.y, gz = s * x.z;
    const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
    const int cx = (int)fx0, cy = (int)fy0, cz = (int)fz0;
    const float rx = gx - fx0, ry = gy - fy0, rz = gz - fz0;
    const TT* tl = tab + (size_t)l * T * 2;
    float ax = 0.f, ay = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
      const float w = (dx ? rx : 1.f - rx) * (dy ? ry : 1.f - ry) * (dz ? rz : 1.f - rz);
      const float2 e = load_entry<TT>(tl, hash3(cx + dx, cy + dy, cz + dz, f.mask));
      ax = fmaf(w, e.x, ax);
      ay = fmaf(w, e.y, ay);
    }
    const float dw = downweight(f.focal, s, t);
    feat[2 * l] = dw * ax;
    feat[2 * l + 1] = dw * ay;
  }
}

// Row stride of the level-major per-row buffers of the hash-grid backward.
__host__ __device__ inline long long gin_stride(long long n_rows) { return (n_rows + 31) / 32 * 32; }

// Hash-grid backward (hash_bwd.cu): table scatter and dL/dD from the feature
// gradient, level-major gin[l * gin_stride(n_rows) + r] = (dL/dh_l0, dL/dh_l1)
// of row r = p * KP + j (pixel p, slot j; KP the power of two >= K).  Writes
// ddepth[p * K + j] of every textured sample.
cudaError_t launch_hash_bwd(const DevCam& c, const FieldDev& fd, int K, int KP, long long n_rows,
                            bool half_table, const int* ids, const float* depths,
                            const float2* gin, float* ddepth, float* d_table, cudaStream_t st);

// Per-view arguments of the hash-grid backward (items: warps, each a slot
// of 32 consecutive pixels; ceil(n_rows / (32 KP)) KP of them per view).
struct HashBwdView {
  DevCam c;
  const int* ids;
  const float* depths;
  const float2* gin;
  float* ddepth;
  uint32_t n_rows, R;  // rows and the gin row stride (gin_stride(n_rows))
};
// One launch over every view of the batch; d_table is shared (summed).
cudaError_t launch_hash_bwd_batch(const FieldDev& fd, int K, int KP, bool half_table,
                                  const ViewBatch<HashBwdView>& b, float* d_table,
                                  cudaStream_t st);
// Warps (work items) of one view's hash-grid backward.
inline int hash_bwd_items(long long n_rows, int KP) {
  return (int)((n_rows + 32LL * KP - 1) / (32LL * KP)) * KP;
}

// FP32 MLP forward; keeps the hidden activations when asked.
template <int IN, int H1, int H2>
__device__ __forceinline__ void mlp_fwd_f32(const float* __restrict__ sW, const float* in,
                                            float* out, float* keep1, float* keep2) {
  using A = MlpArch<IN, H1, H2>;
  float h1[H1];
#pragma unroll
  for (int o = 0; o < H1; ++o) {
    const float4* wr = reinterpret_cast<const float4*>(sW + o * IN);
    float v = 0.f;
#pragma unroll
    for (int i = 0; i < IN / 4; ++i) {
      float4 w4 = wr[i];
      v = fmaf(w4.x, in[4 * i], v);
      v = fmaf(w4.y, in[4 * i + 1], v);
      v = fmaf(w4.z, in[4 * i + 2], v);
      v = fmaf(w4.w, in[4 * i + 3], v);
    }
    h1[o] = fmaxf(v, 0.f);
    if (keep1) keep1[o] = h1[o];
  }
  const float* hl = h1;
  float h2[H2 > 0 ? H2 : 1];
  if constexpr (H2 > 0) {
#pragma unroll
    for (int o = 0; o < H2; ++o) {
      const float4* wr = reinterpret_cast<const float4*>(sW + IN * H1 + o * H1);
      float v = 0.f;
#pragma unroll
      for (int i = 0; i < H1 / 4; ++i) {
        float4 w4 = wr[i];
        v = fmaf(w4.x, h1[4 * i], v);
        v = fmaf(w4.y, h1[4 * i + 1], v);
        v = fmaf(w4.z, h1[4 * i + 2], v);
        v = fmaf(w4.w, h1[4 * i + 3], v);
      }
      h2[o] = fmaxf(v, 0.f);
      if (keep2) keep2[o] = h2[o];
    }
    hl = h2;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float4* wr = reinterpret_cast<const float4*>(sW + A::kOffLast + k * A::HL);
    float v = 0.f;
#pragma unroll
    for (int i = 0; i < A::HL / 4; ++i) {
      float4 w4 = wr[i];
      v = fmaf(w4.x, hl[4 * i], v);
      v = fmaf(w4.y, hl[4 * i + 1], v);
      v = fmaf(w4.z, hl[4 * i + 2], v);
      v = fmaf(w4.w, hl[4 * i + 3], v);
    }
    out[k] = v;
  }
}

// FP32 MLP backward to the input (ReLU masks from the kept activations).
template <int IN, int H1, int H2>
__device__ __forceinline__ void mlp_bwd_input_f32(const float* __restrict__ sW, const float* gT,
                                                  const float* h1, const float* h2, float* gin) {
  using A = MlpArch<IN, H1, H2>;
  constexpr int HL = A::HL;
  const float* W3 = sW + A::kOffLast;
  const float* hl = (H2 > 0) ? h2 : h1;
  float dl[HL];
#pragma unroll
  for (int i = 0; i < HL; ++i) {
    float v = W3[i] * gT[0] + W3[HL + i] * gT[1] + W3[2 * HL + i] * gT[2];
    dl[i] = hl[i] > 0.f ? v : 0.f;
  }
  float d1[H1];
  if constexpr (H2 > 0) {
    const float* W2 = sW + IN * H1;
#pragma unroll
    for (int i = 0; i < H1; ++i) d1[i] = 0.f;
#pragma unroll
    for (int o = 0; o < H2; ++o) {
      const float g = dl[o];
      const float4* wr = reinterpret_cast<const float4*>(W2 + o * H1);
#pragma unroll
      for (int i = 0; i < H1 / 4; ++i) {
        float4 w4 = wr[i];
        d1[4 * i] = fmaf(w4.x, g, d1[4 * i]);
        d1[4 * i + 1] = fmaf(w4.y, g, d1[4 * i + 1]);
        d1[4 * i + 2] = fmaf(w4.z, g, d1[4 * i + 2]);
        d1[4 * i + 3] = fmaf(w4.w, g, d1[4 * i + 3]);
      }
    }
#pragma unroll
    for (int i = 0; i < H1; ++i) d1[i] = h1[i] > 0.f ? d1[i] : 0.f;
  } else {
#pragma unroll
    for (int i = 0; i < H1; ++i) d1[i] = dl[i];
  }
#pragma unroll
  for (int i = 0; i < IN; ++i) gin[i] = 0.f;
#pragma unroll
  for (int o = 0; o < H1; ++o) {
    const float g = d1[o];
    const float4* wr = reinterpret_cast<const float4*>(sW + o * IN);
#pragma unroll
    for (int i = 0; i < IN / 4; ++i) {
      float4 w4 = wr[i];
      gin[4 * i] = fmaf(w4.x, g, gin[4 * i]);
      gin[4 * i + 1] = fmaf(w4.y, g, gin[4 * i + 1]);
      gin[4 * i + 2] = fmaf(w4.z, g, gin[4 * i + 2]);
      gin[4 * i + 3] = fmaf(w4.w, g, gin[4 * i + 3]);
    }
  }
}

// Texturing on tcgen05 (texture_tc.cu), BF16 or FP16 MMA operands
// (s.mlp_dtype).  The forward writes the features to fd.feat when
// fd.feat_mode == 1; the gather pass writes them for a backward without
// cached features; the backward writes dweff and the level-major feature
// gradient and adds the MLP weight gradients to d_mlp (may be null).
// out: 3 (RGB texture) or 48 (degree-3 SH coefficients; FP16 table only)
bool tc_arch_supported(int in, int h1, int h2, int out, bool half_table);
// Per-view arguments of the tcgen05 texturing forward (items: 128-row tiles
// of the view's (pixel, slot) rows, pixel-major with KP rows per pixel).
struct TexFwdView {
  DevCam c;
  const float *notex, *weights;
  const int* ids;
  const float *depths, *T_final;
  float *image, *textures;
  uint32_t* feat_cache;  // nullptr unless a training step caches the features
  int* status;
};
// Per-view arguments of the tcgen05 texturing backward (items: 128-row
// tiles; the rows' features cached by the forward in feat).
struct TexBwdView {
  DevCam c;
  const uint32_t* feat;
  const float* weights;
  const int* ids;
  const float *d_image, *d_weights, *d_textures;
  float* dweff;
  float2* gin;
  long long n_rows;
  int* status;
};
// The tcgen05 backward with three tile groups per CTA (texture_tc_bwd3.cu):
// the shapes it takes, and its launch.
bool tex_bwd_tc3_supported(int in, int h1, int h2, int out);
cudaError_t launch_texture_bwd_tc3(int K, int KP, int in, bool f16, const float* w,
                                   const ViewBatch<TexBwdView>& b, float* d_mlp, cudaStream_t st);
cudaError_t launch_texture_bwd_tc_batch(int K, int KP, int in, int h1, int h2, int out, bool f16,
                                        const float* w, const ViewBatch<TexBwdView>& b,
                                        float* d_mlp, cudaStream_t st);
// One launch over every view of the batch (tile counts in b.item0).
cudaError_t launch_texture_fwd_tc_batch(const nexel_settings& s, const nexel_field& f,
                                        const FieldDev& fd, const ViewBatch<TexFwdView>& b,
                                        cudaStream_t st);
cudaError_t launch_texture_fwd_tc(const DevCam& c, const nexel_settings& s, const nexel_field& f,
                                  const FieldDev& fd, const float* notex, const float* weights,
                                  const int* ids, const float* depths, const float* T_final,
                                  float* image, float* textures, int* status, cudaStream_t st);
cudaError_t launch_texture_gather_tc(const DevCam& c, const nexel_settings& s,
                                     const nexel_field& f, const FieldDev& fd, const int* ids,
                                     const float* depths, uint32_t* feat, cudaStream_t st);
cudaError_t launch_texture_bwd_tc(const DevCam& c, int K, int KP, long long n_rows, int in, int h1,
                                  int h2, int out, bool f16, const float* w, const uint32_t* feat,
                                  const float* weights, const int* ids, const float* d_image,
                                  const float* d_weights, const float* d_textures, float* dweff,
                                  float2* gin, float* d_mlp, int* status, cudaStream_t st);

}  // namespace nexel
