// Texturing pass (Sec. 4.2, Eqs. 3-4, 6) and its backward, FP32 form.
//
// Forward, one thread per (pixel, slot) sample: x = o + D d, L levels of
// hashed trilinear lookups (MapPositive + spatial hash), each level scaled
// by Delta_l (Eq. 3), then the MLP G (no bias, ReLU) with the weights in
// shared memory, then the composite C = N + sum_j W_j T_j + T_final bg of
// Eq. 6 reduced over the slot lanes of the pixel with shuffles.
//
// Backward: the sample kernel recomputes the forward (or reads the features
// the forward of a training step left), runs the MLP backward for the
// feature gradient and forms dL/dW; it leaves the feature gradient (for the
// hash-grid backward, hash_bwd.cu, which scatters it into the table gradient
// and forms dL/dD), the features and the texture gradient in the workspace,
// from which a second kernel forms the MLP weight gradients (a reduction
// over all samples) with per-thread register accumulators.
#pragma once

#include "common.cuh"
#include "texture_common.cuh"

namespace nexel {

// ------------------------------------------------------------- forward
template <int IN, int H1, int H2, typename TT>
__global__ void __launch_bounds__(256) k_tex_fwd_f32(DevCam c, FieldDev f, int K, int KP,
                                                      float bg0, float bg1, float bg2,
                                                      const float* __restrict__ notex,
                                                      const float* __restrict__ weights,
                                                      const int* __restrict__ ids,
                                                      const float* __restrict__ depths,
                                                      const float* __restrict__ T_final,
                                                      float* __restrict__ image,
                                                      float* __restrict__ textures) {
  using A = MlpArch<IN, H1, H2>;
  __shared__ __align__(16) float sW[A::kWeights];
  for (int k = threadIdx.x; k < A::kWeights; k += blockDim.x) sW[k] = f.w[k];
  __syncthreads();
  const long long P = (long long)c.W * c.H;
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long p = s / KP;
  const int j = (int)(s % KP);
  const bool pix_ok = p < P;
  float t0 = 0.f, t1 = 0.f, t2 = 0.f, wj = 0.f;
  if (pix_ok && j < K) {
    const int id = ids[p * K + j];
    if (id >= 0) {
      wj = weights[p * K + j];
      const float D = depths[p * K + j];
      float3 d = pixel_dir(c, (int)(p % c.W), (int)(p / c.W));
      float3 x = make_float3(c.o[0] + D * d.x, c.o[1] + D * d.y, c.o[2] + D * d.z);
      float feat[IN];
      hash_features<IN, TT>(f, x, D, feat);
      if (f.feat_mode == 1) {
        float* fo = reinterpret_cast<float*>(f.feat) + (p * K + j) * IN;
#pragma unroll
        for (int k = 0; k < IN; ++k) fo[k] = feat[k];
      }
      float out[3];
      mlp_fwd_f32<IN, H1, H2>(sW, feat, out, nullptr, nullptr);
      t0 = out[0]; t1 = out[1]; t2 = out[2];
    } else if (f.feat_mode == 1) {
      float* fo = reinterpret_cast<float*>(f.feat) + (p * K + j) * IN;
#pragma unroll
      for (int k = 0; k < IN; ++k) fo[k] = 0.f;
    }
    float* dst = textures + (p * K + j) * 3;
    dst[0] = t0; dst[1] = t1; dst[2] = t2;
  }
  // composite over the KP lanes of this pixel
  float c0 = wj * t0, c1 = wj * t1, c2 = wj * t2;
  for (int d = 1; d < KP; d <<= 1) {
    c0 += __shfl_xor_sync(0xffffffffu, c0, d);
    c1 += __shfl_xor_sync(0xffffffffu, c1, d);
    c2 += __shfl_xor_sync(0xffffffffu, c2, d);
  }
  if (pix_ok && j == 0) {
    const float Tf = T_final[p];
    image[3 * p] = notex[3 * p] + c0 + Tf * bg0;
    image[3 * p + 1] = notex[3 * p + 1] + c1 + Tf * bg1;
    image[3 * p + 2] = notex[3 * p + 2] + c2 + Tf * bg2;
  }
}

// ------------------------------------------------------------ backward
template <int IN, int H1, int H2, typename TT>
__global__ void __launch_bounds__(256) k_tex_bwd_f32(
    DevCam c, FieldDev f, int K, int KP, const float* __restrict__ weights, const int* __restrict__ ids,
    const float* __restrict__ depths, const float* __restrict__ d_image,
    const float* __restrict__ d_weights, const float* __restrict__ d_textures,
    float* __restrict__ dweff, float* __restrict__ ddepth, float* __restrict__ feat_out,
    float4* __restrict__ gtex_out, float* __restrict__ gin_out, float* __restrict__ d_table) {
  using A = MlpArch<IN, H1, H2>;
  __shared__ __align__(16) float sW[A::kWeights];
  for (int k = threadIdx.x; k < A::kWeights; k += blockDim.x) sW[k] = f.w[k];
  __syncthreads();
  const long long S = (long long)c.W * c.H * K;
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in_range = s < S;
  const int id = in_range ? ids[s] : -1;
  const bool active = id >= 0;
  float gin[IN];
#pragma unroll
  for (int k = 0; k < IN; ++k) gin[k] = 0.f;
  float3 x = make_float3(0.f, 0.f, 0.f), d = make_float3(0.f, 0.f, 1.f);
  float D = 1.f;
  if (active) {
    const long long p = s / K;
    const float wj = weights[s];
    D = depths[s];
    d = pixel_dir(c, (int)(p % c.W), (int)(p / c.W));
    x = make_float3(c.o[0] + D * d.x, c.o[1] + D * d.y, c.o[2] + D * d.z);
    float feat[IN];
    if (f.feat_mode == 2) {  // left by the forward of this step
#pragma unroll
      for (int k = 0; k < IN; ++k) feat[k] = feat_out[s * IN + k];
    } else {
      hash_features<IN, TT>(f, x, D, feat);
    }
    float out[3], h1[H1], h2[H2 > 0 ? H2 : 1];
    mlp_fwd_f32<IN, H1, H2>(sW, feat, out, h1, h2);
    const float dc0 = d_image[3 * p], dc1 = d_image[3 * p + 1], dc2 = d_image[3 * p + 2];
    float gT[3] = {wj * dc0, wj * dc1, wj * dc2};
    if (d_textures) {
      gT[0] += d_textures[3 * s]; gT[1] += d_textures[3 * s + 1]; gT[2] += d_textures[3 * s + 2];
    }
    float dwe = out[0] * dc0 + out[1] * dc1 + out[2] * dc2;
    if (d_weights) dwe += d_weights[s];
    dweff[s] = dwe;
    mlp_bwd_input_f32<IN, H1, H2>(sW, gT, h1, h2, gin);
    if (f.feat_mode != 2)
      for (int k = 0; k < IN; ++k) feat_out[s * IN + k] = feat[k];
    gtex_out[s] = make_float4(gT[0], gT[1], gT[2], 0.f);
  } else if (in_range) {
    dweff[s] = 0.f;
    ddepth[s] = 0.f;
    if (f.feat_mode != 2)
      for (int k = 0; k < IN; ++k) feat_out[s * IN + k] = 0.f;
    gtex_out[s] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // the hash-grid backward (k_hash_bwd) reads gin and writes ddepth of
  // textured samples
  if (in_range) {
    // level-major: (dL/dh_l0, dL/dh_l1) of level l at gin_out[l * R + row],
    // row = p * KP + j
    const long long R = gin_stride(S / K * KP);
    const long long row = (s / K) * KP + s % K;
    float2* g2 = reinterpret_cast<float2*>(gin_out);
#pragma unroll
    for (int l = 0; l < IN / 2; ++l) g2[l * R + row] = make_float2(gin[2 * l], gin[2 * l + 1]);
  }
  (void)x;
  (void)d;
  (void)D;
  (void)d_table;
}

// Weight gradients: dW_l = sum_s delta_{l+1}[s] (x) a_l[s].  Each CTA walks
// chunks of kChunk samples: it stages the features, recomputes activations
// and deltas in shared memory (SIMT GEMMs), and every thread accumulates the
// weight-gradient entries it owns in registers; one atomic per entry at the
// end.
template <int IN, int H1, int H2>
__global__ void __launch_bounds__(256) k_mlp_wgrad_f32(long long S, const float* __restrict__ w,
                                                        const float* __restrict__ feat,
                                                        const float4* __restrict__ gtex,
                                                        float* __restrict__ d_mlp) {
  using A = MlpArch<IN, H1, H2>;
  constexpr int kChunk = 32;
  constexpr int HL = (H2 > 0) ? H2 : H1;  // width feeding the output layer
  extern __shared__ __align__(16) float sm[];
  float* sW = sm;                              // kWeights
  float* sA0 = sW + A::kWeights;               // kChunk x IN
  float* sA1 = sA0 + kChunk * IN;              // kChunk x H1
  float* sA2 = sA1 + kChunk * H1;              // kChunk x H2
  float* sD3 = sA2 + kChunk * (H2 > 0 ? H2 : 1);  // kChunk x 3
  float* sD2 = sD3 + kChunk * 4;               // kChunk x H2
  float* sD1 = sD2 + kChunk * (H2 > 0 ? H2 : 1);  // kChunk x H1
  for (int k = threadIdx.x; k < A::kWeights; k += blockDim.x) sW[k] = w[k];
  constexpr int kE = (A::kWeights + 255) / 256;
  float acc[kE];
#pragma unroll
  for (int k = 0; k < kE; ++k) acc[k] = 0.f;
  const float* W1 = sW;
  const float* W2 = sW + H1 * IN;
  const float* W3 = sW + A::kOffLast;
  const long long n_chunks = (S + kChunk - 1) / kChunk;
  for (long long ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const long long s0 = ch * kChunk;
    __syncthreads();
    for (int k = threadIdx.x; k < kChunk * IN; k += 256) {
      long long s = s0 + k / IN;
      sA0[k] = s < S ? feat[s0 * IN + k] : 0.f;
    }
    for (int k = threadIdx.x; k < kChunk; k += 256) {
      long long s = s0 + k;
      float4 g = s < S ? gtex[s] : make_float4(0.f, 0.f, 0.f, 0.f);
      sD3[4 * k] = g.x; sD3[4 * k + 1] = g.y; sD3[4 * k + 2] = g.z; sD3[4 * k + 3] = 0.f;
    }
    __syncthreads();
    // h1 = relu(W1 a0)
    for (int k = threadIdx.x; k < kChunk * H1; k += 256) {
      int r = k / H1, o = k % H1;
      float v = 0.f;
      for (int i = 0; i < IN; ++i) v = fmaf(W1[o * IN + i], sA0[r * IN + i], v);
      sA1[k] = fmaxf(v, 0.f);
    }
    __syncthreads();
    if constexpr (H2 > 0) {
      for (int k = threadIdx.x; k < kChunk * H2; k += 256) {
        int r = k / H2, o = k % H2;
        float v = 0.f;
        for (int i = 0; i < H1; ++i) v = fmaf(W2[o * H1 + i], sA1[r * H1 + i], v);
        sA2[k] = fmaxf(v, 0.f);
      }
      __syncthreads();
    }
    const float* aL = (H2 > 0) ? sA2 : sA1;
    float* dL = (H2 > 0) ? sD2 : sD1;
    // delta of the last hidden layer: W3^T d3, masked by ReLU
    for (int k = threadIdx.x; k < kChunk * HL; k += 256) {
      int r = k / HL, i = k % HL;
      float v = W3[i] * sD3[4 * r] + W3[HL + i] * sD3[4 * r + 1] + W3[2 * HL + i] * sD3[4 * r + 2];
      dL[k] = aL[k] > 0.f ? v : 0.f;
    }
    __syncthreads();
    if constexpr (H2 > 0) {
      for (int k = threadIdx.x; k < kChunk * H1; k += 256) {
        int r = k / H1, i = k % H1;
        float v = 0.f;
        for (int o = 0; o < H2; ++o) v = fmaf(W2[o * H1 + i], sD2[r * H2 + o], v);
        sD1[k] = sA1[k] > 0.f ? v : 0.f;
      }
      __syncthreads();
    }
    // accumulate owned entries
#pragma unroll
    for (int k = 0; k < kE; ++k) {
      int e = threadIdx.x + 256 * k;
      if (e >= A::kWeights) continue;
      const float *dsrc, *asrc;
      int o, i, dstride, astride;
      if (e < H1 * IN) {
        o = e / IN; i = e % IN; dsrc = sD1; dstride = H1; asrc = sA0; astride = IN;
      } else if (H2 > 0 && e < A::kOffLast) {
        int ee = e - H1 * IN;
        o = ee / H1; i = ee % H1; dsrc = sD2; dstride = H2; asrc = sA1; astride = H1;
      } else {
        int ee = e - A::kOffLast;
        o = ee / HL; i = ee % HL; dsrc = sD3; dstride = 4; asrc = aL; astride = HL;
      }
      float v = acc[k];
#pragma unroll 4
      for (int r = 0; r < kChunk; ++r) v = fmaf(dsrc[r * dstride + o], asrc[r * astride + i], v);
      acc[k] = v;
    }
  }
#pragma unroll
  for (int k = 0; k < kE; ++k) {
    int e = threadIdx.x + 256 * k;
    if (e < A::kWeights && acc[k] != 0.f) atomicAdd(d_mlp + e, acc[k]);
  }
}

template <int IN, int H1, int H2>
size_t wgrad_smem_f32() {
  using A = MlpArch<IN, H1, H2>;
  constexpr int kChunk = 32;
  constexpr int H2s = H2 > 0 ? H2 : 1;
  return sizeof(float) * (A::kWeights + kChunk * (IN + H1 + H2s + 4 + H2s + H1));
}

// --------------------------------------------------------------- dispatch
template <int IN, int H1, int H2, typename TT>
cudaError_t tex_fwd_f32(const DevCam& c, const nexel_settings& s, const FieldDev& fd,
                               const float* notex, const float* weights, const int* ids,
                               const float* depths, const float* T_final, float* image,
                               float* textures, cudaStream_t st) {
  int KP = 1;
  while (KP < s.K) KP <<= 1;
  long long n = (long long)c.W * c.H * KP;
  unsigned blocks = (unsigned)((n + 255) / 256);
  {
    NEXEL_PROF("texture_fwd_f32", st);
    k_tex_fwd_f32<IN, H1, H2, TT><<<blocks, 256, 0, st>>>(c, fd, s.K, KP, s.bg[0], s.bg[1], s.bg[2],
                                                          notex, weights, ids, depths, T_final,
                                                          image, textures);
  }
  return cudaGetLastError();
}

template <int IN, int H1, int H2, typename TT>
cudaError_t tex_bwd_f32(const DevCam& c, const nexel_settings& s, const FieldDev& fd,
                               char* bws, const BwdLayout& B, const float* weights, const int* ids,
                               const float* depths, const float* d_image, const float* d_weights,
                               const float* d_textures, float* d_table, float* d_mlp,
                               cudaStream_t st) {
  long long S = (long long)c.W * c.H * s.K;
  if (S == 0) return cudaSuccess;
  int KP = 1;
  while (KP < s.K) KP <<= 1;
  {
    NEXEL_PROF("texture_bwd_f32", st);
    k_tex_bwd_f32<IN, H1, H2, TT><<<(unsigned)((S + 255) / 256), 256, 0, st>>>(
        c, fd, s.K, KP, weights, ids, depths, d_image, d_weights, d_textures, (float*)(bws + B.dweff),
        (float*)(bws + B.ddepth), (float*)(bws + B.feat), (float4*)(bws + B.gtex),
        (float*)(bws + B.gin), d_table);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_hash_bwd(c, fd, s.K, KP, (long long)c.W * c.H * KP, false, ids, depths,
                      (const float2*)(bws + B.gin),
                      (float*)(bws + B.ddepth), d_table, st);
  if (e != cudaSuccess || !d_mlp) return e;
  size_t smem = wgrad_smem_f32<IN, H1, H2>();
  e = cudaFuncSetAttribute(k_mlp_wgrad_f32<IN, H1, H2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  long long chunks = (S + 31) / 32;
  unsigned grid = (unsigned)std::min<long long>(chunks, 4LL * nsm);
  {
    NEXEL_PROF("mlp_wgrad_f32", st);
    k_mlp_wgrad_f32<IN, H1, H2><<<grid, 256, smem, st>>>(S, fd.w, (float*)(bws + B.feat),
                                                        (float4*)(bws + B.gtex), d_mlp);
  }
  return cudaGetLastError();
}


}  // namespace nexel
