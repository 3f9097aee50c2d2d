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

// Register-tiled form for H1 = 64 (the 16-64-3 and 32-64-64-3 MLPs): chunks
// of 64 samples; every GEMM of the chunk (forward recompute, deltas, weight
// gradients) gives each of the 256 threads a 4 x (N / 16) tile of outputs,
// so one k step costs 4 + N / 16 shared loads for 4 N / 16 FMAs.  The
// weight-gradient tiles stay in registers across all chunks of the CTA.
namespace wg {
constexpr int kR = 64;  // samples per chunk
// C[m][n] = sum_k A(m, k) B(n, k), M = 64, thread (ty, tx) = (t / 16, t % 16)
// owns rows 4 ty .. 4 ty + 3 and columns TN tx .. TN tx + TN - 1.
template <int N, int K, typename FA, typename FB>
__device__ __forceinline__ void gemm(FA a, FB b, float (&acc)[4][N / 16]) {
  constexpr int TN = N / 16;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll 4
  for (int k = 0; k < K; ++k) {
    float av[4], bv[TN];
#pragma unroll
    for (int i = 0; i < 4; ++i) av[i] = a(4 * ty + i, k);
#pragma unroll
    for (int j = 0; j < TN; ++j) bv[j] = b(TN * tx + j, k);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
  }
}
template <int N>
__device__ __forceinline__ void zero(float (&acc)[4][N / 16]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < N / 16; ++j) acc[i][j] = 0.f;
}
}  // namespace wg

template <int IN, int H1, int H2>
__global__ void __launch_bounds__(256, 2) k_mlp_wgrad_f32_tiled(long long S,
                                                                 const float* __restrict__ w,
                                                                 const float* __restrict__ feat,
                                                                 const float4* __restrict__ gtex,
                                                                 float* __restrict__ d_mlp) {
  static_assert(H1 == 64 && (H2 == 0 || H2 == 64) && IN % 16 == 0, "tiled shapes");
  using A = MlpArch<IN, H1, H2>;
  constexpr int HL = (H2 > 0) ? H2 : H1;
  constexpr int R = wg::kR;
  constexpr int PX = IN + 1, PH = 64 + 1;  // padded row strides
  constexpr int PW1 = IN + 1, PW2 = H1 + 1;  // padded weight rows (no bank conflicts)
  constexpr int kWs = H1 * PW1 + H2 * PW2 + 3 * HL;
  extern __shared__ __align__(16) float sm[];
  float* sW = sm;                       // weights, rows padded
  float* sX = sW + kWs;                 // R x PX
  float* sH1 = sX + R * PX;             // R x PH
  float* sH2 = sH1 + R * PH;            // R x PH (two hidden layers)
  float* sD3 = sH2 + R * PH;            // R x 4
  float* sDL = sD3 + R * 4;             // R x PH: delta of the last hidden layer
  float* sD1 = sDL + R * PH;            // R x PH: delta of h1 (two hidden layers)
  for (int k = threadIdx.x; k < H1 * IN; k += blockDim.x) sW[(k / IN) * PW1 + k % IN] = w[k];
  for (int k = threadIdx.x; k < H2 * H1; k += blockDim.x)
    sW[H1 * PW1 + (k / H1) * PW2 + k % H1] = w[H1 * IN + k];
  for (int k = threadIdx.x; k < 3 * HL; k += blockDim.x)
    sW[H1 * PW1 + H2 * PW2 + k] = w[A::kOffLast + k];
  const float* W1 = sW;                          // [H1][PW1]
  const float* W2 = sW + H1 * PW1;               // [H2][PW2]
  const float* W3 = sW + H1 * PW1 + H2 * PW2;    // [3][HL]
  const float* sHL = (H2 > 0) ? sH2 : sH1;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  // weight-gradient tiles: dW2 (or dW1 when one hidden layer) as 64 x 64,
  // dW1 as 64 x IN (two hidden layers), dW3 entry per thread
  float g2[4][64 / 16], g1[4][IN / 16];
  wg::zero<64>(g2);
  wg::zero<IN>(g1);
  float g3 = 0.f;
  const long long n_chunks = (S + R - 1) / R;
  for (long long ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const long long s0 = ch * R;
    __syncthreads();
    for (int k = threadIdx.x; k < R * IN; k += 256) {
      const int r = k / IN, i = k % IN;
      sX[r * PX + i] = (s0 + r < S) ? feat[s0 * IN + k] : 0.f;
    }
    for (int r = threadIdx.x; r < R; r += 256) {
      const float4 g = (s0 + r < S) ? gtex[s0 + r] : make_float4(0.f, 0.f, 0.f, 0.f);
      sD3[4 * r] = g.x; sD3[4 * r + 1] = g.y; sD3[4 * r + 2] = g.z; sD3[4 * r + 3] = 0.f;
    }
    __syncthreads();
    {  // h1 = relu(X W1^T)
      float acc[4][64 / 16];
      wg::zero<64>(acc);
      wg::gemm<64, IN>([&](int m, int k) { return sX[m * PX + k]; },
                       [&](int n, int k) { return W1[n * PW1 + k]; }, acc);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sH1[(4 * ty + i) * PH + 4 * tx + j] = fmaxf(acc[i][j], 0.f);
    }
    __syncthreads();
    if constexpr (H2 > 0) {  // h2 = relu(h1 W2^T)
      float acc[4][64 / 16];
      wg::zero<64>(acc);
      wg::gemm<64, H1>([&](int m, int k) { return sH1[m * PH + k]; },
                       [&](int n, int k) { return W2[n * PW2 + k]; }, acc);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) sH2[(4 * ty + i) * PH + 4 * tx + j] = fmaxf(acc[i][j], 0.f);
      __syncthreads();
    }
    // delta of the last hidden layer: (W3^T d3) * [h > 0]
    for (int k = threadIdx.x; k < R * HL; k += 256) {
      const int r = k / HL, c = k % HL;
      const float v = W3[c] * sD3[4 * r] + W3[HL + c] * sD3[4 * r + 1] + W3[2 * HL + c] * sD3[4 * r + 2];
      sDL[r * PH + c] = sHL[r * PH + c] > 0.f ? v : 0.f;
    }
    __syncthreads();
    const float* sDH1 = sDL;  // delta of h1
    if constexpr (H2 > 0) {  // d1 = (d2 W2) * [h1 > 0]
      float acc[4][64 / 16];
      wg::zero<64>(acc);
      wg::gemm<64, H2>([&](int m, int k) { return sDL[m * PH + k]; },
                       [&](int n, int k) { return W2[k * PW2 + n]; }, acc);
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int m = 4 * ty + i, n = 4 * tx + j;
          sD1[m * PH + n] = sH1[m * PH + n] > 0.f ? acc[i][j] : 0.f;
        }
      __syncthreads();
      sDH1 = sD1;
      // dW2[o][i] += sum_r d2[r][o] h1[r][i]
      wg::gemm<64, R>([&](int m, int k) { return sDL[k * PH + m]; },
                      [&](int n, int k) { return sH1[k * PH + n]; }, g2);
    }
    // dW1[o][i] += sum_r d1[r][o] x[r][i]
    if constexpr (H2 > 0) {
      wg::gemm<IN, R>([&](int m, int k) { return sDH1[k * PH + m]; },
                      [&](int n, int k) { return sX[k * PX + n]; }, g1);
    } else {
      wg::gemm<IN, R>([&](int m, int k) { return sDL[k * PH + m]; },
                      [&](int n, int k) { return sX[k * PX + n]; }, g1);
    }
    // dW3[o][i] += sum_r d3[r][o] h_last[r][i]
    if (threadIdx.x < 3 * HL) {
      const int o = threadIdx.x / HL, i = threadIdx.x % HL;
      float v = g3;
#pragma unroll 8
      for (int r = 0; r < R; ++r) v = fmaf(sD3[4 * r + o], sHL[r * PH + i], v);
      g3 = v;
    }
  }
  // one atomic per owned entry
  if constexpr (H2 > 0) {
    float* dW2 = d_mlp + H1 * IN;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) atomicAdd(dW2 + (4 * ty + i) * H1 + 4 * tx + j, g2[i][j]);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < IN / 16; ++j)
      atomicAdd(d_mlp + (4 * ty + i) * IN + (IN / 16) * tx + j, g1[i][j]);
  if (threadIdx.x < 3 * HL) atomicAdd(d_mlp + A::kOffLast + threadIdx.x, g3);
}

template <int IN, int H1, int H2>
size_t wgrad_smem_f32_tiled() {
  using A = MlpArch<IN, H1, H2>;
  constexpr int R = wg::kR;
  constexpr int HL = (H2 > 0) ? H2 : H1;
  (void)sizeof(A);
  return sizeof(float) * (H1 * (IN + 1) + H2 * (H1 + 1) + 3 * HL + R * (IN + 1) + 4 * R * 65 + R * 4);
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
  if constexpr (H1 == 64) {
    const size_t smem = wgrad_smem_f32_tiled<IN, H1, H2>();
    e = cudaFuncSetAttribute(k_mlp_wgrad_f32_tiled<IN, H1, H2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsm = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long chunks = (S + wg::kR - 1) / wg::kR;
    const unsigned grid = (unsigned)std::min<long long>(chunks, 2LL * nsm);
    NEXEL_PROF("mlp_wgrad_f32", st);
    k_mlp_wgrad_f32_tiled<IN, H1, H2><<<grid, 256, smem, st>>>(
        S, fd.w, (float*)(bws + B.feat), (float4*)(bws + B.gtex), d_mlp);
    return cudaGetLastError();
  }
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
