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
//
// The MLPs with 64-wide hidden layers use the chunked forms further below
// instead (register-tiled SIMT GEMMs over 64-row chunks, the weight
// gradients formed in the same backward kernel); the per-sample kernels
// serve the 8-16-3 MLP.
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

// Register-tiled SIMT GEMM for the chunked forms below: every GEMM of a
// 64-row chunk gives each of the 256 threads a 4 x (N / 16) tile of
// outputs, so one k step costs 4 + N / 16 shared loads for 4 N / 16 FMAs.
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
size_t wgrad_smem_f32() {
  using A = MlpArch<IN, H1, H2>;
  constexpr int kChunk = 32;
  constexpr int H2s = H2 > 0 ? H2 : 1;
  return sizeof(float) * (A::kWeights + kChunk * (IN + H1 + H2s + 4 + H2s + H1));
}

// ------------------------------------------- chunked forms for H1 = 64
// The 16-64-3 and 32-64-64-3 MLPs run over chunks of 64 rows (RC = K
// floor(64 / K) samples, whole pixels): the features (gathered, or read back
// in a training step's backward) go to shared memory and every layer is a
// register-tiled SIMT GEMM (wg::gemm).  The backward also forms the MLP
// weight gradients (tiles in registers across all chunks of the CTA).
namespace f32c {
constexpr int kPH = 65;  // padded row stride of 64-wide activation tiles

// Weights, rows padded: W1 [H1][IN + 1], W2 [H2][H1 + 1], W3 [OUT][HL].
template <int IN, int H1, int H2, int OUT = 3>
struct Ws {
  static constexpr int HL = H2 > 0 ? H2 : H1;
  static constexpr int P1 = IN + 1, P2 = H1 + 1;
  static constexpr int o2 = H1 * P1, o3 = o2 + H2 * P2, total = o3 + OUT * HL;
};
template <int IN, int H1, int H2, int OUT = 3>
__device__ __forceinline__ void load_weights(const float* __restrict__ w, float* sW) {
  using W = Ws<IN, H1, H2, OUT>;
  using A = MlpArch<IN, H1, H2, OUT>;
  for (int k = threadIdx.x; k < H1 * IN; k += blockDim.x) sW[(k / IN) * W::P1 + k % IN] = w[k];
  for (int k = threadIdx.x; k < H2 * H1; k += blockDim.x)
    sW[W::o2 + (k / H1) * W::P2 + k % H1] = w[H1 * IN + k];
  for (int k = threadIdx.x; k < OUT * W::HL; k += blockDim.x) sW[W::o3 + k] = w[A::kOffLast + k];
}

// Features of row `row` for the levels of quarter q (0..3) into sX.
template <int IN, typename TT>
__device__ __forceinline__ void gather_row(const DevCam& c, const FieldDev& f, float* sX, int row,
                                           int q, bool valid, long long p, float D) {
  constexpr int LQ = IN / 8;  // levels per quarter (F = 2)
  float3 x = make_float3(0.f, 0.f, 0.f);
  if (valid) {
    const float3 d = pixel_dir(c, (int)(p % c.W), (int)(p / c.W));
    x = make_float3(c.o[0] + D * d.x, c.o[1] + D * d.y, c.o[2] + D * d.z);
  }
  const TT* tab = reinterpret_cast<const TT*>(f.table);
  const size_t T = (size_t)f.mask + 1;
#pragma unroll
  for (int lq = 0; lq < LQ; ++lq) {
    const int l = q * LQ + lq;
    float ax = 0.f, ay = 0.f, dw = 0.f;
    if (valid) {
      const float sl = f.s[l];
      const float gx = sl * x.x, gy = sl * x.y, gz = sl * x.z;
      const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
      const int cx = (int)fx0, cy = (int)fy0, cz = (int)fz0;
      const float rx = gx - fx0, ry = gy - fy0, rz = gz - fz0;
      const TT* tl = tab + (size_t)l * T * 2;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
        const float w = (dx ? rx : 1.f - rx) * (dy ? ry : 1.f - ry) * (dz ? rz : 1.f - rz);
        const float2 e = load_entry<TT>(tl, hash3(cx + dx, cy + dy, cz + dz, f.mask));
        ax = fmaf(w, e.x, ax);
        ay = fmaf(w, e.y, ay);
      }
      dw = downweight(f.focal, sl, D);
    }
    sX[row * (IN + 1) + 2 * l] = dw * ax;
    sX[row * (IN + 1) + 2 * l + 1] = dw * ay;
  }
}

// h = relu(A W^T) for a 64-row tile A (stride pa) and W [NOUT][K] (stride pw).
template <int NOUT, int K>
__device__ __forceinline__ void dense_relu(const float* sA, int pa, const float* sWl, int pw,
                                           float* sOut) {
  float acc[4][NOUT / 16];
  wg::zero<NOUT>(acc);
  wg::gemm<NOUT, K>([&](int m, int k) { return sA[m * pa + k]; },
                    [&](int n, int k) { return sWl[n * pw + k]; }, acc);
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < NOUT / 16; ++j)
      sOut[(4 * ty + i) * kPH + (NOUT / 16) * tx + j] = fmaxf(acc[i][j], 0.f);
}
}  // namespace f32c

template <int IN, int H1, int H2, typename TT, int OUT = 3>
__global__ void __launch_bounds__(256, 2) k_tex_fwd_f32c(
    DevCam c, FieldDev f, int K, int RC, long long n_chunks, float bg0, float bg1, float bg2,
    const float* __restrict__ notex, const float* __restrict__ weights,
    const int* __restrict__ ids, const float* __restrict__ depths,
    const float* __restrict__ T_final, float* __restrict__ image, float* __restrict__ textures) {
  using W = f32c::Ws<IN, H1, H2, OUT>;
  constexpr int HL = W::HL, PH = f32c::kPH;
  extern __shared__ __align__(16) float sm[];
  float* sW = sm;
  float* sX = sW + W::total;            // 64 x (IN + 1)
  float* sH1 = sX + 64 * (IN + 1);      // 64 x PH
  float* sH2 = sH1 + 64 * PH;           // 64 x PH (two hidden layers)
  float* sT = sH2 + (H2 > 0 ? 64 * PH : 0);  // 64 x 4: textures of the rows
  f32c::load_weights<IN, H1, H2, OUT>(f.w, sW);
  const long long P = (long long)c.W * c.H, S = P * K;
  const int row = threadIdx.x & 63, q = threadIdx.x >> 6;
  for (long long ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const long long s0 = ch * RC;
    __syncthreads();
    {
      const long long s = s0 + row;
      const bool in_rows = row < RC && s < S;
      const bool valid = in_rows && ids[s] >= 0;
      const float D = valid ? depths[s] : 1.f;
      f32c::gather_row<IN, TT>(c, f, sX, row, q, valid, s / K, D);
      if (f.feat_mode == 1 && in_rows) {
        float* fo = reinterpret_cast<float*>(f.feat) + s * IN + q * (IN / 4);
#pragma unroll
        for (int k = 0; k < IN / 4; ++k) fo[k] = sX[row * (IN + 1) + q * (IN / 4) + k];
      }
    }
    __syncthreads();
    f32c::dense_relu<H1, IN>(sX, IN + 1, sW, W::P1, sH1);
    __syncthreads();
    if constexpr (H2 > 0) {
      f32c::dense_relu<H2, H1>(sH1, PH, sW + W::o2, W::P2, sH2);
      __syncthreads();
    }
    const float* sHL = H2 > 0 ? sH2 : sH1;
    if (threadIdx.x < 3 * 64) {  // textures T = W3 h_last (OUT = 48: SH in the ray direction)
      const int r = threadIdx.x / 3, ch3 = threadIdx.x % 3;
      const long long s = s0 + r;
      const bool valid = r < RC && s < S && ids[s] >= 0;
      float v = 0.f;
      if constexpr (OUT == 3) {
        const float* w3 = sW + W::o3 + ch3 * HL;
#pragma unroll 8
        for (int i = 0; i < HL; ++i) v = fmaf(w3[i], sHL[r * PH + i], v);
      } else if (valid) {
        const Sh3 Y = pixel_sh3(c, s / K);
        for (int k = 0; k < 16; ++k) {
          const float* w3 = sW + W::o3 + (3 * k + ch3) * HL;
          float o = 0.f;
#pragma unroll 8
          for (int i = 0; i < HL; ++i) o = fmaf(w3[i], sHL[r * PH + i], o);
          v = fmaf(Y.y[k], o, v);
        }
      }
      v = valid ? v : 0.f;
      sT[4 * r + ch3] = v;
      if (r < RC && s < S) textures[3 * s + ch3] = v;
    }
    __syncthreads();
    if (threadIdx.x < RC / K) {  // composite (Eq. 6) per pixel of the chunk
      const long long p = s0 / K + threadIdx.x;
      if (p < P) {
        float c0 = 0.f, c1 = 0.f, c2 = 0.f;
        for (int j = 0; j < K; ++j) {
          const int r = threadIdx.x * K + j;
          const float wj = weights[p * K + j];
          c0 = fmaf(wj, sT[4 * r], c0);
          c1 = fmaf(wj, sT[4 * r + 1], c1);
          c2 = fmaf(wj, sT[4 * r + 2], c2);
        }
        const float Tf = T_final[p];
        image[3 * p] = notex[3 * p] + c0 + Tf * bg0;
        image[3 * p + 1] = notex[3 * p + 1] + c1 + Tf * bg1;
        image[3 * p + 2] = notex[3 * p + 2] + c2 + Tf * bg2;
      }
    }
  }
}

template <int IN, int H1, int H2, typename TT, int OUT = 3>
__global__ void __launch_bounds__(256, 2) k_tex_bwd_f32c(
    DevCam c, FieldDev f, int K, int KP, int RC, long long n_chunks,
    const float* __restrict__ weights, const int* __restrict__ ids,
    const float* __restrict__ depths, const float* __restrict__ d_image,
    const float* __restrict__ d_weights, const float* __restrict__ d_textures,
    float* __restrict__ dweff, float2* __restrict__ gin, float* __restrict__ d_mlp) {
  using W = f32c::Ws<IN, H1, H2, OUT>;
  using A = MlpArch<IN, H1, H2, OUT>;
  constexpr int HL = W::HL, PH = f32c::kPH, PX = IN + 1;
  constexpr int NG3 = OUT * HL / 256;  // last-layer weight gradients per thread (OUT = 48)
  extern __shared__ __align__(16) float sm[];
  float* sW = sm;
  float* sX = sW + W::total;                  // 64 x PX
  float* sH1 = sX + 64 * PX;                  // 64 x PH
  float* sH2 = sH1 + 64 * PH;                 // 64 x PH (two hidden layers)
  float* sDL = sH2 + (H2 > 0 ? 64 * PH : 0);  // 64 x PH: delta of the last hidden layer
  float* sD1 = sDL + 64 * PH;                 // 64 x PH: delta of h1 (two hidden layers)
  float* sG = sD1 + (H2 > 0 ? 64 * PH : 0);   // 64 x 8: texture gradient, dL/dC, dL/dW
  float* sGin = sH1;                          // 64 x PX: feature gradient (after h1 is used)
  float* sY = sG + 64 * 8;                    // 64 x 16: SH basis of the rows (OUT = 48)
  f32c::load_weights<IN, H1, H2, OUT>(f.w, sW);
  const float* W1 = sW;
  const float* W2 = sW + W::o2;
  const float* W3 = sW + W::o3;
  const long long P = (long long)c.W * c.H, S = P * K;
  const long long R = gin_stride(P * KP);
  const int row = threadIdx.x & 63, q = threadIdx.x >> 6;
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  float g2[4][4], g1[4][IN / 16];
  wg::zero<64>(g2);
  wg::zero<IN>(g1);
  float g3 = 0.f;
  float g3s[OUT == 48 ? NG3 : 1];
#pragma unroll
  for (int j = 0; j < (OUT == 48 ? NG3 : 1); ++j) g3s[j] = 0.f;
  const float* sHL = H2 > 0 ? sH2 : sH1;
  for (long long ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const long long s0 = ch * RC;
    __syncthreads();
    {
      const long long s = s0 + row;
      const bool in_rows = row < RC && s < S;
      const bool valid = in_rows && ids[s] >= 0;
      if (f.feat_mode == 2) {  // the forward of this step left the features
        const float* fi = reinterpret_cast<const float*>(f.feat) + s * IN + q * (IN / 4);
#pragma unroll
        for (int k = 0; k < IN / 4; ++k) sX[row * PX + q * (IN / 4) + k] = in_rows ? fi[k] : 0.f;
      } else {
        const float D = valid ? depths[s] : 1.f;
        f32c::gather_row<IN, TT>(c, f, sX, row, q, valid, s / K, D);
      }
      if (q == 0) {
        float gT0 = 0.f, gT1 = 0.f, gT2 = 0.f, dc0 = 0.f, dc1 = 0.f, dc2 = 0.f, dwx = 0.f;
        if (valid) {
          const long long p = s / K;
          const float wj = weights[s];
          dc0 = d_image[3 * p]; dc1 = d_image[3 * p + 1]; dc2 = d_image[3 * p + 2];
          gT0 = wj * dc0; gT1 = wj * dc1; gT2 = wj * dc2;
          if (d_textures) {
            gT0 += d_textures[3 * s]; gT1 += d_textures[3 * s + 1]; gT2 += d_textures[3 * s + 2];
          }
          if (d_weights) dwx = d_weights[s];
        }
        float* g = sG + 8 * row;
        g[0] = gT0; g[1] = gT1; g[2] = gT2; g[3] = dc0; g[4] = dc1; g[5] = dc2; g[6] = dwx;
        g[7] = valid ? 1.f : 0.f;
        if constexpr (OUT == 48) {
          const Sh3 Y = pixel_sh3(c, valid ? s / K : 0);
#pragma unroll
          for (int k = 0; k < 16; ++k) sY[16 * row + k] = valid ? Y.y[k] : 0.f;
        }
      }
    }
    __syncthreads();
    f32c::dense_relu<H1, IN>(sX, PX, W1, W::P1, sH1);
    __syncthreads();
    if constexpr (H2 > 0) {
      f32c::dense_relu<H2, H1>(sH1, PH, W2, W::P2, sH2);
      __syncthreads();
    }
    // dL/dW_j = T . dL/dC + dL/dW_j (upstream), T = W3 h_last
    if (threadIdx.x < 64) {
      const int r = threadIdx.x;
      const long long s = s0 + r;
      if (r < RC && s < S) {
        const float* g = sG + 8 * r;
        float T0 = 0.f, T1 = 0.f, T2 = 0.f;
        if constexpr (OUT == 3) {
#pragma unroll 8
          for (int i = 0; i < HL; ++i) {
            const float h = sHL[r * PH + i];
            T0 = fmaf(W3[i], h, T0);
            T1 = fmaf(W3[HL + i], h, T1);
            T2 = fmaf(W3[2 * HL + i], h, T2);
          }
        } else if (g[7] != 0.f) {
          for (int k = 0; k < 16; ++k) {
            float o0 = 0.f, o1 = 0.f, o2 = 0.f;
            const float* w3 = W3 + 3 * k * HL;
#pragma unroll 8
            for (int i = 0; i < HL; ++i) {
              const float h = sHL[r * PH + i];
              o0 = fmaf(w3[i], h, o0);
              o1 = fmaf(w3[HL + i], h, o1);
              o2 = fmaf(w3[2 * HL + i], h, o2);
            }
            const float y = sY[16 * r + k];
            T0 = fmaf(y, o0, T0);
            T1 = fmaf(y, o1, T1);
            T2 = fmaf(y, o2, T2);
          }
        }
        dweff[s] = g[7] != 0.f ? T0 * g[3] + T1 * g[4] + T2 * g[5] + g[6] : 0.f;
      }
    }
    // delta of the last hidden layer: (W3^T gT) * [h > 0]
    for (int k = threadIdx.x; k < 64 * HL; k += 256) {
      const int r = k / HL, cc = k % HL;
      const float* g = sG + 8 * r;
      float v;
      if constexpr (OUT == 3) {
        v = W3[cc] * g[0] + W3[HL + cc] * g[1] + W3[2 * HL + cc] * g[2];
      } else {
        // the output gradient is Y_k gT_ch at output 3k + ch
        v = 0.f;
        for (int kk = 0; kk < 16; ++kk) {
          const float* w3 = W3 + 3 * kk * HL + cc;
          v = fmaf(sY[16 * r + kk], w3[0] * g[0] + w3[HL] * g[1] + w3[2 * HL] * g[2], v);
        }
      }
      sDL[r * PH + cc] = sHL[r * PH + cc] > 0.f ? v : 0.f;
    }
    __syncthreads();
    const float* sDH1 = sDL;  // delta of h1
    if constexpr (H2 > 0) {  // d1 = (d2 W2) * [h1 > 0]
      float acc[4][4];
      wg::zero<64>(acc);
      wg::gemm<64, H2>([&](int m, int k) { return sDL[m * PH + k]; },
                       [&](int n, int k) { return W2[k * W::P2 + n]; }, acc);
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
      wg::gemm<64, 64>([&](int m, int k) { return sDL[k * PH + m]; },
                       [&](int n, int k) { return sH1[k * PH + n]; }, g2);
    }
    // dW1[o][i] += sum_r d1[r][o] x[r][i]
    wg::gemm<IN, 64>([&](int m, int k) { return sDH1[k * PH + m]; },
                     [&](int n, int k) { return sX[k * PX + n]; }, g1);
    // dW3[o][i] += sum_r gT[r][o] h_last[r][i]
    if constexpr (OUT == 3) {
      if (threadIdx.x < 3 * HL) {
        const int o = threadIdx.x / HL, i = threadIdx.x % HL;
        float v = g3;
#pragma unroll 8
        for (int r = 0; r < 64; ++r) v = fmaf(sG[8 * r + o], sHL[r * PH + i], v);
        g3 = v;
      }
    } else {
      // weight (3k + ch, i): sum_r Y_k[r] gT_ch[r] h_last[r][i]
#pragma unroll
      for (int j = 0; j < NG3; ++j) {
        const int e = threadIdx.x + 256 * j, o = e / HL, i = e % HL;
        const int kk = o / 3, chn = o % 3;
        float v = g3s[j];
        for (int r = 0; r < 64; ++r)
          v = fmaf(sY[16 * r + kk] * sG[8 * r + chn], sHL[r * PH + i], v);
        g3s[j] = v;
      }
    }
    // feature gradient d1 W1 -> sGin (h1 is no longer needed)
    {
      float acc[4][IN / 16];
      wg::zero<IN>(acc);
      wg::gemm<IN, H1>([&](int m, int k) { return sDH1[m * PH + k]; },
                       [&](int n, int k) { return W1[k * W::P1 + n]; }, acc);
      __syncthreads();  // every thread is done reading h1
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < IN / 16; ++j) sGin[(4 * ty + i) * PX + (IN / 16) * tx + j] = acc[i][j];
    }
    __syncthreads();
    // level-major feature gradient, row p KP + j
    for (int k = threadIdx.x; k < 64 * (IN / 2); k += 256) {
      const int r = k % 64, l = k / 64;
      const long long s = s0 + r;
      if (r < RC && s < S) {
        const long long rk = (s / K) * KP + s % K;
        gin[(long long)l * R + rk] = make_float2(sGin[r * PX + 2 * l], sGin[r * PX + 2 * l + 1]);
      }
    }
  }
  if (!d_mlp) return;
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
  if constexpr (OUT == 3) {
    if (threadIdx.x < 3 * HL) atomicAdd(d_mlp + A::kOffLast + threadIdx.x, g3);
  } else {
#pragma unroll
    for (int j = 0; j < NG3; ++j) atomicAdd(d_mlp + A::kOffLast + threadIdx.x + 256 * j, g3s[j]);
  }
}

template <int IN, int H1, int H2, int OUT = 3>
constexpr size_t f32c_fwd_smem() {
  using W = f32c::Ws<IN, H1, H2, OUT>;
  return sizeof(float) * (W::total + 64 * (IN + 1) + 64 * f32c::kPH * (H2 > 0 ? 2 : 1) + 64 * 4);
}
template <int IN, int H1, int H2, int OUT = 3>
constexpr size_t f32c_bwd_smem() {
  using W = f32c::Ws<IN, H1, H2, OUT>;
  return sizeof(float) * (W::total + 64 * (IN + 1) + 64 * f32c::kPH * (H2 > 0 ? 4 : 2) + 64 * 8 +
                          (OUT == 48 ? 64 * 16 : 0));
}

// --------------------------------------------------------------- dispatch
template <int IN, int H1, int H2, typename TT, int OUT = 3>
cudaError_t tex_fwd_f32(const DevCam& c, const nexel_settings& s, const FieldDev& fd,
                               const float* notex, const float* weights, const int* ids,
                               const float* depths, const float* T_final, float* image,
                               float* textures, cudaStream_t st) {
  static_assert(OUT == 3 || H1 == 64, "SH outputs need the chunked kernels");
  if constexpr (H1 == 64) {
    const long long S = (long long)c.W * c.H * s.K;
    if (S == 0) return cudaSuccess;
    const int RC = s.K * (64 / s.K);
    const long long n_chunks = (S + RC - 1) / RC;
    const size_t smem = f32c_fwd_smem<IN, H1, H2, OUT>();
    cudaError_t e = cudaFuncSetAttribute(k_tex_fwd_f32c<IN, H1, H2, TT, OUT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsm = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid =
        (unsigned)std::min<long long>(n_chunks, (long long)current_tuning().f32_ctas * nsm);
    NEXEL_PROF("texture_fwd_f32", st);
    k_tex_fwd_f32c<IN, H1, H2, TT, OUT><<<grid, 256, smem, st>>>(c, fd, s.K, RC, n_chunks, s.bg[0],
                                                           s.bg[1], s.bg[2], notex, weights, ids,
                                                           depths, T_final, image, textures);
    return cudaGetLastError();
  }
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

template <int IN, int H1, int H2, typename TT, int OUT = 3>
cudaError_t tex_bwd_f32(const DevCam& c, const nexel_settings& s, const FieldDev& fd,
                               char* bws, const BwdLayout& B, const float* weights, const int* ids,
                               const float* depths, const float* d_image, const float* d_weights,
                               const float* d_textures, float* d_table, float* d_mlp,
                               cudaStream_t st) {
  long long S = (long long)c.W * c.H * s.K;
  if (S == 0) return cudaSuccess;
  int KP = 1;
  while (KP < s.K) KP <<= 1;
  static_assert(OUT == 3 || H1 == 64, "SH outputs need the chunked kernels");
  if constexpr (H1 == 64) {
    const int RC = s.K * (64 / s.K);
    const long long n_chunks = (S + RC - 1) / RC;
    const size_t smem = f32c_bwd_smem<IN, H1, H2, OUT>();
    cudaError_t e = cudaFuncSetAttribute(k_tex_bwd_f32c<IN, H1, H2, TT, OUT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsm = 152, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid =
        (unsigned)std::min<long long>(n_chunks, (long long)current_tuning().f32_ctas * nsm);
    {
      NEXEL_PROF("texture_bwd_f32", st);
      k_tex_bwd_f32c<IN, H1, H2, TT, OUT><<<grid, 256, smem, st>>>(
          c, fd, s.K, KP, RC, n_chunks, weights, ids, depths, d_image, d_weights, d_textures,
          (float*)(bws + B.dweff), (float2*)(bws + B.gin), d_mlp);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_hash_bwd(c, fd, s.K, KP, (long long)c.W * c.H * KP, false, ids, depths,
                           (const float2*)(bws + B.gin), (float*)(bws + B.ddepth), d_table, st);
  }
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
