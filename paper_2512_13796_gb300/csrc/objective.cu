// Training objective of Sec. 5 ("Losses") and the Adam step of the 3DGS
// training scheme the paper follows.
//
// Image-space terms (nexel_loss_image), per pixel, in five launches:
//   k_ssim_h    horizontal 11-tap Gaussian sums of x, y, x^2, y^2, xy per
//               channel (x = render, y = target)
//   k_loss_px   vertical sums -> local statistics -> SSIM and its partial
//               derivatives A, B, C with respect to the local mean, E[x^2]
//               and E[xy]; the L1, texture and alpha terms with their
//               gradients (d_weights, d_textures); per-block partial sums
//   k_ssim_h3   horizontal sums of A, B, C
//   k_ssim_grad vertical sums -> dSSIM/dx = sum_p w(p - q) (A + 2 x_q B +
//               y_q C) (the window is symmetric, so the adjoint of the
//               zero-padded correlation is the same correlation); d_image
//   k_values    the partial sums in a fixed order (deterministic values)
// Parameter-space terms (nexel_loss_params): the opacity and grid
// regularisers, added into the parameter gradients, and the total.
#include "common.cuh"

#include <cmath>

namespace nexel {
namespace {

constexpr int kWin = 11, kHalf = 5;
constexpr float kC1 = 0.01f * 0.01f, kC2 = 0.03f * 0.03f;
constexpr int kLossThreads = 256;
constexpr int kParamBlocks = 1024;

struct Taps {
  float w[kWin];
};

Taps gaussian_taps() {
  // normalised 1-D Gaussian, sigma 1.5 (the 2-D window is its outer product)
  Taps t;
  double g[kWin], s = 0.0;
  for (int i = 0; i < kWin; ++i) {
    const double r = i - kHalf;
    g[i] = std::exp(-r * r / (2.0 * 1.5 * 1.5));
    s += g[i];
  }
  for (int i = 0; i < kWin; ++i) t.w[i] = (float)(g[i] / s);
  return t;
}

struct LossLayout {
  size_t hstat, abc, habc, partial, total;
  long long P;
  int nblk;
};

size_t al(size_t x) { return (x + 255) & ~size_t(255); }

LossLayout loss_layout(int W, int H) {
  LossLayout L;
  L.P = (long long)W * H;
  L.nblk = (int)((L.P + kLossThreads - 1) / kLossThreads);
  size_t o = 0;
  L.hstat = o; o += al((size_t)L.P * 15 * 4);    // [P][3][5]
  L.abc = o; o += al((size_t)L.P * 9 * 4);       // [P][3][3]
  L.habc = o; o += al((size_t)L.P * 9 * 4);      // [P][3][3]
  L.partial = o;
  o += al((size_t)std::max(L.nblk, kParamBlocks) * 4 * 4);
  L.total = o;
  return L;
}

__global__ void k_ssim_h(int W, int H, Taps t, const float* __restrict__ x,
                         const float* __restrict__ y, float* __restrict__ hstat) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)W * H) return;
  const int px = (int)(p % W);
  const long long row = p - px;
  float s[3][5] = {};
#pragma unroll
  for (int k = 0; k < kWin; ++k) {
    const int xx = px + k - kHalf;
    if (xx < 0 || xx >= W) continue;  // zero padding
    const float w = t.w[k];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float a = __ldg(x + 3 * (row + xx) + c), b = __ldg(y + 3 * (row + xx) + c);
      s[c][0] = fmaf(w, a, s[c][0]);
      s[c][1] = fmaf(w, b, s[c][1]);
      s[c][2] = fmaf(w, a * a, s[c][2]);
      s[c][3] = fmaf(w, b * b, s[c][3]);
      s[c][4] = fmaf(w, a * b, s[c][4]);
    }
  }
  float* o = hstat + (size_t)p * 15;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int q = 0; q < 5; ++q) o[5 * c + q] = s[c][q];
}

__device__ __forceinline__ float block_sum(float v, float* s_w) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s_w[warp] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w];
  return t;  // valid in thread 0
}

__device__ __forceinline__ float sgnf(float v) { return v > 0.f ? 1.f : (v < 0.f ? -1.f : 0.f); }

template <int K>
__global__ void __launch_bounds__(kLossThreads) k_loss_px(
    int W, int H, Taps t, float lam_texture, float lam_alpha, const float* __restrict__ hstat,
    const float* __restrict__ target, const float* __restrict__ weights,
    const float* __restrict__ textures, float* __restrict__ abc, float* __restrict__ d_weights,
    float* __restrict__ d_textures, float* __restrict__ partial) {
  __shared__ float s_w[32];
  const long long P = (long long)W * H;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float ssum = 0.f, tsum = 0.f, asum = 0.f;
  if (p < P) {
    const int px = (int)(p % W), py = (int)(p / W);
    float s[3][5] = {};
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
      const int yy = py + k - kHalf;
      if (yy < 0 || yy >= H) continue;
      const float w = t.w[k];
      const float* h = hstat + ((size_t)yy * W + px) * 15;
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int q = 0; q < 5; ++q) s[c][q] = fmaf(w, __ldg(h + 5 * c + q), s[c][q]);
    }
    float* o = abc + (size_t)p * 9;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float mx = s[c][0], my = s[c][1];
      const float vx = s[c][2] - mx * mx, vy = s[c][3] - my * my, cxy = s[c][4] - mx * my;
      const float l1 = 2.f * mx * my + kC1, l2 = mx * mx + my * my + kC1;
      const float c1 = 2.f * cxy + kC2, c2 = vx + vy + kC2;
      const float S = (l1 * c1) / (l2 * c2);
      ssum += S;
      o[3 * c] = S * (2.f * my / l1 - 2.f * my / c1 - 2.f * mx / l2 + 2.f * mx / c2);
      o[3 * c + 1] = -S / c2;
      o[3 * c + 2] = 2.f * S / c1;
    }
    if constexpr (K > 0) {
      // L_texture (pixels without textured weight add nothing) and L_alpha
      const float n3 = 1.f / (3.f * (float)P), n1 = 1.f / (float)P;
      float Wj[K], sw = 0.f, tb[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int j = 0; j < K; ++j) {
        Wj[j] = weights[p * K + j];
        sw += Wj[j];
#pragma unroll
        for (int c = 0; c < 3; ++c) tb[c] = fmaf(Wj[j], textures[(p * K + j) * 3 + c], tb[c]);
      }
      asum = 1.f - sw;
      float sg[3] = {0.f, 0.f, 0.f};
      const float inv = sw > 0.f ? 1.f / sw : 0.f;
      if (sw > 0.f) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          tb[c] *= inv;
          const float r = tb[c] - target[3 * p + c];
          tsum += fabsf(r);
          sg[c] = sgnf(r) * n3;
        }
      }
#pragma unroll
      for (int j = 0; j < K; ++j) {
        float g = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float tj = textures[(p * K + j) * 3 + c];
          g = fmaf(sg[c], tj - tb[c], g);
          d_textures[(p * K + j) * 3 + c] = lam_texture * sg[c] * Wj[j] * inv;
        }
        d_weights[p * K + j] = lam_texture * g * inv - lam_alpha * n1;
      }
    }
  }
  // per-block sums: SSIM, texture, alpha (L1 is summed in k_ssim_grad)
  const float a = block_sum(ssum, s_w);
  const float b = block_sum(tsum, s_w);
  const float c = block_sum(asum, s_w);
  if (threadIdx.x == 0) {
    partial[4 * blockIdx.x + 1] = a;
    partial[4 * blockIdx.x + 2] = b;
    partial[4 * blockIdx.x + 3] = c;
  }
}

__global__ void k_ssim_h3(int W, int H, Taps t, const float* __restrict__ abc,
                          float* __restrict__ habc) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (long long)W * H) return;
  const int px = (int)(p % W);
  const long long row = p - px;
  float s[9] = {};
#pragma unroll
  for (int k = 0; k < kWin; ++k) {
    const int xx = px + k - kHalf;
    if (xx < 0 || xx >= W) continue;
    const float w = t.w[k];
    const float* a = abc + (size_t)(row + xx) * 9;
#pragma unroll
    for (int q = 0; q < 9; ++q) s[q] = fmaf(w, __ldg(a + q), s[q]);
  }
  float* o = habc + (size_t)p * 9;
#pragma unroll
  for (int q = 0; q < 9; ++q) o[q] = s[q];
}

__global__ void __launch_bounds__(kLossThreads) k_ssim_grad(
    int W, int H, Taps t, float lam_dssim, const float* __restrict__ habc,
    const float* __restrict__ x, const float* __restrict__ y, float* __restrict__ d_image,
    float* __restrict__ partial) {
  __shared__ float s_w[32];
  const long long P = (long long)W * H;
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float l1sum = 0.f;
  if (p < P) {
    const int px = (int)(p % W), py = (int)(p / W);
    float s[9] = {};
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
      const int yy = py + k - kHalf;
      if (yy < 0 || yy >= H) continue;
      const float w = t.w[k];
      const float* a = habc + ((size_t)yy * W + px) * 9;
#pragma unroll
      for (int q = 0; q < 9; ++q) s[q] = fmaf(w, __ldg(a + q), s[q]);
    }
    const float invM = 1.f / (3.f * (float)P);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const float xv = x[3 * p + c], yv = y[3 * p + c];
      const float dS = s[3 * c] + 2.f * xv * s[3 * c + 1] + yv * s[3 * c + 2];
      const float r = xv - yv;
      l1sum += fabsf(r);
      d_image[3 * p + c] = (1.f - lam_dssim) * sgnf(r) * invM - lam_dssim * dS * invM;
    }
  }
  const float a = block_sum(l1sum, s_w);
  if (threadIdx.x == 0) partial[4 * blockIdx.x] = a;
}

// values[0..4] = L1, D-SSIM, L_texture, L_alpha, L_image + lambda-weighted
// texture and alpha terms; fixed summation order.
__global__ void k_values(int nblk, long long P, int K, float lam_dssim, float lam_texture,
                         float lam_alpha, const float* __restrict__ partial,
                         float* __restrict__ values) {
  __shared__ float s_w[32];
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[q] += partial[4 * b + q];
  float tot[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) tot[q] = block_sum(acc[q], s_w);
  if (threadIdx.x == 0) {
    const float M = 3.f * (float)P;
    const float l1 = tot[0] / M, dssim = 1.f - tot[1] / M;
    const float tex = K > 0 ? tot[2] / M : 0.f, alpha = K > 0 ? tot[3] / (float)P : 0.f;
    values[0] = l1;
    values[1] = dssim;
    values[2] = tex;
    values[3] = alpha;
    values[4] = (1.f - lam_dssim) * l1 + lam_dssim * dssim + lam_texture * tex + lam_alpha * alpha;
  }
}

struct InvS3 {
  float v[NEXEL_MAX_LEVELS];  // s_l^-3
};

// Opacity and grid regularisers: gradients added, per-block partial sums.
__global__ void k_loss_params(int N, const float* __restrict__ opacity, long long n_table,
                              long long level_size, int L, InvS3 inv_s3,
                              const float* __restrict__ table, float lam_opacity, float lam_grid,
                              float* __restrict__ d_opacity, float* __restrict__ d_table,
                              float* __restrict__ partial) {
  __shared__ float s_w[32];
  float osum = 0.f, gsum = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
    osum += opacity[i];
    if (d_opacity) d_opacity[i] += lam_opacity / (float)N;
  }
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_table; i += stride) {
    const int l = (int)min((long long)(L - 1), i / level_size);
    const float h = table[i], w = inv_s3.v[l];
    gsum = fmaf(w * h, h, gsum);
    if (d_table) d_table[i] += lam_grid * 2.f * w * h;
  }
  const float a = block_sum(osum, s_w);
  const float b = block_sum(gsum, s_w);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = a;
    partial[2 * blockIdx.x + 1] = b;
  }
}

__global__ void k_values_params(int nblk, int N, float lam_opacity, float lam_grid,
                                const float* __restrict__ partial, float* __restrict__ values) {
  __shared__ float s_w[32];
  float a = 0.f, b = 0.f;
  for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
    a += partial[2 * i];
    b += partial[2 * i + 1];
  }
  a = block_sum(a, s_w);
  b = block_sum(b, s_w);
  if (threadIdx.x == 0) {
    const float lo = N > 0 ? a / (float)N : 0.f;
    values[5] = lo;
    values[6] = b;
    values[7] = values[4] + lam_opacity * lo + lam_grid * b;
  }
}

// Adam over up to kAdamMax tensors per launch (blockIdx.y = tensor).
constexpr int kAdamMax = 16;
struct AdamArgs {
  float* p[kAdamMax];
  const float* g[kAdamMax];
  float* m[kAdamMax];
  float* v[kAdamMax];
  long long n[kAdamMax];
  float lr[kAdamMax];
};

__global__ void k_adam(AdamArgs a, float beta1, float beta2, float eps, float c1, float c2) {
  const int t = blockIdx.y;
  float* __restrict__ p = a.p[t];
  const float* __restrict__ g = a.g[t];
  float* __restrict__ m = a.m[t];
  float* __restrict__ v = a.v[t];
  const long long n = a.n[t];
  const float lr = a.lr[t];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float gi = g[i];
    const float mi = fmaf(beta1, m[i], (1.f - beta1) * gi);
    const float vi = fmaf(beta2, v[i], (1.f - beta2) * gi * gi);
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

bool lw_ok(const nexel_loss_weights* lw) {
  return lw && std::isfinite(lw->dssim) && std::isfinite(lw->alpha) &&
         std::isfinite(lw->texture) && std::isfinite(lw->opacity) && std::isfinite(lw->grid);
}

}  // namespace
}  // namespace nexel

using namespace nexel;

extern "C" {

int nexel_loss_workspace_size(int width, int height, size_t* bytes) {
  if (width <= 0 || height <= 0 || width > 16384 || height > 16384 || !bytes)
    return NEXEL_ERR_INVALID_ARG;
  *bytes = loss_layout(width, height).total;
  return NEXEL_OK;
}

int nexel_loss_image(int width, int height, int K, const nexel_loss_weights* lw,
                     const float* image, const float* target, const float* weights,
                     const float* textures, void* ws, size_t ws_bytes, float* values,
                     float* d_image, float* d_weights, float* d_textures, nexel_stream_t stream) {
  if (width <= 0 || height <= 0 || width > 16384 || height > 16384 || K < 0 ||
      K > NEXEL_MAX_K || !lw_ok(lw) || !image || !target || !ws || !values || !d_image)
    return NEXEL_ERR_INVALID_ARG;
  if (K > 0 && (!weights || !textures || !d_weights || !d_textures)) return NEXEL_ERR_INVALID_ARG;
  const LossLayout L = loss_layout(width, height);
  if (ws_bytes < L.total) return NEXEL_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)ws;
  const Taps t = gaussian_taps();
  const unsigned grid = (unsigned)L.nblk;
  float* hstat = (float*)(w + L.hstat);
  float* abc = (float*)(w + L.abc);
  float* habc = (float*)(w + L.habc);
  float* part = (float*)(w + L.partial);
  {
    NEXEL_PROF("loss_ssim_h", st);
    k_ssim_h<<<grid, kLossThreads, 0, st>>>(width, height, t, image, target, hstat);
  }
  {
    NEXEL_PROF("loss_px", st);
    switch (K) {
#define NEXEL_LPX(k)                                                                            \
  case k:                                                                                       \
    k_loss_px<k><<<grid, kLossThreads, 0, st>>>(width, height, t, lw->texture, lw->alpha, hstat, \
                                                target, weights, textures, abc, d_weights,      \
                                                d_textures, part);                              \
    break;
      NEXEL_LPX(0) NEXEL_LPX(1) NEXEL_LPX(2) NEXEL_LPX(3) NEXEL_LPX(4) NEXEL_LPX(5) NEXEL_LPX(6)
      NEXEL_LPX(7) NEXEL_LPX(8)
#undef NEXEL_LPX
      default: return NEXEL_ERR_INVALID_ARG;
    }
  }
  {
    NEXEL_PROF("loss_ssim_h3", st);
    k_ssim_h3<<<grid, kLossThreads, 0, st>>>(width, height, t, abc, habc);
  }
  {
    NEXEL_PROF("loss_ssim_grad", st);
    k_ssim_grad<<<grid, kLossThreads, 0, st>>>(width, height, t, lw->dssim, habc, image, target,
                                               d_image, part);
  }
  {
    NEXEL_PROF("loss_values", st);
    k_values<<<1, 1024, 0, st>>>(L.nblk, L.P, K, lw->dssim, lw->texture, lw->alpha, part, values);
  }
  return cudaGetLastError() == cudaSuccess ? NEXEL_OK : NEXEL_ERR_CUDA;
}

int nexel_loss_params(int N, const float* opacity, const nexel_field* field, const float* table,
                      const nexel_loss_weights* lw, void* ws, size_t ws_bytes, int width,
                      int height, float* values, float* d_opacity, float* d_table,
                      nexel_stream_t stream) {
  if (N < 0 || (N > 0 && !opacity) || !lw_ok(lw) || !ws || !values) return NEXEL_ERR_INVALID_ARG;
  if (field && (field->L <= 0 || field->L > NEXEL_MAX_LEVELS || field->T <= 0 || field->F <= 0 ||
                !table))
    return NEXEL_ERR_INVALID_ARG;
  if (width <= 0 || height <= 0 || width > 16384 || height > 16384) return NEXEL_ERR_INVALID_ARG;
  const LossLayout L = loss_layout(width, height);
  if (ws_bytes < L.total) return NEXEL_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  float* part = (float*)((char*)ws + L.partial);
  InvS3 inv_s3 = {};
  const int nl = field ? field->L : 0;
  for (int l = 0; l < nl; ++l) {
    const double s = field->level_scale[l];
    if (!(s > 0.0)) return NEXEL_ERR_INVALID_ARG;
    inv_s3.v[l] = (float)(1.0 / (s * s * s));
  }
  const long long level_size = field ? (long long)field->T * field->F : 1;
  const long long n_table = field ? level_size * field->L : 0;
  {
    NEXEL_PROF("loss_params", st);
    k_loss_params<<<kParamBlocks, kLossThreads, 0, st>>>(N, opacity, n_table, level_size,
                                                        std::max(nl, 1), inv_s3, table,
                                                        lw->opacity, lw->grid, d_opacity,
                                                        d_table, part);
  }
  {
    NEXEL_PROF("loss_values", st);
    k_values_params<<<1, 1024, 0, st>>>(kParamBlocks, N, lw->opacity, lw->grid, part, values);
  }
  return cudaGetLastError() == cudaSuccess ? NEXEL_OK : NEXEL_ERR_CUDA;
}

int nexel_adam_step(int n_tensors, float* const* params, const float* const* grads,
                    float* const* m, float* const* v, const long long* sizes, const float* lrs,
                    float beta1, float beta2, float eps, int step, nexel_stream_t stream) {
  if (n_tensors < 0 || (n_tensors > 0 && (!params || !grads || !m || !v || !sizes || !lrs)) ||
      step < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
    return NEXEL_ERR_INVALID_ARG;
  for (int i = 0; i < n_tensors; ++i)
    if (sizes[i] < 0 || (sizes[i] > 0 && (!params[i] || !grads[i] || !m[i] || !v[i])) ||
        !std::isfinite(lrs[i]))
      return NEXEL_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const float c1 = (float)(1.0 / (1.0 - std::pow((double)beta1, step)));
  const float c2 = (float)(1.0 / (1.0 - std::pow((double)beta2, step)));
  for (int b = 0; b < n_tensors; b += kAdamMax) {
    AdamArgs a = {};
    const int n = std::min(kAdamMax, n_tensors - b);
    long long mx = 0;
    for (int i = 0; i < n; ++i) {
      a.p[i] = params[b + i];
      a.g[i] = grads[b + i];
      a.m[i] = m[b + i];
      a.v[i] = v[b + i];
      a.n[i] = sizes[b + i];
      a.lr[i] = lrs[b + i];
      mx = std::max(mx, sizes[b + i]);
    }
    if (mx == 0) continue;
    const unsigned gx = (unsigned)std::min<long long>((mx + 255) / 256, 2048);
    NEXEL_PROF("adam", st);
    k_adam<<<dim3(gx, (unsigned)n), 256, 0, st>>>(a, beta1, beta2, eps, c1, c2);
  }
  return cudaGetLastError() == cudaSuccess ? NEXEL_OK : NEXEL_ERR_CUDA;
}

}  // extern "C"
