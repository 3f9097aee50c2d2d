// Adaptive density control (supp. Sec. 7.2 and Sec. 5, "Adaptive Density
// Control"): farthest point sampling initialisation, the blended-error pass,
// the error-weighted selection of the surfels to split, the split along the
// long axis, and the opacity prune.
#include "common.cuh"

#include <cmath>

namespace nexel {
namespace {

constexpr int kFpsThreads = 1024;

// Farthest point sampling in one CTA: per iteration every thread lowers the
// minimum squared distance of its points to the newest sample, then the
// block takes the farthest point (lowest index on ties).  Squared distances
// are formed with explicitly rounded FP32 operations, so the decisions are
// reproducible.
__global__ void __launch_bounds__(kFpsThreads) k_fps(int n, int m, const float* __restrict__ x,
                                                     float* __restrict__ mind,
                                                     int* __restrict__ idx,
                                                     float* __restrict__ d2sel,
                                                     float* __restrict__ scale) {
  __shared__ float s_v[32];
  __shared__ int s_k[32];
  __shared__ int s_cur;
  for (int k = threadIdx.x; k < n; k += kFpsThreads) mind[k] = INFINITY;
  if (threadIdx.x == 0) s_cur = 0;
  __syncthreads();
  for (int it = 0; it < m; ++it) {
    const int cur = s_cur;
    if (threadIdx.x == 0) {
      idx[it] = cur;
      d2sel[it] = it == 0 ? INFINITY : mind[cur];
    }
    __syncthreads();  // mind[cur] read before it is overwritten
    const float cx = x[3 * cur], cy = x[3 * cur + 1], cz = x[3 * cur + 2];
    float best = -INFINITY;
    int bk = 0x7fffffff;
    for (int k = threadIdx.x; k < n; k += kFpsThreads) {
      const float dx = __fsub_rn(x[3 * k], cx), dy = __fsub_rn(x[3 * k + 1], cy),
                  dz = __fsub_rn(x[3 * k + 2], cz);
      const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
      float v = fminf(mind[k], d2);
      if (k == cur) v = -1.f;  // selected
      else if (mind[k] < 0.f) v = -1.f;
      mind[k] = v;
      if (v > best || (v == best && k < bk)) { best = v; bk = k; }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, best, d);
      const int ok = __shfl_xor_sync(0xffffffffu, bk, d);
      if (ov > best || (ov == best && ok < bk)) { best = ov; bk = ok; }
    }
    if ((threadIdx.x & 31) == 0) { s_v[threadIdx.x >> 5] = best; s_k[threadIdx.x >> 5] = bk; }
    __syncthreads();
    if (threadIdx.x < 32) {
      best = s_v[threadIdx.x];
      bk = s_k[threadIdx.x];
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, d);
        const int ok = __shfl_xor_sync(0xffffffffu, bk, d);
        if (ov > best || (ov == best && ok < bk)) { best = ov; bk = ok; }
      }
      if (threadIdx.x == 0) s_cur = bk < n ? bk : 0;
    }
    __syncthreads();
  }
  // initial scales (supp. Sec. 7.2): the distance at which each point was
  // selected, the nearest neighbour among the points sampled before it; the
  // first point has no predecessor and takes the second's
  if (scale) {
    __syncthreads();
    for (int i = threadIdx.x; i < m; i += kFpsThreads) {
      const int src = (i == 0) ? 1 : i;
      scale[i] = src < m ? __fsqrt_rn(d2sel[src]) : 0.f;
    }
  }
}

// Selection keys E_i / err_i (FP32, correctly rounded), +inf for a zero
// error; non-negative floats sort as their bit patterns.
__global__ void k_select_keys(int n, const float* __restrict__ err, const float* __restrict__ expo,
                              uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float e = err[i];
  const float k = e > 0.f ? __fdiv_rn(expo[i], e) : INFINITY;
  key[i] = __float_as_uint(fmaxf(k, 0.f));
  val[i] = (uint32_t)i;
}

__global__ void k_copy_sel(int n_sel, const uint32_t* __restrict__ v, int* __restrict__ sel) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n_sel) sel[r] = (int)v[r];
}

// Split of the selected surfels: slot i takes the first child, slot N + r
// the second; the long axis is v1 if sigma1 >= sigma2, else v2.
__global__ void k_split(int N, int n_sel, int color_dim, const int* __restrict__ sel,
                        float* __restrict__ mu, float* __restrict__ quat, float* __restrict__ scale,
                        float* __restrict__ opacity, float* __restrict__ gamma,
                        float* __restrict__ color) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_sel) return;
  const int i = sel[r], o = N + r;
  float qw = quat[4 * i], qx = quat[4 * i + 1], qy = quat[4 * i + 2], qz = quat[4 * i + 3];
  const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  qw *= qn; qx *= qn; qy *= qn; qz *= qn;
  float3 v1, v2, nn;
  quat_cols(qw, qx, qy, qz, v1, v2, nn);
  const float s1 = scale[2 * i], s2 = scale[2 * i + 1];
  const int a = s1 >= s2 ? 0 : 1;
  const float sl = a == 0 ? s1 : s2;
  const float3 v = a == 0 ? v1 : v2;
  const float h = 0.5f * sl;
  const float m0 = mu[3 * i], m1 = mu[3 * i + 1], m2 = mu[3 * i + 2];
  for (int k = 0; k < 4; ++k) quat[4 * o + k] = quat[4 * i + k];
  scale[2 * o] = scale[2 * i];
  scale[2 * o + 1] = scale[2 * i + 1];
  scale[2 * o + a] = h;
  scale[2 * i + a] = h;
  opacity[o] = opacity[i];
  gamma[2 * o] = gamma[2 * i];
  gamma[2 * o + 1] = gamma[2 * i + 1];
  for (int k = 0; k < color_dim; ++k) color[(size_t)color_dim * o + k] = color[(size_t)color_dim * i + k];
  mu[3 * o] = m0 + h * v.x; mu[3 * o + 1] = m1 + h * v.y; mu[3 * o + 2] = m2 + h * v.z;
  mu[3 * i] = m0 - h * v.x; mu[3 * i + 1] = m1 - h * v.y; mu[3 * i + 2] = m2 - h * v.z;
}

__global__ void k_keep(int n, float thr, const float* __restrict__ opacity,
                       uint32_t* __restrict__ flag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = opacity[i] >= thr ? 1u : 0u;
}

__global__ void k_compact(int n, int color_dim, float thr, const uint32_t* __restrict__ pos,
                          const float* __restrict__ mu, const float* __restrict__ quat,
                          const float* __restrict__ scale, const float* __restrict__ opacity,
                          const float* __restrict__ gamma, const float* __restrict__ color,
                          float* __restrict__ mu_o, float* __restrict__ quat_o,
                          float* __restrict__ scale_o, float* __restrict__ opacity_o,
                          float* __restrict__ gamma_o, float* __restrict__ color_o) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !(opacity[i] >= thr)) return;
  const uint32_t o = pos[i];
  for (int k = 0; k < 3; ++k) mu_o[3 * (size_t)o + k] = mu[3 * (size_t)i + k];
  for (int k = 0; k < 4; ++k) quat_o[4 * (size_t)o + k] = quat[4 * (size_t)i + k];
  for (int k = 0; k < 2; ++k) scale_o[2 * (size_t)o + k] = scale[2 * (size_t)i + k];
  opacity_o[o] = opacity[i];
  for (int k = 0; k < 2; ++k) gamma_o[2 * (size_t)o + k] = gamma[2 * (size_t)i + k];
  for (int k = 0; k < color_dim; ++k)
    color_o[(size_t)color_dim * o + k] = color[(size_t)color_dim * i + k];
}

// scratch of the selection and the prune: keys and values x 2, sort
// histograms and scan sums
struct DensityLayout {
  size_t k0, k1, v0, v1, hist, sums, total;
};
DensityLayout density_layout(long long n) {
  DensityLayout L;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t c = (size_t)std::max(n, 1LL);
  const size_t nb = (c + 1023) / 1024;
  size_t o = 0;
  L.k0 = o; o += al(c * 4);
  L.k1 = o; o += al(c * 4);
  L.v0 = o; o += al(c * 4);
  L.v1 = o; o += al(c * 4);
  L.hist = o; o += al(256 * nb * 4);
  L.sums = o; o += al(((256 * nb + kScanTile - 1) / kScanTile + 2) * 4 + ((c + kScanTile - 1) / kScanTile + 2) * 4);
  L.total = o;
  return L;
}

}  // namespace
}  // namespace nexel

using namespace nexel;

extern "C" {

int nexel_fps(int n, const float* points, int m, float* scratch, int* idx, float* d2sel,
              float* scale, nexel_stream_t stream) {
  if (n < 0 || m < 0 || m > n || (n > 0 && (!points || !scratch)) ||
      (m > 0 && (!idx || !d2sel)))
    return NEXEL_ERR_INVALID_ARG;
  if (m == 0) return NEXEL_OK;
  cudaStream_t st = (cudaStream_t)stream;
  NEXEL_PROF("fps", st);
  k_fps<<<1, kFpsThreads, 0, st>>>(n, m, points, scratch, idx, d2sel, scale);
  return cudaGetLastError() == cudaSuccess ? NEXEL_OK : NEXEL_ERR_CUDA;
}

int nexel_blend_error(const nexel_camera* cam, const nexel_settings* settings, int N, void* ws,
                      size_t ws_bytes, const float* image, const float* target, float* err,
                      nexel_stream_t stream) {
  if (!cam || !settings || N < 0 || !ws || !image || !target || (N > 0 && !err))
    return NEXEL_ERR_INVALID_ARG;
  if (cam->width <= 0 || cam->height <= 0) return NEXEL_ERR_INVALID_ARG;
  WsLayout L = ws_layout_for_bytes(*cam, settings->K, N, ws_bytes);
  if (L.cap < 0) return NEXEL_ERR_INVALID_ARG;
  cudaError_t e = launch_blend_error(make_devcam(*cam), *settings, (char*)ws, L, image, target, err,
                                     (cudaStream_t)stream);
  return e == cudaSuccess ? NEXEL_OK : NEXEL_ERR_CUDA;
}

int nexel_density_workspace_size(int N, size_t* bytes) {
  if (N < 0 || !bytes) return NEXEL_ERR_INVALID_ARG;
  *bytes = density_layout(N).total;
  return NEXEL_OK;
}

int nexel_densify_count(int N, long long budget, int* n_select) {
  if (N < 0 || !n_select) return NEXEL_ERR_INVALID_ARG;
  // 5 % of the current primitives, rounded up; no more than the budget
  // leaves room for (the paper caps the primitive count at P)
  const long long want = ((long long)N * 5 + 99) / 100;
  const long long room = budget - (long long)N;
  *n_select = (int)std::max(0LL, std::min(want, room));
  return NEXEL_OK;
}

int nexel_densify_select(int N, const float* err, const float* expo, long long budget, void* ws,
                         size_t ws_bytes, int* sel, int* n_select_out, nexel_stream_t stream) {
  int n_select = 0;
  if (nexel_densify_count(N, budget, &n_select) != NEXEL_OK || !n_select_out)
    return NEXEL_ERR_INVALID_ARG;
  if ((N > 0 && (!err || !expo)) || !ws || (n_select > 0 && !sel))
    return NEXEL_ERR_INVALID_ARG;
  *n_select_out = n_select;
  const DensityLayout L = density_layout(N);
  if (ws_bytes < L.total) return NEXEL_ERR_INVALID_ARG;
  if (n_select == 0) return NEXEL_OK;
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)ws;
  uint32_t *k0 = (uint32_t*)(w + L.k0), *k1 = (uint32_t*)(w + L.k1);
  uint32_t *v0 = (uint32_t*)(w + L.v0), *v1 = (uint32_t*)(w + L.v1);
  {
    NEXEL_PROF("select_keys", st);
    k_select_keys<<<(N + 255) / 256, 256, 0, st>>>(N, err, expo, k0, v0);
  }
  int which = 0;
  cudaError_t e = sort_pairs_u32(k0, k1, v0, v1, N, (uint32_t*)(w + L.hist),
                                 (uint32_t*)(w + L.sums), st, &which);
  if (e != cudaSuccess) return NEXEL_ERR_CUDA;
  {
    NEXEL_PROF("select_copy", st);
    k_copy_sel<<<(n_select + 255) / 256, 256, 0, st>>>(n_select, which ? v1 : v0, sel);
  }
  return cudaGetLastError() == cudaSuccess ? NEXEL_OK : NEXEL_ERR_CUDA;
}

int nexel_densify_split(int N, int n_select, const int* sel, int color_dim, float* mu, float* quat,
                        float* scale, float* opacity, float* gamma, float* color,
                        nexel_stream_t stream) {
  if (N < 0 || n_select < 0 || n_select > N || (color_dim != 3 && color_dim != 48) ||
      (n_select > 0 && (!sel || !mu || !quat || !scale || !opacity || !gamma || !color)))
    return NEXEL_ERR_INVALID_ARG;
  if (n_select == 0) return NEXEL_OK;
  cudaStream_t st = (cudaStream_t)stream;
  NEXEL_PROF("split", st);
  k_split<<<(n_select + 127) / 128, 128, 0, st>>>(N, n_select, color_dim, sel, mu, quat, scale,
                                                  opacity, gamma, color);
  return cudaGetLastError() == cudaSuccess ? NEXEL_OK : NEXEL_ERR_CUDA;
}

int nexel_prune(int N, float threshold, int color_dim, const float* mu, const float* quat,
                const float* scale, const float* opacity, const float* gamma, const float* color,
                void* ws, size_t ws_bytes, float* mu_out, float* quat_out, float* scale_out,
                float* opacity_out, float* gamma_out, float* color_out, int* n_out,
                nexel_stream_t stream) {
  if (N < 0 || (color_dim != 3 && color_dim != 48) || !ws || !n_out || !std::isfinite(threshold))
    return NEXEL_ERR_INVALID_ARG;
  if (N > 0 && (!mu || !quat || !scale || !opacity || !gamma || !color || !mu_out ||
                !quat_out || !scale_out || !opacity_out || !gamma_out || !color_out))
    return NEXEL_ERR_INVALID_ARG;
  const DensityLayout L = density_layout(N);
  if (ws_bytes < L.total) return NEXEL_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  char* w = (char*)ws;
  if (N == 0) return cudaMemsetAsync(n_out, 0, 4, st) == cudaSuccess ? NEXEL_OK : NEXEL_ERR_CUDA;
  uint32_t* pos = (uint32_t*)(w + L.k0);
  {
    NEXEL_PROF("prune_keep", st);
    k_keep<<<(N + 255) / 256, 256, 0, st>>>(N, threshold, opacity, pos);
  }
  cudaError_t e = exclusive_scan_u32(pos, N, (uint32_t*)(w + L.sums), (uint32_t*)n_out, st);
  if (e != cudaSuccess) return NEXEL_ERR_CUDA;
  {
    NEXEL_PROF("prune_compact", st);
    k_compact<<<(N + 255) / 256, 256, 0, st>>>(N, color_dim, threshold, pos, mu, quat, scale,
                                               opacity, gamma, color, mu_out, quat_out, scale_out,
                                               opacity_out, gamma_out, color_out);
  }
  return cudaGetLastError() == cudaSuccess ? NEXEL_OK : NEXEL_ERR_CUDA;
}

}  // extern "C"
