// Collection pass (Sec. 4.2) forward and backward.
//
// One CTA per 16x16 tile, one thread per pixel.  The tile's surfel list (in
// centre-depth order) is streamed through shared memory in batches of 256
// packed records; every thread walks the batch front to back, evaluates the
// ray-surfel intersection and the generalised-Gaussian opacity, composites
// (Eq. 1) and keeps a register-resident top-K buffer of (weight, rank, depth)
// sorted by descending weight.  A surfel that is not (or no longer) among
// the K goes into the non-textured render N (Eq. 5).
//
// The backward replays each pixel's list back to front from its last
// composited surfel, restoring T_i = T_{i+1} / (1 - alpha_i), and carries the
// weighted colour of everything behind (R) so that
// dL/dalpha_i = T_i (e_i - R_i), where e_i is the colour-side gradient of
// surfel i: c_i . dL/dC if it is not textured, dL/dW_j if it fills slot j.
// Per-surfel gradients are pre-reduced across the warp with a transposing
// shuffle butterfly and added to the rank-ordered gradient records with one
// atomic per value, issued by 20 lanes at once.
#include "common.cuh"

namespace nexel {

template <typename KeyT>
__device__ __forceinline__ uint32_t rank_of(KeyT k, uint32_t mask) {
  return (uint32_t)k & mask;
}

// The tile's surfel list: instance i's depth rank, from a 32-bit (tile,
// rank) key or a 64-bit key whose low 32 bits are the rank.
__device__ __forceinline__ uint32_t key_rank(const KeySrc& k, uint32_t i) {
  return k.key64 ? (uint32_t)reinterpret_cast<const unsigned long long*>(k.keys)[i]
                 : reinterpret_cast<const uint32_t*>(k.keys)[i] & k.rmask;
}

// The work item a CTA takes next: with a queue, persistent CTAs pull items
// (the tiles of every view of a batch, view after view) from a device
// counter; without one, CTA b takes item b once.  Returns -1 when none is
// left.  Every thread of the CTA calls it.
__device__ __forceinline__ int next_item(unsigned* queue, int it, int total, int* s_item) {
  if (!queue) return (it == 0 && (int)blockIdx.x < total) ? (int)blockIdx.x : -1;
  __syncthreads();  // the previous item's shared-memory use is over
  if (threadIdx.x == 0) *s_item = (int)atomicAdd(queue, 1u);
  __syncthreads();
  const int item = *s_item;
  return item < total ? item : -1;
}

// One 16 x 16 tile of the collection forward.  BATCH: surfel records staged
// per batch (128, 256 or 512; a launch-shape knob of the autotuner: smaller
// batches test for early termination more often, larger ones synchronise
// less).
template <int K, int BATCH>
__device__ __forceinline__ void collect_fwd_tile(const CollectFwdView& V, int tile,
                                                 float alpha_min, float alpha_max, float T_min,
                                                 float4 (*s_rec)[BATCH], uint32_t* s_rank) {
  const DevCam& c = V.c;
  const float4* __restrict__ recs = V.recs;
  const int tx = tile % c.tiles_x, ty = tile / c.tiles_x;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py = ty * kTile + (threadIdx.x / kTile);
  const bool inside = px < c.W && py < c.H;
  const float fpx = px + 0.5f, fpy = py + 0.5f;
  const uint2 rg = V.ranges[tile];
  float T = 1.f, n0 = 0.f, n1 = 0.f, n2 = 0.f;
  float Wk[K > 0 ? K : 1], Dk[K > 0 ? K : 1];
  int Rk[K > 0 ? K : 1];
#pragma unroll
  for (int k = 0; k < K; ++k) { Wk[k] = 0.f; Dk[k] = 0.f; Rk[k] = -1; }
  int last = 0;
  bool done = !inside;
  for (uint32_t b0 = rg.x; b0 < rg.y; b0 += BATCH) {
    if (__syncthreads_count(done) == kTilePix) break;
#pragma unroll
    for (int t = threadIdx.x; t < BATCH; t += kTilePix) {
      const uint32_t i = b0 + t;
      if (i < rg.y) {
        const uint32_t r = key_rank(V.keys, i);
        s_rank[t] = r;
        const float4* src = recs + (size_t)r * kRecF4;
#pragma unroll
        for (int k = 0; k < kRecF4; ++k) s_rec[k][t] = __ldg(src + k);
      }
    }
    __syncthreads();
    const int nb = (int)min((uint32_t)BATCH, rg.y - b0);
    if (!done) {
      for (int j = 0; j < nb; ++j) {
        const float4 q0 = s_rec[0][j], q1 = s_rec[1][j], q2 = s_rec[2][j], q3 = s_rec[3][j];
        Hit h;
        if (!eval_surfel(q0, q1, q2, q3, fpx, fpy, c.near_, alpha_min, h)) continue;
        const float a = fminf(h.alpha, alpha_max);
        const float test = T * (1.f - a);
        if (test < T_min) { done = true; break; }
        const float w = a * T;
        if constexpr (K > 0) {
          if (w > Wk[K - 1]) {
            if (Rk[K - 1] >= 0) {  // evicted: back into N
              float4 ce = __ldg(recs + (size_t)Rk[K - 1] * kRecF4 + 4);
              n0 = fmaf(Wk[K - 1], ce.x, n0); n1 = fmaf(Wk[K - 1], ce.y, n1); n2 = fmaf(Wk[K - 1], ce.z, n2);
            }
            Wk[K - 1] = w; Rk[K - 1] = (int)s_rank[j]; Dk[K - 1] = h.t;
#pragma unroll
            for (int k = K - 1; k > 0; --k) {
              if (Wk[k] > Wk[k - 1]) {
                float tw = Wk[k]; Wk[k] = Wk[k - 1]; Wk[k - 1] = tw;
                float td = Dk[k]; Dk[k] = Dk[k - 1]; Dk[k - 1] = td;
                int tr = Rk[k]; Rk[k] = Rk[k - 1]; Rk[k - 1] = tr;
              }
            }
          } else {
            const float4 q4 = s_rec[4][j];
            n0 = fmaf(w, q4.x, n0); n1 = fmaf(w, q4.y, n1); n2 = fmaf(w, q4.z, n2);
          }
        } else {
          const float4 q4 = s_rec[4][j];
          n0 = fmaf(w, q4.x, n0); n1 = fmaf(w, q4.y, n1); n2 = fmaf(w, q4.z, n2);
        }
        T = test;
        last = (int)(b0 - rg.x) + j + 1;
      }
    }
  }
  if (!inside) return;
  const size_t p = (size_t)py * c.W + px;
  V.notex[3 * p] = n0; V.notex[3 * p + 1] = n1; V.notex[3 * p + 2] = n2;
  V.T_final[p] = T;
  V.n_contrib[p] = last;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    int id = -1;
    if (Rk[k] >= 0) id = (int)__float_as_uint(__ldg(recs + (size_t)Rk[k] * kRecF4 + 4).w);
    V.weights[p * K + k] = Wk[k];
    V.ids[p * K + k] = id;
    V.depths[p * K + k] = Dk[k];
  }
}

// Collection forward over the tiles of one view (one CTA per tile) or, with
// a queue, of every view of a batch in one launch of persistent CTAs.
template <int K, int BATCH, bool MV>
__global__ void __launch_bounds__(kTilePix, 5) k_collect_fwd(
    const __grid_constant__ ViewBatch<CollectFwdView> b, float alpha_min, float alpha_max,
    float T_min, unsigned* queue) {
  __shared__ float4 s_rec[kRecF4][BATCH];
  __shared__ uint32_t s_rank[BATCH];
  __shared__ int s_item;
  const int total = b.item0[b.n];
  for (int it = 0;; ++it) {
    const int item = next_item(queue, it, total, &s_item);
    if (item < 0) break;
    // MV: a batch of views (else one view, at a fixed index)
    const int v = MV ? view_of(b, item) : 0;
    collect_fwd_tile<K, BATCH>(b.v[v], MV ? item - b.item0[v] : item, alpha_min, alpha_max,
                               T_min, s_rec, s_rank);
  }
}

// Warp sum of the 16 per-lane gradient values, added to dst[0..15] with one
// atomic per nonzero total.  A transposing butterfly: at each xor step a lane
// keeps one half of its partial sums and sends the other half to its
// partner (16 -> 8 -> 4 -> 2 -> 1 values, then the last pair: 16 shuffles
// instead of 5 x 16), so that in the end each total sits in two lanes, at
// index 8 b4 + 4 b3 + 2 b2 + b1 (b = lane bits); the even lanes issue the
// atomics in the same instruction.
__device__ __forceinline__ void warp_sum16_add(const float (&g)[kGradStride], float* dst) {
  static_assert(kGradStride == 16, "the butterfly below is laid out for 16 values");
  const int lane = threadIdx.x & 31;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float u[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float keep = b4 ? g[8 + i] : g[i], send = b4 ? g[i] : g[8 + i];
    u[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float keep = b3 ? u[4 + i] : u[i], send = b3 ? u[i] : u[4 + i];
    w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float x[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float keep = b2 ? w[2 + i] : w[i], send = b2 ? w[i] : w[2 + i];
    x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  const float keep = b1 ? x[1] : x[0], send = b1 ? x[0] : x[1];
  const float y = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  const float z = y + __shfl_xor_sync(0xffffffffu, y, 1);
  if (!(lane & 1) && z != 0.f) atomicAdd(dst + 8 * (int)b4 + 4 * (int)b3 + 2 * (int)b2 + (int)b1, z);
}

// One 16 x 16 tile of the collection backward (BATCH as in the forward).
template <int K, int BATCH>
__device__ __forceinline__ void collect_bwd_tile(const CollectBwdView& V, int tile,
                                                 float alpha_min, float alpha_max, float bg0,
                                                 float bg1, float bg2, float4 (*s_rec)[BATCH],
                                                 float4 (*s_aux)[BATCH], uint32_t* s_rank,
                                                 int* s_max) {
  const DevCam& c = V.c;
  const float4* __restrict__ recs = V.recs;
  const float4* __restrict__ aux = V.aux;
  const int tx = tile % c.tiles_x, ty = tile / c.tiles_x;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py = ty * kTile + (threadIdx.x / kTile);
  const bool inside = px < c.W && py < c.H;
  const float fpx = px + 0.5f, fpy = py + 0.5f;
  // camera-space ray direction of this pixel (z component 1)
  const float rdx = (fpx - c.cx) / c.fx, rdy = (fpy - c.cy) / c.fy;
  const uint2 rg = V.ranges[tile];
  const size_t p = inside ? (size_t)py * c.W + px : 0;
  float T = 1.f, dC0 = 0.f, dC1 = 0.f, dC2 = 0.f;
  int last = 0;
  int Ik[K > 0 ? K : 1];
  float dWe[K > 0 ? K : 1], dDk[K > 0 ? K : 1];
#pragma unroll
  for (int k = 0; k < K; ++k) { Ik[k] = -1; dWe[k] = 0.f; dDk[k] = 0.f; }
  if (inside) {
    T = V.T_final[p];
    last = V.n_contrib[p];
    dC0 = V.d_image[3 * p]; dC1 = V.d_image[3 * p + 1]; dC2 = V.d_image[3 * p + 2];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      Ik[k] = V.ids[p * K + k];
      dWe[k] = V.dweff[p * K + k];
      dDk[k] = V.ddepth[p * K + k];
    }
  }
  float R = bg0 * dC0 + bg1 * dC1 + bg2 * dC2;  // background behind everything
  if (threadIdx.x == 0) *s_max = 0;
  __syncthreads();
  atomicMax(s_max, last);
  __syncthreads();
  const uint32_t list_end = rg.x + (uint32_t)*s_max;
  for (uint32_t bend = list_end; bend > rg.x;) {
    const uint32_t bstart = (bend - rg.x > (uint32_t)BATCH) ? bend - BATCH : rg.x;
    __syncthreads();
#pragma unroll
    for (int t = threadIdx.x; t < BATCH; t += kTilePix) {
      const uint32_t i = bstart + t;
      if (i < bend) {
        const uint32_t r = key_rank(V.keys, i);
        s_rank[t] = r;
        const float4* src = recs + (size_t)r * kRecF4;
#pragma unroll
        for (int k = 0; k < kRecF4; ++k) s_rec[k][t] = __ldg(src + k);
        const float4* asrc = aux + (size_t)r * kAuxF4;
#pragma unroll
        for (int k = 0; k < kAuxF4; ++k) s_aux[k][t] = __ldg(asrc + k);
      }
    }
    __syncthreads();
    for (int j = (int)(bend - bstart) - 1; j >= 0; --j) {
      const int pos = (int)(bstart - rg.x) + j;
      const float4 q0 = s_rec[0][j], q1 = s_rec[1][j], q2 = s_rec[2][j], q3 = s_rec[3][j];
      Hit h;
      bool ok = pos < last && eval_surfel(q0, q1, q2, q3, fpx, fpy, c.near_, alpha_min, h);
      if (!__any_sync(0xffffffffu, ok)) continue;
      // per-surfel gradient record (sums over the surfel's pixels), from
      // which the preprocess backward forms the camera-space gradients with
      // the surfel's own frame v1, v2, n and scales s1, s2 (the hit offset
      // in the plane is r = u s1 v1 + v s2 v2):
      //   0 du1, 1 dv2, 2 gd          (mu_c = -v1 S0 - v2 S1 + n S2)
      //   3 du1 u s1, 4 du1 v s2      (v1_c = v1 S3 + v2 S4; sigma1 = -S3 / s1)
      //   5 dv2 u s1, 6 dv2 v s2      (v2_c = v1 S5 + v2 S6; sigma2 = -S6 / s2)
      //   7 gd u s1, 8 gd v s2        (n_c = -v1 S7 - v2 S8)
      //   9 opacity, 10-11 gamma, 12-14 colour, 15 unused
      float g[kGradStride];
#pragma unroll
      for (int k = 0; k < kGradStride; ++k) g[k] = 0.f;
      if (ok) {
        const float4 q4 = s_rec[4][j];
        const float a = fminf(h.alpha, alpha_max);
        const bool clamped = h.alpha > alpha_max;
        T = T / (1.f - a);
        const int id = (int)__float_as_uint(q4.w);
        int slot = -1;
#pragma unroll
        for (int k = 0; k < K; ++k)
          if (Ik[k] == id) slot = k;
        float e, dt = 0.f;
        if (slot >= 0) {
          float ew = 0.f, ed = 0.f;
#pragma unroll
          for (int k = 0; k < K; ++k)
            if (k == slot) { ew = dWe[k]; ed = dDk[k]; }
          e = ew;
          dt = ed;
        } else {
          e = q4.x * dC0 + q4.y * dC1 + q4.z * dC2;
          const float w = a * T;
          g[12] = w * dC0; g[13] = w * dC1; g[14] = w * dC2;
        }
        const float da = T * (e - R);
        R = a * e + (1.f - a) * R;
        float du = 0.f, dv = 0.f;
        if (!clamped) {
          const float al = h.alpha;
          g[9] = da * h.e;             // d alpha / d opacity = e
          const float cpa = -da * al;  // dL/d(pu) * 2 = -dalpha * alpha
          // d pu / d u = 2 g pu / u, d pu / d g = 2 pu ln|u| (|u| > 0: the
          // quotient and the logarithm in fast form, a few ulp, well inside
          // the gradients' tolerance)
          constexpr float kLn2 = 0.6931471805599453f;
          if (h.u != 0.f) {
            du = cpa * q1.z * __fdividef(h.pu, h.u);
            g[10] = cpa * h.pu * (kLn2 * __log2f(fabsf(h.u)));
          }
          if (h.v != 0.f) {
            dv = cpa * q1.w * __fdividef(h.pv, h.v);
            g[11] = cpa * h.pv * (kLn2 * __log2f(fabsf(h.v)));
          }
        }
        // camera-space chain (the hit x = t d lies on the plane, so
        // x - mu = u s1 v1 + v s2 v2 exactly): u = (x - mu) . v1 / s1 with
        // t = (mu . n) / (d . n); the per-surfel vectors v1, v2, n multiply
        // the sums in the preprocess backward
        const float4 a0 = s_aux[0][j], a1 = s_aux[1][j], a2 = s_aux[2][j], a3 = s_aux[3][j];
        const float us = h.u * a0.w, vs = h.v * a1.w;   // u s1, v s2
        const float du1 = du * a2.w, dv2 = dv * a3.w;  // du / s1, dv / s2
        // dL/dt through u and v: (du1 v1 + dv2 v2) . d, d = (rdx, rdy, 1)
        const float v1d = fmaf(a1.x, rdx, fmaf(a1.y, rdy, a1.z));
        const float v2d = fmaf(a2.x, rdx, fmaf(a2.y, rdy, a2.z));
        const float gd = fmaf(du1, v1d, fmaf(dv2, v2d, dt)) * h.inv;
        g[0] = du1; g[1] = dv2; g[2] = gd;
        g[3] = du1 * us; g[4] = du1 * vs;
        g[5] = dv2 * us; g[6] = dv2 * vs;
        g[7] = gd * us; g[8] = gd * vs;
      }
      warp_sum16_add(g, V.grad + (size_t)s_rank[j] * kGradStride);
    }
    bend = bstart;
  }
}

// Four CTAs per SM (64 registers, no spills): the replay is issue-bound and
// gains from the fourth tile in flight.  One view (a CTA per tile) or, with
// a queue, every view of a batch in one launch of persistent CTAs.
template <int K, int BATCH, bool MV>
__global__ void __launch_bounds__(kTilePix, 4) k_collect_bwd(
    const __grid_constant__ ViewBatch<CollectBwdView> b, float alpha_min, float alpha_max,
    float bg0, float bg1, float bg2, unsigned* queue) {
  __shared__ float4 s_rec[kRecF4][BATCH];
  __shared__ float4 s_aux[kAuxF4][BATCH];
  __shared__ uint32_t s_rank[BATCH];
  __shared__ int s_max;
  __shared__ int s_item;
  const int total = b.item0[b.n];
  for (int it = 0;; ++it) {
    const int item = next_item(queue, it, total, &s_item);
    if (item < 0) break;
    const int v = MV ? view_of(b, item) : 0;
    collect_bwd_tile<K, BATCH>(b.v[v], MV ? item - b.item0[v] : item, alpha_min, alpha_max, bg0,
                               bg1, bg2, s_rec, s_aux, s_rank, &s_max);
  }
}

CollectFwdView collect_fwd_view(const DevCam& c, char* ws, const WsLayout& L, float* notex,
                                float* weights, int* ids, float* depths, float* T_final) {
  CollectFwdView v;
  v.c = c;
  v.ranges = (const uint2*)(ws + L.ranges);
  v.keys.keys = ws + L.inst0;
  v.keys.key64 = L.key64 ? 1 : 0;
  v.keys.rmask = L.key64 ? 0xFFFFFFFFu : ((1u << L.rank_bits) - 1u);
  v.recs = (const float4*)(ws + L.geom_sorted);
  v.notex = notex;
  v.weights = weights;
  v.ids = ids;
  v.depths = depths;
  v.T_final = T_final;
  v.n_contrib = (int*)(ws + L.n_contrib);
  return v;
}

CollectBwdView collect_bwd_view(const DevCam& c, char* ws, const WsLayout& L, const char* bws,
                                const BwdLayout& B, const int* ids, const float* T_final,
                                const float* d_image) {
  CollectBwdView v;
  v.c = c;
  v.ranges = (const uint2*)(ws + L.ranges);
  v.keys.keys = ws + L.inst0;
  v.keys.key64 = L.key64 ? 1 : 0;
  v.keys.rmask = L.key64 ? 0xFFFFFFFFu : ((1u << L.rank_bits) - 1u);
  v.recs = (const float4*)(ws + L.geom_sorted);
  v.aux = (const float4*)(ws + L.aux_sorted);
  v.ids = ids;
  v.T_final = T_final;
  v.n_contrib = (const int*)(ws + L.n_contrib);
  v.d_image = d_image;
  v.dweff = (const float*)(bws + B.dweff);
  v.ddepth = (const float*)(bws + B.ddepth);
  v.grad = (float*)(ws + L.grad_sorted);
  return v;
}

namespace {

// Grid of a launch: one CTA per item, or (with a queue) as many persistent
// CTAs as fit on the GPU at once.
template <typename Kern>
unsigned batch_grid(Kern kern, int total, bool persistent) {
  if (!persistent) return (unsigned)total;
  int dev = 0, nsm = 152, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTilePix, 0) != cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  return (unsigned)std::min<long long>(total, (long long)per_sm * nsm);
}

}  // namespace

cudaError_t launch_collect_fwd_batch(const nexel_settings& s, const ViewBatch<CollectFwdView>& b,
                                     unsigned* queue, cudaStream_t st) {
  const int total = b.item0[b.n];
  if (total <= 0) return cudaSuccess;
  if (queue) {
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
  }
  const int batch = current_tuning().collect_batch;
  NEXEL_PROF("collect_fwd", st);
#define NEXEL_CF1(KK, BB)                                                                   \
  do {                                                                                      \
    auto kern = queue ? k_collect_fwd<KK, BB, true> : k_collect_fwd<KK, BB, false>;          \
    kern<<<batch_grid(kern, total, queue != nullptr), kTilePix, 0, st>>>(                   \
        b, s.alpha_min, s.alpha_max, s.T_min, queue);                                       \
  } while (0)
#define NEXEL_CF(KK)                                          \
  do {                                                        \
    if (batch == 128) NEXEL_CF1(KK, 128);                     \
    else if (batch == 512) NEXEL_CF1(KK, 512);                \
    else NEXEL_CF1(KK, 256);                                  \
  } while (0)
  switch (s.K) {
    case 0: NEXEL_CF(0); break;
    case 1: NEXEL_CF(1); break;
    case 2: NEXEL_CF(2); break;
    case 3: NEXEL_CF(3); break;
    case 4: NEXEL_CF(4); break;
    case 5: NEXEL_CF(5); break;
    case 6: NEXEL_CF(6); break;
    case 7: NEXEL_CF(7); break;
    case 8: NEXEL_CF(8); break;
    default: return cudaErrorInvalidValue;
  }
#undef NEXEL_CF
#undef NEXEL_CF1
  return cudaGetLastError();
}

cudaError_t launch_collect_fwd(const DevCam& c, const nexel_settings& s, char* ws,
                               const WsLayout& L, float* notex, float* weights, int* ids,
                               float* depths, float* T_final, cudaStream_t st) {
  ViewBatch<CollectFwdView> b;
  b.n = 1;
  b.item0[0] = 0;
  b.item0[1] = L.n_tiles;
  b.v[0] = collect_fwd_view(c, ws, L, notex, weights, ids, depths, T_final);
  return launch_collect_fwd_batch(s, b, nullptr, st);
}

cudaError_t launch_collect_bwd_batch(const nexel_settings& s, const ViewBatch<CollectBwdView>& b,
                                     unsigned* queue, cudaStream_t st) {
  const int total = b.item0[b.n];
  if (total <= 0) return cudaSuccess;
  if (queue) {
    cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
  }
  const int batch = current_tuning().collect_batch;
  NEXEL_PROF("collect_bwd", st);
#define NEXEL_CB1(KK, BB)                                                                   \
  do {                                                                                      \
    auto kern = queue ? k_collect_bwd<KK, BB, true> : k_collect_bwd<KK, BB, false>;          \
    kern<<<batch_grid(kern, total, queue != nullptr), kTilePix, 0, st>>>(                   \
        b, s.alpha_min, s.alpha_max, s.bg[0], s.bg[1], s.bg[2], queue);                     \
  } while (0)
#define NEXEL_CB(KK)                                          \
  do {                                                        \
    if (batch == 128) NEXEL_CB1(KK, 128);                     \
    else if (batch == 512) NEXEL_CB1(KK, 512);                \
    else NEXEL_CB1(KK, 256);                                  \
  } while (0)
  switch (s.K) {
    case 0: NEXEL_CB(0); break;
    case 1: NEXEL_CB(1); break;
    case 2: NEXEL_CB(2); break;
    case 3: NEXEL_CB(3); break;
    case 4: NEXEL_CB(4); break;
    case 5: NEXEL_CB(5); break;
    case 6: NEXEL_CB(6); break;
    case 7: NEXEL_CB(7); break;
    case 8: NEXEL_CB(8); break;
    default: return cudaErrorInvalidValue;
  }
#undef NEXEL_CB
#undef NEXEL_CB1
  return cudaGetLastError();
}

cudaError_t launch_collect_bwd(const DevCam& c, const nexel_settings& s, char* ws,
                               const WsLayout& L, const char* bws, const BwdLayout& B,
                               const int* ids, const float* T_final, const float* d_image,
                               cudaStream_t st) {
  float* grad = (float*)(ws + L.grad_sorted);
  cudaError_t e = cudaMemsetAsync(grad, 0, sizeof(float) * kGradStride * (size_t)L.N, st);
  if (e != cudaSuccess) return e;
  ViewBatch<CollectBwdView> b;
  b.n = 1;
  b.item0[0] = 0;
  b.item0[1] = L.n_tiles;
  b.v[0] = collect_bwd_view(c, ws, L, bws, B, ids, T_final, d_image);
  return launch_collect_bwd_batch(s, b, nullptr, st);
}


// Blended error (supp. Sec. 7.2, after Rota Bulo et al.): err[id] += sum over
// pixels of w e_p, w = alpha T the compositing weight of the surfel at the
// pixel, e_p the pixel's L1 error (mean over channels of |image - target|).
// The forward's walk without the top-K; per staged surfel the warp sums its
// lanes' w e_p with shuffles and one lane adds it.
template <typename KeyT>
__global__ void __launch_bounds__(kTilePix) k_blend_error(
    DevCam c, float alpha_min, float alpha_max, float T_min, uint32_t rmask,
    const uint2* __restrict__ ranges, const KeyT* __restrict__ keys,
    const float4* __restrict__ recs, const float* __restrict__ image,
    const float* __restrict__ target, float* __restrict__ err) {
  __shared__ float4 s_rec[kRecF4][kTilePix];
  const int tile = blockIdx.x;
  const int tx = tile % c.tiles_x, ty = tile / c.tiles_x;
  const int px = tx * kTile + (threadIdx.x & (kTile - 1));
  const int py = ty * kTile + (threadIdx.x / kTile);
  const bool inside = px < c.W && py < c.H;
  const float fpx = px + 0.5f, fpy = py + 0.5f;
  const uint2 rg = ranges[tile];
  float e = 0.f;
  if (inside) {
    const size_t p = (size_t)py * c.W + px;
    e = (fabsf(image[3 * p] - target[3 * p]) + fabsf(image[3 * p + 1] - target[3 * p + 1]) +
         fabsf(image[3 * p + 2] - target[3 * p + 2])) * (1.f / 3.f);
  }
  float T = 1.f;
  bool done = !inside || e == 0.f;
  for (uint32_t b0 = rg.x; b0 < rg.y; b0 += kTilePix) {
    if (__syncthreads_count(done) == kTilePix) break;
    uint32_t i = b0 + threadIdx.x;
    if (i < rg.y) {
      const float4* src = recs + (size_t)rank_of(keys[i], rmask) * kRecF4;
#pragma unroll
      for (int k = 0; k < kRecF4; ++k) s_rec[k][threadIdx.x] = __ldg(src + k);
    }
    __syncthreads();
    const int nb = (int)min((uint32_t)kTilePix, rg.y - b0);
    for (int j = 0; j < nb; ++j) {
      float we = 0.f;
      if (!done) {
        Hit h;
        if (eval_surfel(s_rec[0][j], s_rec[1][j], s_rec[2][j], s_rec[3][j], fpx, fpy, c.near_,
                        alpha_min, h)) {
          const float a = fminf(h.alpha, alpha_max);
          const float test = T * (1.f - a);
          if (test < T_min) {
            done = true;
          } else {
            we = a * T * e;
            T = test;
          }
        }
      }
      if (__ballot_sync(0xffffffffu, we != 0.f) == 0u) continue;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) we += __shfl_xor_sync(0xffffffffu, we, d);
      if ((threadIdx.x & 31) == 0 && we != 0.f)
        atomicAdd(err + __float_as_uint(s_rec[4][j].w), we);
    }
    __syncthreads();
  }
}

cudaError_t launch_blend_error(const DevCam& c, const nexel_settings& s, char* ws,
                               const WsLayout& L, const float* image, const float* target,
                               float* err, cudaStream_t st) {
  const uint32_t rmask = L.key64 ? 0xFFFFFFFFu : ((1u << L.rank_bits) - 1u);
  dim3 grid(L.n_tiles), block(kTilePix);
  auto* rg = (const uint2*)(ws + L.ranges);
  auto* recs = (const float4*)(ws + L.geom_sorted);
  NEXEL_PROF("blend_error", st);
  if (L.key64)
    k_blend_error<unsigned long long><<<grid, block, 0, st>>>(
        c, s.alpha_min, s.alpha_max, s.T_min, rmask, rg,
        (const unsigned long long*)(ws + L.inst0), recs, image, target, err);
  else
    k_blend_error<uint32_t><<<grid, block, 0, st>>>(c, s.alpha_min, s.alpha_max, s.T_min, rmask,
                                                    rg, (const uint32_t*)(ws + L.inst0), recs,
                                                    image, target, err);
  return cudaGetLastError();
}

}  // namespace nexel
