// C ABI of libnexel: argument checks, workspace layout and the launch
// sequence of each entry point.
#include "common.cuh"
#include "texture_common.cuh"

#include <cmath>
#include <cstring>

namespace nexel {

static size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

static int ceil_log2(long long n) {
  int b = 0;
  while ((1LL << b) < n) ++b;
  return b;
}

static void ws_fixed(const nexel_camera& cam, int N, WsLayout& L) {
  L.N = N;
  L.P = cam.width * cam.height;
  L.K = 0;
  int tx = (cam.width + kTile - 1) / kTile, ty = (cam.height + kTile - 1) / kTile;
  L.n_tiles = tx * ty;
  L.tile_bits = ceil_log2(L.n_tiles);
  L.rank_bits = std::max(1, ceil_log2(std::max(N, 2)));
  // direct placement by tile up to kPlaceMaxTiles tiles, whatever the key
  // width: a placed key needs no tile field (its slot gives the tile), so
  // when tile and rank bits exceed 32 it holds the rank alone; the tile sort
  // (more tiles) keeps (tile, rank) keys, 64-bit where they do not fit
  const bool fits32 = L.tile_bits + L.rank_bits <= 32;
  L.place_ok = L.n_tiles <= kPlaceMaxTiles ? 1 : 0;
  L.key64 = (!L.place_ok && !fits32) ? 1 : 0;
  L.rank_only = (L.place_ok && !fits32) ? 1 : 0;
  L.tile_passes = (L.tile_bits + 7) / 8;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += align_up(bytes);
    return at;
  };
  size_t n = (size_t)std::max(N, 1);
  L.geom_orig = take(n * kRecF4 * 16);
  L.geom_sorted = take(n * kRecF4 * 16);
  L.aux_orig = take(n * kAuxF4 * 16);
  L.aux_sorted = take(n * kAuxF4 * 16);
  L.dkey0 = take(n * 4);
  L.dkey1 = take(n * 4);
  L.did0 = take(n * 4);
  L.did1 = take(n * 4);  // after the depth sort: each surfel's rank (inverse permutation)
  L.rect = take(n * 8);
  L.conic = take(n * 48);
  L.tmask = take(n * 16);
  L.shj = take(n * 36);  // SH colour mode: d colour / d direction per surfel
  L.count = take(n * 4);
  L.offs = take((n + 1) * 4);
  L.ranges = take((size_t)L.n_tiles * 8);
  L.n_contrib = take((size_t)std::max(L.P, 1) * 4);
  L.grad_sorted = take(n * kGradStride * 4);
  L.counters = take(256);
  // direct placement by tile: [rank block][tile] counts and the tile starts
  const size_t place_blocks = L.place_ok ? (n + kPlaceRanks - 1) / kPlaceRanks : 0;
  L.place = take(place_blocks * (size_t)L.n_tiles * 4);
  L.place_tiles = take(L.place_ok ? (size_t)L.n_tiles * 4 : 0);
  L.mword_off = take(L.place_ok ? (n + 1) * 4 : 0);
  L.mword_cap = L.place_ok ? (long long)n * kMaskWordsPerSurfel : 0;
  L.mwords = take((size_t)L.mword_cap * 4);
  L.fixed_end = o;
}

static void ws_cap(WsLayout& L, long long cap) {
  L.cap = cap;
  size_t o = L.fixed_end;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += align_up(bytes);
    return at;
  };
  size_t kb = L.key64 ? 8 : 4;
  size_t c = (size_t)std::max(cap, 1LL);
  L.inst0 = take(c * kb);
  L.inst1 = take(c * kb);
  const size_t depth_tile = (size_t)kSortThreads * kSortItemsDepth;
  long long nb = std::max((c + kSortTile - 1) / kSortTile, ((size_t)L.N + depth_tile - 1) / depth_tile);
  L.hist = take((size_t)256 * nb * 4);
  // the scans: radix histograms, the N + 1 surfel counts, the tile starts
  long long scan_n = std::max(std::max(256LL * nb, (long long)L.N + 1), (long long)L.n_tiles);
  L.scan_sums = take(((size_t)(scan_n + kScanTile - 1) / kScanTile + 1) * 4);
  L.total = o;
}

WsLayout ws_layout(const nexel_camera& cam, int K, int N, long long cap) {
  WsLayout L;
  ws_fixed(cam, N, L);
  L.K = K;
  ws_cap(L, cap);
  return L;
}

WsLayout ws_layout_for_bytes(const nexel_camera& cam, int K, int N, size_t ws_bytes) {
  WsLayout L;
  ws_fixed(cam, N, L);
  L.K = K;
  ws_cap(L, 1);
  if (L.total > ws_bytes) {
    L.cap = -1;
    return L;
  }
  size_t kb = L.key64 ? 8 : 4;
  long long cap = (long long)((ws_bytes - L.fixed_end) / (2 * kb + 1));
  ws_cap(L, cap);
  while (L.total > ws_bytes && cap > 1) {
    cap -= std::max(1LL, cap / 1024);
    ws_cap(L, cap);
  }
  if (L.total > ws_bytes) L.cap = -1;
  return L;
}

BwdLayout bwd_layout(const nexel_camera& cam, int K, int feat_dim, bool recompute) {
  // per-sample gradients are indexed p * K + j; the features and texture
  // gradients by padded row (pixel-major, next power of two >= K rows per
  // pixel, rounded up to 16-row MMA tiles)
  BwdLayout B;
  const size_t P = (size_t)cam.width * cam.height;
  int KP = 1;
  while (KP < K) KP <<= 1;
  const size_t S = P * (size_t)std::max(K, 0);
  const size_t rows = ((P * (size_t)KP + 15) / 16) * 16;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += align_up(bytes);
    return at;
  };
  B.dweff = take(std::max<size_t>(S, 1) * 4);
  B.ddepth = take(std::max<size_t>(S, 1) * 4);
  B.feat = take(std::max<size_t>(rows, 1) * (size_t)std::max(feat_dim, 1) * 4);
  B.gtex = take(std::max<size_t>(rows, 1) * 16);
  // level-major (row stride rounded up to 32 rows)
  B.gin = take((std::max<size_t>(rows, 1) + 32) * (size_t)std::max(feat_dim, 1) * 4);
  const size_t rc = recompute ? 1 : 0;
  B.rc_notex = take(rc * P * 12);
  B.rc_weights = take(rc * S * 4);
  B.rc_ids = take(rc * S * 4);
  B.rc_depths = take(rc * S * 4);
  B.rc_T = take(rc * P * 4);
  B.status = take(256);
  B.total = o;
  return B;
}

DevCam make_devcam(const nexel_camera& cam) {
  DevCam c;
  c.W = cam.width;
  c.H = cam.height;
  c.tiles_x = (cam.width + kTile - 1) / kTile;
  c.tiles_y = (cam.height + kTile - 1) / kTile;
  c.fx = cam.fx; c.fy = cam.fy; c.cx = cam.cx; c.cy = cam.cy;
  const float* m = cam.world_to_cam;
  for (int r = 0; r < 3; ++r) {
    for (int k = 0; k < 3; ++k) c.R[3 * r + k] = m[4 * r + k];
    c.t[r] = m[4 * r + 3];
  }
  for (int a = 0; a < 3; ++a)
    c.o[a] = (float)-((double)c.R[a] * c.t[0] + (double)c.R[3 + a] * c.t[1] +
                      (double)c.R[6 + a] * c.t[2]);
  c.near_ = cam.near_plane;
  return c;
}

// Composite without textures (K = 0): C = N + T_final bg.
__global__ void k_composite_notex(long long P, float bg0, float bg1, float bg2,
                                  const float* __restrict__ notex, const float* __restrict__ Tf,
                                  float* __restrict__ image) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  float t = Tf[p];
  image[3 * p] = notex[3 * p] + t * bg0;
  image[3 * p + 1] = notex[3 * p + 1] + t * bg1;
  image[3 * p + 2] = notex[3 * p + 2] + t * bg2;
}

static bool cam_ok(const nexel_camera* c) {
  return c && c->width > 0 && c->height > 0 && c->width <= 16384 && c->height <= 16384 &&
         std::isfinite(c->fx) && std::isfinite(c->fy) && c->fx > 0 && c->fy > 0 &&
         c->near_plane > 0 && std::isfinite(c->near_plane) &&
         (long long)((c->width + kTile - 1) / kTile) * ((c->height + kTile - 1) / kTile) < (1 << 24);
}

static bool settings_ok(const nexel_settings* s) {
  return s && s->K >= 0 && s->K <= NEXEL_MAX_K && s->alpha_min > 0.f && s->alpha_max > 0.f &&
         s->alpha_max <= 1.f && s->alpha_min <= s->alpha_max && s->T_min >= 0.f &&
         s->T_min < 1.f && (s->grid_dtype == NEXEL_F32 || s->grid_dtype == NEXEL_F16) &&
         (s->mlp_dtype == NEXEL_F32 || s->mlp_dtype == NEXEL_BF16 || s->mlp_dtype == NEXEL_F16) &&
         (s->sh_degree == 0 || s->sh_degree == 3);
}

static bool field_ok(const nexel_field* f) {
  if (!f || !f->table || !f->weights) return false;
  if (f->L <= 0 || f->L > NEXEL_MAX_LEVELS || f->F != 2 || f->T <= 0) return false;
  if ((f->T & (f->T - 1)) != 0) return false;
  if (f->n_layers < 2 || f->n_layers > NEXEL_MAX_LAYERS) return false;
  for (int l = 0; l < f->L; ++l)
    if (!(f->level_scale[l] > 0.f) || !std::isfinite(f->level_scale[l])) return false;
  return true;
}

static int cuda_status(cudaError_t e) { return e == cudaSuccess ? NEXEL_OK : NEXEL_ERR_CUDA; }

template <typename KeyT>
__global__ void k_instance_list(long long n, int rank_bits, uint32_t rmask,
                                const KeyT* __restrict__ keys, const uint32_t* __restrict__ did,
                                const uint32_t* __restrict__ dkey, int* __restrict__ tile_out,
                                int* __restrict__ id_out, float* __restrict__ depth_out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  KeyT k = keys[i];
  uint32_t r = (uint32_t)k & rmask;
  if (tile_out) tile_out[i] = (int)(k >> rank_bits);
  if (id_out) id_out[i] = (int)did[r];
  if (depth_out) depth_out[i] = __uint_as_float(dkey[r]);
}

// Rank-only keys (placed instances whose tile and rank bits exceed 32): the
// tile of instance i is the last tile whose list starts at or before i (the
// lists are consecutive, in tile order; empty ones start where the next
// begins).
__global__ void k_instance_list_placed(long long n, int n_tiles, const uint2* __restrict__ ranges,
                                       const uint32_t* __restrict__ keys,
                                       const uint32_t* __restrict__ did,
                                       const uint32_t* __restrict__ dkey, int* __restrict__ tile_out,
                                       int* __restrict__ id_out, float* __restrict__ depth_out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t r = keys[i];
  if (tile_out) {
    int lo = 0, hi = n_tiles;  // first tile whose list starts after i
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if ((long long)ranges[mid].x <= i) lo = mid + 1;
      else hi = mid;
    }
    tile_out[i] = lo - 1;
  }
  if (id_out) id_out[i] = (int)did[r];
  if (depth_out) depth_out[i] = __uint_as_float(dkey[r]);
}

// Work statistics of the last forward on a workspace, reduced on the device
// into out[0..4] (64-bit counters in the counters block): Sigma_p last_p
// (list positions up to each pixel's last composited surfel), Sigma_tiles
// list length x pixels of the tile, the longest list, the surfels with at
// least one instance, and Sigma_tiles (max_p in tile last_p) x pixels of the
// tile (the lane iterations of the collection backward, which walks every
// tile from its largest last position down).
__global__ void __launch_bounds__(256) k_render_stats(int W, int H, int tiles_x, int n_tiles,
                                                      int N, const int* __restrict__ n_contrib,
                                                      const uint2* __restrict__ ranges,
                                                      const uint32_t* __restrict__ count,
                                                      unsigned long long* __restrict__ out) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  unsigned long long last = 0, walk = 0, vis = 0, longest = 0, bwalk = 0;
  for (long long p = tid; p < (long long)W * H; p += stride) last += (unsigned)n_contrib[p];
  for (long long t = tid; t < n_tiles; t += stride) {
    const uint2 r = ranges[t];
    const unsigned long long len = r.y > r.x ? r.y - r.x : 0;
    const int tx = (int)(t % tiles_x), ty = (int)(t / tiles_x);
    const int pw = min(kTile, W - tx * kTile), ph = min(kTile, H - ty * kTile);
    walk += len * (unsigned long long)(pw * ph);
    longest = max(longest, len);
    int tmax = 0;
    for (int y = 0; y < ph; ++y)
      for (int x = 0; x < pw; ++x)
        tmax = max(tmax, n_contrib[(size_t)(ty * kTile + y) * W + tx * kTile + x]);
    bwalk += (unsigned long long)tmax * (unsigned long long)(pw * ph);
  }
  for (long long i = tid; i < N; i += stride) vis += count[i] > 0 ? 1 : 0;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    last += __shfl_xor_sync(0xffffffffu, last, d);
    walk += __shfl_xor_sync(0xffffffffu, walk, d);
    vis += __shfl_xor_sync(0xffffffffu, vis, d);
    bwalk += __shfl_xor_sync(0xffffffffu, bwalk, d);
    longest = max(longest, __shfl_xor_sync(0xffffffffu, longest, d));
  }
  if ((threadIdx.x & 31) == 0) {
    if (last) atomicAdd(out + 0, last);
    if (walk) atomicAdd(out + 1, walk);
    if (longest) atomicMax(out + 2, longest);
    if (vis) atomicAdd(out + 3, vis);
    if (bwalk) atomicAdd(out + 4, bwalk);
  }
}

// ------------------------------------------------ per-view implementations
// Shared by the single-view entry points and the batched ones (batch.cu).

int check_fwd(const nexel_camera* cam, const nexel_settings* settings, const nexel_field* field,
              int N, const void* ws, size_t ws_bytes, const void* bwd_ws, size_t bwd_ws_bytes,
              const float* image, const float* notex, const float* weights, const int* ids,
              const float* depths, const float* textures, const float* T_final) {
  if (!cam_ok(cam) || !settings_ok(settings) || N < 0 || !ws || !image || !notex || !T_final)
    return NEXEL_ERR_INVALID_ARG;
  const int K = settings->K;
  if (K > 0 && (!weights || !ids || !depths || !textures)) return NEXEL_ERR_INVALID_ARG;
  if (K > 0 && !field_ok(field)) return NEXEL_ERR_INVALID_ARG;
  if (K > 0 && !texture_arch_supported(*settings, *field)) return NEXEL_ERR_UNSUPPORTED;
  if (K > 0 && settings->cache_features != 0) {
    BwdLayout B = bwd_layout(*cam, K, field->L * field->F, settings->recompute_buffers != 0);
    if (!bwd_ws || bwd_ws_bytes < B.total) return NEXEL_ERR_INVALID_ARG;
  }
  WsLayout L = ws_layout_for_bytes(*cam, K, N, ws_bytes);
  if (L.cap < 0) return NEXEL_ERR_INVALID_ARG;
  return NEXEL_OK;
}

int check_bwd(const nexel_camera* cam, const nexel_settings* settings, const nexel_field* field,
              int N, const float* mu, const float* quat, const float* scale, const float* opacity,
              const float* gamma, const void* ws, size_t ws_bytes, const void* bwd_ws,
              size_t bwd_ws_bytes, const float* weights, const int* ids, const float* depths,
              const float* T_final, const float* d_image) {
  const bool rc = settings && settings->recompute_buffers != 0;
  if (!cam_ok(cam) || !settings_ok(settings) || N < 0 || !ws || !d_image)
    return NEXEL_ERR_INVALID_ARG;
  if (!rc && !T_final) return NEXEL_ERR_INVALID_ARG;
  if (!(settings->alpha_max < 1.f)) return NEXEL_ERR_INVALID_ARG;
  if (N > 0 && (!mu || !quat || !scale || !opacity || !gamma)) return NEXEL_ERR_INVALID_ARG;
  const int K = settings->K;
  if (K > 0 && !rc && (!weights || !ids || !depths)) return NEXEL_ERR_INVALID_ARG;
  if ((K > 0 || rc) && !bwd_ws) return NEXEL_ERR_INVALID_ARG;
  if (K > 0 && !field_ok(field)) return NEXEL_ERR_INVALID_ARG;
  if (K > 0 && !texture_arch_supported(*settings, *field)) return NEXEL_ERR_UNSUPPORTED;
  WsLayout L = ws_layout_for_bytes(*cam, K, N, ws_bytes);
  if (L.cap < 0) return NEXEL_ERR_INVALID_ARG;
  BwdLayout B = bwd_layout(*cam, K, K > 0 ? field->L * field->F : 0, rc);
  if ((K > 0 || rc) && bwd_ws_bytes < B.total) return NEXEL_ERR_INVALID_ARG;
  return NEXEL_OK;
}

int preprocess_impl(const nexel_camera* cam, const nexel_settings* settings, int N,
                    const float* mu, const float* quat, const float* scale, const float* opacity,
                    const float* gamma, const float* color, void* ws, size_t ws_bytes,
                    long long* n_instances_out, cudaStream_t st) {
  if (!cam_ok(cam) || !settings_ok(settings) || N < 0 || !ws) return NEXEL_ERR_INVALID_ARG;
  if (N > 0 && (!mu || !quat || !scale || !opacity || !gamma || !color))
    return NEXEL_ERR_INVALID_ARG;
  WsLayout L = ws_layout_for_bytes(*cam, settings->K, N, ws_bytes);
  if (L.cap < 0) return NEXEL_ERR_INVALID_ARG;
  DevCam c = make_devcam(*cam);
  char* w = (char*)ws;
  cudaError_t e = cudaMemsetAsync(w + L.counters, 0, 256, st);
  if (e == cudaSuccess)
    e = launch_preprocess(c, *settings, N, mu, quat, scale, opacity, gamma, color, w, L, st);
  if (e == cudaSuccess) e = launch_depth_sort(N, w, L, st);
  if (e == cudaSuccess) e = launch_count_scan(N, w, L, st);
  if (e != cudaSuccess) return NEXEL_ERR_CUDA;
  if (!n_instances_out)  // device-count form: no host synchronisation
    return cuda_status(launch_binning(c, N, -1, w, L, st));
  uint32_t n_inst = 0;
  e = cudaMemcpyAsync(&n_inst, w + L.counters + kCountersInst, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return NEXEL_ERR_CUDA;
  *n_instances_out = (long long)n_inst;
  if ((long long)n_inst > L.cap) return NEXEL_ERR_CAPACITY;
  return cuda_status(launch_binning(c, N, (long long)n_inst, w, L, st));
}

int render_fwd_impl(const nexel_camera* cam, const nexel_settings* settings,
                    const nexel_field* field, int N, void* ws, size_t ws_bytes, void* bwd_ws,
                    float* image, float* notex, float* weights, int* ids, float* depths,
                    float* textures, float* T_final, cudaStream_t st) {
  const int K = settings->K;
  void* feat_cache = nullptr;
  if (K > 0 && settings->cache_features != 0) {
    BwdLayout B = bwd_layout(*cam, K, field->L * field->F, settings->recompute_buffers != 0);
    feat_cache = (char*)bwd_ws + B.feat;
  }
  WsLayout L = ws_layout_for_bytes(*cam, K, N, ws_bytes);
  DevCam c = make_devcam(*cam);
  char* w = (char*)ws;
  cudaError_t e = launch_collect_fwd(c, *settings, w, L, notex, weights, ids, depths, T_final, st);
  if (e != cudaSuccess) return NEXEL_ERR_CUDA;
  if (K == 0) {
    long long P = (long long)cam->width * cam->height;
    {
      NEXEL_PROF("composite_notex", st);
      k_composite_notex<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(
          P, settings->bg[0], settings->bg[1], settings->bg[2], notex, T_final, image);
    }
    return cuda_status(cudaGetLastError());
  }
  e = launch_texture_fwd(c, *settings, *field, notex, weights, ids, depths, T_final, image,
                         textures, feat_cache, (int*)(w + L.counters + kStatusOffset), st);
  return cuda_status(e);
}

int zero_grads(const nexel_settings* settings, const nexel_field* field, int N, float* d_mu,
               float* d_quat, float* d_scale, float* d_opacity, float* d_gamma, float* d_color,
               float* d_table, float* d_mlp, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  const size_t n = (size_t)std::max(N, 0);
  auto z = [&](float* p, size_t count) {
    if (e == cudaSuccess && p && count) e = cudaMemsetAsync(p, 0, sizeof(float) * count, st);
  };
  z(d_mu, 3 * n);
  z(d_quat, 4 * n);
  z(d_scale, 2 * n);
  z(d_opacity, n);
  z(d_gamma, 2 * n);
  z(d_color, (settings->sh_degree == 3 ? 48 : 3) * n);  // RGB, or 16 SH coefficients x 3
  if (settings->K > 0 && field) {
    z(d_table, (size_t)field->L * field->T * field->F);
    size_t nw = 0;
    for (int l = 0; l < field->n_layers; ++l) nw += (size_t)field->widths[l] * field->widths[l + 1];
    z(d_mlp, nw);
  }
  return cuda_status(e);
}

int render_bwd_impl(const nexel_camera* cam, const nexel_settings* settings,
                    const nexel_field* field, int N, const float* mu, const float* quat,
                    const float* scale, const float* opacity, const float* gamma, void* ws,
                    size_t ws_bytes, void* bwd_ws, const float* weights, const int* ids,
                    const float* depths, const float* T_final, const float* d_image,
                    const float* d_weights, const float* d_textures, float* d_mu, float* d_quat,
                    float* d_scale, float* d_opacity, float* d_gamma, float* d_color,
                    float* d_table, float* d_mlp, int grad_mode, cudaStream_t st) {
  const bool atomic_params = grad_mode == kGradShared;
  const bool rc = settings->recompute_buffers != 0;
  const int K = settings->K;
  WsLayout L = ws_layout_for_bytes(*cam, K, N, ws_bytes);
  BwdLayout B = bwd_layout(*cam, K, K > 0 ? field->L * field->F : 0, rc);
  DevCam c = make_devcam(*cam);
  char* w = (char*)ws;
  char* bw = (char*)bwd_ws;
  // the scratch is the caller's uninitialised memory: the backward's status
  // word (read by nexel_read_status) starts at zero on every backward that
  // has a scratch (K > 0 or recompute), in every form
  cudaError_t e = (bw && (K > 0 || rc)) ? cudaMemsetAsync(bw + B.status, 0, 4, st) : cudaSuccess;
  if (e == cudaSuccess && rc) {
    // recompute I, W, D, T_final with the collection pass (same kernel, same
    // inputs, hence the same values the forward produced)
    weights = (const float*)(bw + B.rc_weights);
    ids = (const int*)(bw + B.rc_ids);
    depths = (const float*)(bw + B.rc_depths);
    T_final = (const float*)(bw + B.rc_T);
    e = launch_collect_fwd(c, *settings, w, L, (float*)(bw + B.rc_notex), (float*)weights,
                           (int*)ids, (float*)depths, (float*)T_final, st);
  }
  if (e == cudaSuccess && K > 0)
    e = launch_texture_bwd(c, *settings, *field, bw, B, weights, ids, depths, d_image, d_weights,
                           d_textures, d_table, d_mlp, settings->cache_features != 0,
                           grad_mode, st);
  if (e == cudaSuccess) e = launch_collect_bwd(c, *settings, w, L, bw, B, ids, T_final, d_image, st);
  if (e == cudaSuccess)
    e = launch_preprocess_bwd(c, *settings, N, mu, quat, scale, opacity, gamma, w, L, 1, d_mu,
                              d_quat, d_scale, d_opacity, d_gamma, d_color, atomic_params, st);
  return cuda_status(e);
}

}  // namespace nexel

using namespace nexel;

extern "C" {

int nexel_version(void) { return 100; }

const char* nexel_status_string(int status) {
  switch (status) {
    case NEXEL_OK: return "ok";
    case NEXEL_ERR_INVALID_ARG: return "invalid argument";
    case NEXEL_ERR_CUDA: return "CUDA error";
    case NEXEL_ERR_CAPACITY: return "instance capacity exceeded";
    case NEXEL_ERR_UNSUPPORTED: return "unsupported configuration";
    case NEXEL_ERR_TIMEOUT: return "device wait timed out";
    case NEXEL_ERR_NUMERIC: return "numeric check failed";
    default: return "unknown status";
  }
}

int nexel_workspace_size(const nexel_camera* cam, int N, long long max_instances, size_t* bytes) {
  if (!cam_ok(cam) || N < 0 || max_instances < 0 || !bytes) return NEXEL_ERR_INVALID_ARG;
  if (max_instances >= (1LL << 32) - 1) return NEXEL_ERR_UNSUPPORTED;
  WsLayout L = ws_layout(*cam, 0, N, max_instances);
  *bytes = L.total;
  return NEXEL_OK;
}

int nexel_bwd_workspace_size(const nexel_camera* cam, const nexel_settings* settings,
                             const nexel_field* field, size_t* bytes) {
  if (!cam_ok(cam) || !settings_ok(settings) || !bytes) return NEXEL_ERR_INVALID_ARG;
  int fd = (settings->K > 0 && field) ? field->L * field->F : 0;
  *bytes = bwd_layout(*cam, settings->K, fd, settings->recompute_buffers != 0).total;
  return NEXEL_OK;
}

int nexel_preprocess(const nexel_camera* cam, const nexel_settings* settings, int N,
                     const float* mu, const float* quat, const float* scale,
                     const float* opacity, const float* gamma, const float* color, void* ws,
                     size_t ws_bytes, long long* n_instances_out, nexel_stream_t stream) {
  if (!n_instances_out) return NEXEL_ERR_INVALID_ARG;
  return preprocess_impl(cam, settings, N, mu, quat, scale, opacity, gamma, color, ws, ws_bytes,
                         n_instances_out, (cudaStream_t)stream);
}

int nexel_preprocess_async(const nexel_camera* cam, const nexel_settings* settings, int N,
                           const float* mu, const float* quat, const float* scale,
                           const float* opacity, const float* gamma, const float* color,
                           void* ws, size_t ws_bytes, nexel_stream_t stream) {
  return preprocess_impl(cam, settings, N, mu, quat, scale, opacity, gamma, color, ws, ws_bytes,
                         nullptr, (cudaStream_t)stream);
}

int nexel_render_fwd(const nexel_camera* cam, const nexel_settings* settings,
                     const nexel_field* field, int N, void* ws, size_t ws_bytes, void* bwd_ws,
                     size_t bwd_ws_bytes, float* image, float* notex, float* weights, int* ids,
                     float* depths, float* textures, float* T_final, nexel_stream_t stream) {
  int rc = check_fwd(cam, settings, field, N, ws, ws_bytes, bwd_ws, bwd_ws_bytes, image, notex,
                     weights, ids, depths, textures, T_final);
  if (rc != NEXEL_OK) return rc;
  return render_fwd_impl(cam, settings, field, N, ws, ws_bytes, bwd_ws, image, notex, weights,
                         ids, depths, textures, T_final, (cudaStream_t)stream);
}

int nexel_render_bwd(const nexel_camera* cam, const nexel_settings* settings,
                     const nexel_field* field, int N, const float* mu, const float* quat,
                     const float* scale, const float* opacity, const float* gamma, void* ws,
                     size_t ws_bytes, void* bwd_ws, size_t bwd_ws_bytes, const float* weights,
                     const int* ids, const float* depths, const float* T_final,
                     const float* d_image, const float* d_weights, const float* d_textures,
                     int accumulate, float* d_mu, float* d_quat, float* d_scale, float* d_opacity,
                     float* d_gamma, float* d_color, float* d_table, float* d_mlp,
                     nexel_stream_t stream) {
  int rc = check_bwd(cam, settings, field, N, mu, quat, scale, opacity, gamma, ws, ws_bytes,
                     bwd_ws, bwd_ws_bytes, weights, ids, depths, T_final, d_image);
  if (rc != NEXEL_OK) return rc;
  if (settings->sh_degree == 3 && ((uintptr_t)d_color & 15)) return NEXEL_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (!accumulate) {
    rc = zero_grads(settings, field, N, d_mu, d_quat, d_scale, d_opacity, d_gamma, d_color,
                    d_table, d_mlp, st);
    if (rc != NEXEL_OK) return rc;
  }
  return render_bwd_impl(cam, settings, field, N, mu, quat, scale, opacity, gamma, ws, ws_bytes,
                         bwd_ws, weights, ids, depths, T_final, d_image, d_weights, d_textures,
                         d_mu, d_quat, d_scale, d_opacity, d_gamma, d_color, d_table, d_mlp,
                         accumulate ? kGradExclusive : kGradZeroed, st);
}

int nexel_read_status(const nexel_camera* cam, const nexel_settings* settings,
                      const nexel_field* field, int N, void* ws, size_t ws_bytes, void* bwd_ws,
                      size_t bwd_ws_bytes, nexel_stream_t stream) {
  if (!cam_ok(cam) || !settings_ok(settings) || N < 0 || !ws) return NEXEL_ERR_INVALID_ARG;
  WsLayout L = ws_layout_for_bytes(*cam, settings->K, N, ws_bytes);
  if (L.cap < 0) return NEXEL_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int words[2] = {0, 0};
  char* w = (char*)ws;
  cudaError_t e = cudaMemcpyAsync(&words[0], w + L.counters + kStatusOffset, 4,
                                  cudaMemcpyDeviceToHost, st);
  char* bstat = nullptr;
  // the backward's status word exists where it has a scratch (K > 0 or
  // recompute)
  if (bwd_ws && (settings->K > 0 || settings->recompute_buffers != 0)) {
    const int K = settings->K;
    const int fd = (K > 0 && field_ok(field)) ? field->L * field->F : 0;
    BwdLayout B = bwd_layout(*cam, K, fd, settings->recompute_buffers != 0);
    if (bwd_ws_bytes < B.total) return NEXEL_ERR_INVALID_ARG;
    bstat = (char*)bwd_ws + B.status;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(&words[1], bstat, 4, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemsetAsync(w + L.counters + kStatusOffset, 0, 4, st);
  if (e == cudaSuccess && bstat) e = cudaMemsetAsync(bstat, 0, 4, st);
  if (e != cudaSuccess) return NEXEL_ERR_CUDA;
  const int f = words[0] | words[1];
  if (f & kStatusTimeout) return NEXEL_ERR_TIMEOUT;
  if (f & kStatusCapacity) return NEXEL_ERR_CAPACITY;
  if (f & kStatusNumeric) return NEXEL_ERR_NUMERIC;
  return NEXEL_OK;
}

int nexel_instance_list(const nexel_camera* cam, int N, const void* ws, size_t ws_bytes,
                        long long n_instances, int* tile_out, int* id_out, float* depth_out,
                        nexel_stream_t stream) {
  if (!cam_ok(cam) || N < 0 || !ws || n_instances < 0) return NEXEL_ERR_INVALID_ARG;
  WsLayout L = ws_layout_for_bytes(*cam, 0, N, ws_bytes);
  if (L.cap < 0 || n_instances > L.cap) return NEXEL_ERR_INVALID_ARG;
  if (n_instances == 0) return NEXEL_OK;
  const char* w = (const char*)ws;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned grid = (unsigned)((n_instances + 255) / 256);
  const uint32_t* did = (const uint32_t*)(w + L.did0);
  const uint32_t* dk = (const uint32_t*)(w + L.dkey0);
  if (L.rank_only)
    {
      NEXEL_PROF("instance_list", st);
      k_instance_list_placed<<<grid, 256, 0, st>>>(n_instances, L.n_tiles,
                                                   (const uint2*)(w + L.ranges),
                                                   (const uint32_t*)(w + L.inst0), did, dk,
                                                   tile_out, id_out, depth_out);
    }
  else if (L.key64)
    {
      NEXEL_PROF("instance_list", st);
      k_instance_list<unsigned long long><<<grid, 256, 0, st>>>(
          n_instances, 32, 0xFFFFFFFFu, (const unsigned long long*)(w + L.inst0), did, dk, tile_out,
          id_out, depth_out);
    }
  else
    {
      NEXEL_PROF("instance_list", st);
      k_instance_list<uint32_t><<<grid, 256, 0, st>>>(n_instances, L.rank_bits,
                                                      (1u << L.rank_bits) - 1u,
                                                      (const uint32_t*)(w + L.inst0), did, dk,
                                                      tile_out, id_out, depth_out);
    }
  return cuda_status(cudaGetLastError());
}

int nexel_render_stats(const nexel_camera* cam, const nexel_settings* settings, int N,
                       void* ws, size_t ws_bytes, long long* out, nexel_stream_t stream) {
  if (!cam_ok(cam) || !settings_ok(settings) || N < 0 || !ws || !out)
    return NEXEL_ERR_INVALID_ARG;
  WsLayout L = ws_layout_for_bytes(*cam, settings->K, N, ws_bytes);
  if (L.cap < 0) return NEXEL_ERR_INVALID_ARG;
  char* w = (char*)ws;
  cudaStream_t st = (cudaStream_t)stream;
  auto* acc = (unsigned long long*)(w + L.counters + kStatsOffset);
  cudaError_t e = cudaMemsetAsync(acc, 0, 5 * sizeof(unsigned long long), st);
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    NEXEL_PROF("render_stats", st);
    k_render_stats<<<2 * nsm, 256, 0, st>>>(cam->width, cam->height,
                                            (cam->width + kTile - 1) / kTile, L.n_tiles, N,
                                            (const int*)(w + L.n_contrib),
                                            (const uint2*)(w + L.ranges),
                                            (const uint32_t*)(w + L.count), acc);
    e = cudaGetLastError();
  }
  unsigned long long h[5] = {0, 0, 0, 0, 0};
  uint32_t n_inst = 0, n_bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&n_inst, w + L.counters + kCountersInst, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&n_bad, w + L.counters + kCountersNonFinite, 4, cudaMemcpyDeviceToHost,
                        st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return NEXEL_ERR_CUDA;
  out[0] = (long long)n_inst;
  out[1] = (long long)h[3];
  out[2] = (long long)h[0];
  out[3] = (long long)h[1];
  out[4] = (long long)h[2];
  out[5] = (long long)L.n_tiles;
  out[6] = (long long)h[4];
  out[7] = (long long)n_bad;
  return NEXEL_OK;
}

}  // extern "C"
