// Hash-grid backward (shared by the FP32 and BF16 forms): the scatter of
// the feature gradient into the table gradient (the adjoint of the
// trilinear lookup of Eq. 4 with the down-weighting of Eq. 3) and dL/dD of
// every textured sample through x = o + D d and Delta(D).
//
// Layout: a warp handles one slot j of 32 consecutive pixels (lane = pixel)
// and walks all L levels, keeping dL/dD of its samples in registers, so the
// kernel writes dL/dD directly.  The KP warps of a pixel group (its KP
// slots) sit side by side and move through the levels together, so the
// 32-byte sectors of the slot-interleaved feature gradient they read are
// shared in L1; successive pixel groups start at successive levels, so the
// warps in flight spread over all levels (updates to the few entries of a
// coarse level would otherwise pile up on the same L2 lines).
//
// Atomics: at one level, neighbouring pixels of the same slot share cells
// once a cell spans a pixel or more.  Per level the warp finds the runs of
// consecutive lanes in the same cell (shuffles + ballot); per corner it sums
// each run with a segmented shuffle scan (as many steps as the longest run
// needs, none when every lane has its own cell) and lets the run's last lane
// issue one vector atomic per entry.  A run whose successor lies in the
// x-adjacent cell hands its entries at x + 1 to the successor's entries at
// x, so they are added once.
//
// Paired table-gradient order: for an odd lattice x (either sign), the
// MapPositive values of x and x + 1 differ in bit 1 only, so the entries of
// a corner at x and at x + 1 (same y, z) are i and i ^ 2.  While the kernel
// runs, the table gradient is held with bits 0 and 1 of every entry index
// swapped (a pass before and one after, each swapping entries 1 and 2 of
// every 4-entry group), which makes i and i ^ 2 one aligned 16-byte pair:
// an odd-x run adds both with one 4-wide vector reduction.  L2 vector
// reductions cost the same per instruction whether 8 or 16 bytes wide, so
// this removes a quarter of the reductions wherever every lane has its own
// cell.
#include "texture_common.cuh"

namespace nexel {

namespace {

constexpr int kHbThreads = 256;
constexpr int kHbMinBlocks = 5;

// Inclusive segmented scan of (vx, vy) over the lanes; seg_start is the
// first lane of the calling lane's segment, max_len (warp-uniform) the
// longest segment.
__device__ __forceinline__ void seg_scan2(float& vx, float& vy, int lane, int seg_start,
                                          int max_len) {
  for (int d = 1; d < max_len; d <<= 1) {
    const float ox = __shfl_up_sync(0xffffffffu, vx, d);
    const float oy = __shfl_up_sync(0xffffffffu, vy, d);
    if (lane - d >= seg_start) {
      vx += ox;
      vy += oy;
    }
  }
}

// bits 0 and 1 of an entry index swapped: its position in the paired order
__device__ __forceinline__ uint32_t swap01(uint32_t i) {
  return (i & ~3u) | ((i & 1u) << 1) | ((i >> 1) & 1u);
}

// Natural <-> paired table-gradient order (an involution): entries 1 and 2
// of every 4-entry (32-byte) group trade places.
__global__ void k_swap_pairs(float4* __restrict__ t, long long groups) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (g >= groups) return;
  const float4 a = t[2 * g], b = t[2 * g + 1];  // entries 0, 1 | 2, 3
  t[2 * g] = make_float4(a.x, a.y, b.x, b.y);
  t[2 * g + 1] = make_float4(a.z, a.w, b.z, b.w);
}

}  // namespace

template <typename TT, bool MV>
__global__ void __launch_bounds__(kHbThreads, kHbMinBlocks) k_hash_bwd(
    const __grid_constant__ ViewBatch<HashBwdView> b, FieldDev f, int K, int log2KP,
    float* __restrict__ d_table, bool paired) {
  const int lane = threadIdx.x & 31;
  const int item = (int)(blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5));
  if (item >= b.item0[b.n]) return;  // whole warps
  const int vi = MV ? view_of(b, item) : 0;  // MV: a batch of views
  const HashBwdView& V = b.v[vi];
  const DevCam& c = V.c;
  const uint32_t n_rows = V.n_rows, R = V.R;
  const int* __restrict__ ids = V.ids;
  const float* __restrict__ depths = V.depths;
  const float2* __restrict__ gin = V.gin;
  // the view's own warp index
  const uint32_t gw = (uint32_t)(MV ? item - b.item0[vi] : item);
  // warp gw: slot j = gw % KP of the 32 consecutive pixels 32 (gw / KP) ..
  const int KP = 1 << log2KP;
  const uint32_t r = ((gw >> log2KP) * 32u + (uint32_t)lane) * (uint32_t)KP + (gw & (KP - 1));
  if ((gw >> log2KP) * 32u * (uint32_t)KP >= n_rows) return;  // whole warps
  const uint32_t P = (uint32_t)c.W * (uint32_t)c.H;
  const uint32_t p = r >> log2KP;
  const int j = (int)(r & (uint32_t)(KP - 1));
  const uint32_t s = p * (uint32_t)K + (uint32_t)j;
  bool valid = r < n_rows && p < P && j < K;
  if (valid) valid = ids[s] >= 0;
  if (!__any_sync(0xffffffffu, valid)) return;  // whole warps
  float D = 1.f;
  float3 d = make_float3(0.f, 0.f, 1.f);
  if (valid) {
    D = depths[s];
    d = pixel_dir(c, (int)(p % (uint32_t)c.W), (int)(p / (uint32_t)c.W));
  }
  const float iD = 1.f / D, fD = c.fx * iD;  // f of Eq. 3: the view's focal length
  const float3 x = make_float3(c.o[0] + D * d.x, c.o[1] + D * d.y, c.o[2] + D * d.z);
  const size_t T = (size_t)f.mask + 1;
  const int L = f.L;
  float dt = 0.f;
  // pixel groups start at successive levels; the KP warps of a group move
  // together
  int l = (int)((gw >> log2KP) % (uint32_t)L);
  for (int it = 0; it < L; ++it, l = (l + 1 == L) ? 0 : l + 1) {
    // the feature gradient is streamed once: evict-first, so that the table
    // and its gradient keep their L2 lines
    const float2 g = valid ? __ldcs(gin + (size_t)l * R + r) : make_float2(0.f, 0.f);
    const float sl = f.s[l];
    const float gx = sl * x.x, gy = sl * x.y, gz = sl * x.z;
    const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
    const int cx = (int)fx0, cy = (int)fy0, cz = (int)fz0;
    const float rx = gx - fx0, ry = gy - fy0, rz = gz - fz0;
    const float rr = fD * f.inv_s[l];  // cell size in pixels at depth D
    // Eq. 3: Delta = 1 - exp(-r^2 / 2pi), r = f / (s D)
    const float dw = one_minus_exp_neg(rr * rr * 0.15915494309189535f);
    // per-axis parts of the spatial hash (MapPositive, times the primes)
    const uint32_t hx[2] = {map_pos(cx), map_pos(cx + 1)};
    const uint32_t hy[2] = {map_pos(cy) * 2654435761u, map_pos(cy + 1) * 2654435761u};
    const uint32_t hz[2] = {map_pos(cz) * 805459861u, map_pos(cz + 1) * 805459861u};
    const float wx[2] = {1.f - rx, rx}, wy[2] = {1.f - ry, ry}, wz[2] = {1.f - rz, rz};
    const TT* tl = reinterpret_cast<const TT*>(f.table) + (size_t)l * T * 2;
    float2* dl = d_table ? reinterpret_cast<float2*>(d_table + (size_t)l * T * 2) : nullptr;
    // neighbour structure along the warp (consecutive pixels of one slot):
    // a lane whose successor lies in the same cell shares all 8 entries
    // with it; one whose successor lies in the next cell along x shares its
    // 4 entries at x + 1 with the successor's entries at x
    const int ncx = __shfl_down_sync(0xffffffffu, cx, 1);
    const int ncy = __shfl_down_sync(0xffffffffu, cy, 1);
    const int ncz = __shfl_down_sync(0xffffffffu, cz, 1);
    const bool nvalid = __shfl_down_sync(0xffffffffu, valid, 1) && lane < 31;
    const bool yz_next = valid && nvalid && ncy == cy && ncz == cz;
    const bool same_next = yz_next && ncx == cx, adj_next = yz_next && ncx == cx + 1;
    const bool same_prev = __shfl_up_sync(0xffffffffu, same_next, 1) && lane > 0;
    const bool adj_prev = __shfl_up_sync(0xffffffffu, adj_next, 1) && lane > 0;
    const unsigned heads = __ballot_sync(0xffffffffu, !same_prev);
    // runs of one cell are summed with a segmented scan whose step count
    // follows the longest run (no steps when every lane has its own cell)
    const int seg_start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
    const int max_len = (int)__reduce_max_sync(0xffffffffu, (unsigned)(lane - seg_start)) + 1;
    const bool tail = !same_next;
    // odd x: the entries at x and x + 1 form one 16-byte pair (paired order)
    const bool pair = paired && (cx & 1) != 0;
    const float gsx = dw * g.x, gsy = dw * g.y;
    float ax = 0.f, ay = 0.f, qx = 0.f, qy = 0.f, qz = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
      const uint32_t idx = (hx[dx] ^ hy[dy] ^ hz[dz]) & f.mask;
      const float wyz = wy[dy] * wz[dz], wxz = wx[dx] * wz[dz], wxy = wx[dx] * wy[dy];
      const float w = wxy * wz[dz];
      if (valid) {
        const float2 e = load_entry<TT>(tl, idx);
        ax = fmaf(w, e.x, ax);
        ay = fmaf(w, e.y, ay);
        const float ge = fmaf(g.x, e.x, g.y * e.y);
        qx = fmaf(ge, dx ? wyz : -wyz, qx);
        qy = fmaf(ge, dy ? wxz : -wxz, qy);
        qz = fmaf(ge, dz ? wxy : -wxy, qz);
      }
    }
    if (dl) {
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {  // (dy, dz) pairs: entries at x and x + 1
        const int dy = kk & 1, dz = kk >> 1;
        const uint32_t hyz = hy[dy] ^ hz[dz];
        const float wyz = wy[dy] * wz[dz];
        float v0x = wx[0] * wyz * gsx, v0y = wx[0] * wyz * gsy;
        float v1x = wx[1] * wyz * gsx, v1y = wx[1] * wyz * gsy;
        seg_scan2(v1x, v1y, lane, seg_start, max_len);
        // the run ending here hands its x + 1 sums to the next run's x entry
        // (unless it adds them in its own pair); px is 0 when nothing came
        const bool hand = tail && adj_next && !pair;
        const float px = __shfl_up_sync(0xffffffffu, hand ? v1x : 0.f, 1);
        const float py = __shfl_up_sync(0xffffffffu, hand ? v1y : 0.f, 1);
        if (adj_prev && lane > 0) {
          v0x += px;
          v0y += py;
        }
        seg_scan2(v0x, v0y, lane, seg_start, max_len);
        if (valid && tail) {
          const uint32_t i0 = (hx[0] ^ hyz) & f.mask, i1 = (hx[1] ^ hyz) & f.mask;
          const uint32_t q0 = paired ? swap01(i0) : i0;
          if (pair) {  // entries x and x + 1 at q0 and q0 ^ 1
            const float4 v = (q0 & 1u) ? make_float4(v1x, v1y, v0x, v0y)
                                       : make_float4(v0x, v0y, v1x, v1y);
            atomicAdd(reinterpret_cast<float4*>(dl + (q0 & ~1u)), v);
          } else {
            atomicAdd(dl + q0, make_float2(v0x, v0y));
            if (!adj_next) atomicAdd(dl + (paired ? swap01(i1) : i1), make_float2(v1x, v1y));
          }
        }
      }
    }
    // Delta = 1 - exp(-r^2 / 2pi), r = f / (s D): dDelta/dD = -(1 - Delta) r^2 / (pi D)
    const float ddw = -(1.f - dw) * rr * rr * 0.3183098861837907f * iD;
    dt += (g.x * ax + g.y * ay) * ddw + dw * sl * (qx * d.x + qy * d.y + qz * d.z);
  }
  if (valid) V.ddepth[s] = dt;
}

cudaError_t launch_hash_bwd_batch(const FieldDev& fd, int K, int KP, bool half_table,
                                  const ViewBatch<HashBwdView>& b, float* d_table,
                                  cudaStream_t st) {
  int log2KP = 0;
  while ((1 << log2KP) < KP) ++log2KP;
  if ((1 << log2KP) != KP || KP > 32 || fd.L < 1 || fd.L > NEXEL_MAX_LEVELS || K <= 0)
    return cudaErrorInvalidValue;
  const long long warps = b.item0[b.n];
  if (warps <= 0) return cudaSuccess;
  // CTA size: 256 threads, or 128 when the tuning asks (a multiple of the
  // KP warps of a pixel group either way)
  const unsigned block = current_tuning().hash_block == 128 ? 128u : (unsigned)kHbThreads;
  const unsigned grid = (unsigned)((warps * 32 + block - 1) / block);
  auto kern = half_table ? (b.n > 1 ? k_hash_bwd<__half, true> : k_hash_bwd<__half, false>)
                         : (b.n > 1 ? k_hash_bwd<float, true> : k_hash_bwd<float, false>);
  // the table gradient in paired order while the kernel runs (when no
  // other work writes it meanwhile, T >= 4 and it is 16-byte aligned; else
  // natural order)
  const bool paired =
      fd.grad_mode != kGradShared && d_table && fd.mask >= 3u && ((uintptr_t)d_table & 15u) == 0;
  const long long groups = paired ? (long long)fd.L * ((long long)fd.mask + 1) / 4 : 0;
  const unsigned sgrid = (unsigned)((groups + 255) / 256);
  if (paired && fd.grad_mode != kGradZeroed) {  // zeros need no reordering
    NEXEL_PROF("hash_bwd_order", st);
    k_swap_pairs<<<sgrid, 256, 0, st>>>(reinterpret_cast<float4*>(d_table), groups);
  }
  {
    NEXEL_PROF("hash_bwd", st);
    kern<<<grid, block, 0, st>>>(b, fd, K, log2KP, d_table, paired);
  }
  if (paired) {
    NEXEL_PROF("hash_bwd_order", st);
    k_swap_pairs<<<sgrid, 256, 0, st>>>(reinterpret_cast<float4*>(d_table), groups);
  }
  return cudaGetLastError();
}

cudaError_t launch_hash_bwd(const DevCam& c, const FieldDev& fd, int K, int KP, long long n_rows,
                            bool half_table, const int* ids, const float* depths,
                            const float2* gin, float* ddepth, float* d_table, cudaStream_t st) {
  if (n_rows <= 0 || K <= 0) return cudaSuccess;
  if (gin_stride(n_rows) >= (1LL << 32)) return cudaErrorInvalidValue;
  ViewBatch<HashBwdView> b;
  b.n = 1;
  b.item0[0] = 0;
  b.item0[1] = hash_bwd_items(n_rows, KP);
  b.v[0] = HashBwdView{c, ids, depths, gin, ddepth, (uint32_t)n_rows, (uint32_t)gin_stride(n_rows)};
  return launch_hash_bwd_batch(fd, K, KP, half_table, b, d_table, st);
}

}  // namespace nexel
