// Hash-grid backward (shared by the FP32 and BF16 forms).
//
// Thread layout: warp w covers 32 consecutive sample rows at level w mod L,
// so lanes are neighbouring pixels (and slots) — spatially coherent
// samples — while the warps in flight spread over all levels.  Each lane recomputes its intersection point
// x = o + D d, the cell and trilinear weights at its level, reads the 8
// corner entries (for the positional gradient) and adds
// Delta_l * w_corner * dL/dh_l into the FP32 table gradient.
//
// Atomics: at coarse levels thousands of samples update the same few
// entries, and the L2 serialises updates to one address.  Per corner, the
// warp therefore finds runs of consecutive lanes with the same entry
// (shfl_up + ballot); when there are few runs it sums each run with a
// segmented shuffle scan and lets the run's last lane issue one vector
// atomic.  Warps with many distinct entries (fine levels) issue plain
// per-lane atomics.
//
// Each lane's share of dL/dD (through Delta_l and the trilinear weights with
// x = o + D d) goes to dtl[level][row]; k_sum_levels adds the levels.
#include "texture_common.cuh"

namespace nexel {

__device__ __forceinline__ void run_atomic_add2(float2* base, uint32_t idx, float vx, float vy,
                                                bool valid) {
  const int lane = threadIdx.x & 31;
  const uint32_t key = valid ? idx : 0xFFFFFFFFu;
  const uint32_t prev = __shfl_up_sync(0xffffffffu, key, 1);
  const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
  if (__popc(heads) > 12) {  // many distinct entries: plain atomics
    if (valid) atomicAdd(base + idx, make_float2(vx, vy));
    return;
  }
  // inclusive segmented scan: lane accumulates lanes of its run below it
  const int seg_start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float ox = __shfl_up_sync(0xffffffffu, vx, d);
    const float oy = __shfl_up_sync(0xffffffffu, vy, d);
    if (lane - d >= seg_start) {
      vx += ox;
      vy += oy;
    }
  }
  const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
  if (valid && tail) atomicAdd(base + idx, make_float2(vx, vy));
}

template <typename TT>
__global__ void __launch_bounds__(256) k_hash_bwd(DevCam c, FieldDev f, int K, int KP,
                                                  long long n_rows, long long R,
                                                  const int* __restrict__ ids,
                                                  const float* __restrict__ depths,
                                                  const float2* __restrict__ gin,
                                                  float* __restrict__ dtl,
                                                  float* __restrict__ d_table) {
  // warp gw handles level gw % L for rows 32 (gw / L) .. + 31: the warps in
  // flight at any moment spread over all levels.  Within the warp, lanes are
  // slot-major (lane -> pixel lane % (32 / KP), slot lane / (32 / KP)), so
  // neighbouring lanes hold the same slot of neighbouring pixels, which at
  // coarse levels fall in the same cells.
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int l = (int)(gw % f.L);
  const int lane = threadIdx.x & 31, ppw = (32 % KP == 0) ? 32 / KP : 0;
  const long long r = (gw / f.L) * 32 + (ppw ? (lane % ppw) * KP + lane / ppw : lane);
  if ((gw / f.L) * 32 >= R) return;  // whole warps (R is a multiple of 32)
  const long long P = (long long)c.W * c.H;
  const long long p = r / KP;
  const int j = (int)(r % KP);
  bool valid = r < n_rows && p < P && j < K;
  const long long s = p * K + j;
  if (valid) valid = ids[s] >= 0;
  float D = 1.f;
  float3 d = make_float3(0.f, 0.f, 1.f), x = make_float3(0.f, 0.f, 0.f);
  float2 g = make_float2(0.f, 0.f);
  if (valid) {
    D = depths[s];
    d = pixel_dir(c, (int)(p % c.W), (int)(p / c.W));
    x = make_float3(c.o[0] + D * d.x, c.o[1] + D * d.y, c.o[2] + D * d.z);
    g = gin[(long long)l * R + r];
  }
  const size_t T = (size_t)f.mask + 1;
  const TT* tl = reinterpret_cast<const TT*>(f.table) + (size_t)l * T * 2;
  float2* dl = d_table ? reinterpret_cast<float2*>(d_table + (size_t)l * T * 2) : nullptr;
  const float sl = f.s[l];
  const float gx = sl * x.x, gy = sl * x.y, gz = sl * x.z;
  const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
  const int cx = (int)fx0, cy = (int)fy0, cz = (int)fz0;
  const float rx = gx - fx0, ry = gy - fy0, rz = gz - fz0;
  const float rr = f.focal / (sl * D);
  const float dw = downweight(f.focal, sl, D);
  float ax = 0.f, ay = 0.f, px = 0.f, py = 0.f, pz = 0.f;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
    const float wx = dx ? rx : 1.f - rx, wy = dy ? ry : 1.f - ry, wz = dz ? rz : 1.f - rz;
    const float sx = dx ? 1.f : -1.f, sy = dy ? 1.f : -1.f, sz = dz ? 1.f : -1.f;
    const uint32_t idx = hash3(cx + dx, cy + dy, cz + dz, f.mask);
    const float w = wx * wy * wz;
    if (valid) {
      const float2 e = load_entry<TT>(tl, idx);
      ax = fmaf(w, e.x, ax);
      ay = fmaf(w, e.y, ay);
      const float ge = g.x * e.x + g.y * e.y;
      px = fmaf(ge, sx * wy * wz, px);
      py = fmaf(ge, wx * sy * wz, py);
      pz = fmaf(ge, wx * wy * sz, pz);
    }
    if (dl) {
      const float sc = dw * w;
      run_atomic_add2(dl, idx, sc * g.x, sc * g.y, valid);
    }
  }
  // Delta = 1 - exp(-r^2 / 2pi), r = f / (s D): dDelta/dD = -(1 - Delta) r^2 / (pi D)
  const float ddw = -(1.f - dw) * rr * rr * 0.3183098861837907f / D;
  const float dt = (g.x * ax + g.y * ay) * ddw + dw * sl * (px * d.x + py * d.y + pz * d.z);
  if (r < n_rows) dtl[(long long)l * R + r] = valid ? dt : 0.f;
}

// dL/dD of each textured sample: the sum of its levels' shares.
__global__ void k_sum_levels(int L, int K, int KP, long long n_rows, long long R, long long P,
                             const int* __restrict__ ids, const float* __restrict__ dtl,
                             float* __restrict__ ddepth) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_rows) return;
  const long long p = r / KP;
  const int j = (int)(r % KP);
  if (p >= P || j >= K) return;
  const long long s = p * K + j;
  if (ids[s] < 0) return;
  float acc = 0.f;
  for (int l = 0; l < L; ++l) acc += dtl[(long long)l * R + r];
  ddepth[s] = acc;
}

cudaError_t launch_hash_bwd(const DevCam& c, const FieldDev& fd, int K, int KP, long long n_rows,
                            bool half_table, const int* ids, const float* depths,
                            const float2* gin, float* dtl, float* ddepth, float* d_table,
                            cudaStream_t st) {
  if (n_rows <= 0) return cudaSuccess;
  const long long R = gin_stride(n_rows);
  const long long threads = R * fd.L;
  const unsigned grid = (unsigned)((threads + 255) / 256);
  {
    NEXEL_PROF("hash_bwd", st);
    if (half_table)
      k_hash_bwd<__half><<<grid, 256, 0, st>>>(c, fd, K, KP, n_rows, R, ids, depths, gin, dtl,
                                               d_table);
    else
      k_hash_bwd<float><<<grid, 256, 0, st>>>(c, fd, K, KP, n_rows, R, ids, depths, gin, dtl,
                                              d_table);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  {
    NEXEL_PROF("sum_levels", st);
    k_sum_levels<<<(unsigned)((n_rows + 255) / 256), 256, 0, st>>>(
        fd.L, K, KP, n_rows, R, (long long)c.W * c.H, ids, dtl, ddepth);
  }
  return cudaGetLastError();
}

}  // namespace nexel
