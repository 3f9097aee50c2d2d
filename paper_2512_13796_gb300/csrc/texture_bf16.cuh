// BF16 tensor-core texturing pass: hash gather straight into MMA operand
// fragments, MLP layers chained in registers, composite in the epilogue.
//
// One warp owns a 16-row tile of samples (rows = (pixel, slot) pairs,
// pixel-major, KP = next power of two >= K rows per pixel).  With the
// m16n8k16 fragment layout, lane (g = lane / 4, t = lane % 4) holds rows g and
// g + 8 and, in K-tile kt, columns 16 kt + 2t (+1, +8, +9); because the
// features are level-major with F = 2, those columns are levels
// 8 kt + t and 8 kt + t + 4.  So every lane gathers 4 levels (IN = 32) of two
// samples and writes them into its A fragment directly, with no shared-memory
// staging.  An FP32 accumulator of layer l has exactly the A-fragment layout
// of layer l + 1 after ReLU and packing to BF16.  The input gradient of the
// backward comes out in the same column-to-lane map, so each lane scatters
// the table gradient of the very levels it gathered.
#pragma once

#include "common.cuh"
#include "texture_common.cuh"

namespace nexel {

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void* p) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x2_trans(uint32_t& r0, uint32_t& r1, const void* p) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n"
               : "=r"(r0), "=r"(r1)
               : "r"(a));
}

// Shared-memory weights, BF16, rows padded by 8 elements (16 bytes) so that
// the 8 rows a fragment load touches fall in distinct banks.
template <int IN, int H1, int H2>
struct Bf16W {
  static constexpr int HL = H2 > 0 ? H2 : H1;
  static constexpr int P = 8;
  // forward operands: W as stored, [out][in]
  static constexpr int s1 = IN + P, s2 = H1 + P, s3 = HL + P;
  static constexpr int o1 = 0, o2 = o1 + H1 * s1, o3 = o2 + (H2 > 0 ? H2 * s2 : 0);
  static constexpr int fwd_elems = o3 + 8 * s3;  // W3 padded to 8 output rows
  // backward operands: W^T, [in][out]
  static constexpr int t1 = H1 + P, t2 = (H2 > 0 ? H2 : 8) + P, t3 = 16 + P;
  static constexpr int p1 = fwd_elems, p2 = p1 + IN * t1, p3 = p2 + (H2 > 0 ? H1 * t2 : 0);
  static constexpr int all_elems = p3 + HL * t3;
};

// Loads FP32 weights (packed, [out][in] per layer) into the BF16 layout.
template <int IN, int H1, int H2>
__device__ void load_weights_bf16(const float* __restrict__ w, __nv_bfloat16* s, bool transposed) {
  using B = Bf16W<IN, H1, H2>;
  constexpr int HL = B::HL;
  const int n = transposed ? B::all_elems : B::fwd_elems;
  for (int k = threadIdx.x; k < n; k += blockDim.x) s[k] = __float2bfloat16(0.f);
  __syncthreads();
  const float* w1 = w;
  const float* w2 = w + IN * H1;
  const float* w3 = w + IN * H1 + (H2 > 0 ? H1 * H2 : 0);
  for (int k = threadIdx.x; k < H1 * IN; k += blockDim.x) {
    int o = k / IN, i = k % IN;
    __nv_bfloat16 v = __float2bfloat16(w1[k]);
    s[B::o1 + o * B::s1 + i] = v;
    if (transposed) s[B::p1 + i * B::t1 + o] = v;
  }
  if constexpr (H2 > 0) {
    for (int k = threadIdx.x; k < H2 * H1; k += blockDim.x) {
      int o = k / H1, i = k % H1;
      __nv_bfloat16 v = __float2bfloat16(w2[k]);
      s[B::o2 + o * B::s2 + i] = v;
      if (transposed) s[B::p2 + i * B::t2 + o] = v;
    }
  }
  for (int k = threadIdx.x; k < 3 * HL; k += blockDim.x) {
    int o = k / HL, i = k % HL;
    __nv_bfloat16 v = __float2bfloat16(w3[k]);
    s[B::o3 + o * B::s3 + i] = v;
    if (transposed) s[B::p3 + i * B::t3 + o] = v;
  }
  __syncthreads();
}

// B fragment (k = 16 kt + 2t.., n = 8 nt + g) of a row-major [n][k] matrix.
__device__ __forceinline__ void ldB(const __nv_bfloat16* m, int stride, int kt, int nt, int g,
                                    int t, uint32_t& b0, uint32_t& b1) {
  const __nv_bfloat16* r = m + (8 * nt + g) * stride + 16 * kt + 2 * t;
  b0 = *reinterpret_cast<const uint32_t*>(r);
  b1 = *reinterpret_cast<const uint32_t*>(r + 8);
}

// Dense layer: acc[nt] = A x B^T over K = KIN (A fragments per k-tile).
template <int KIN, int NOUT>
__device__ __forceinline__ void layer(const uint32_t (&a)[KIN / 16][4], const __nv_bfloat16* m,
                                      int stride, int g, int t, float (&acc)[NOUT / 8][4]) {
#pragma unroll
  for (int nt = 0; nt < NOUT / 8; ++nt) {
    acc[nt][0] = acc[nt][1] = acc[nt][2] = acc[nt][3] = 0.f;
#pragma unroll
    for (int kt = 0; kt < KIN / 16; ++kt) {
      uint32_t b0, b1;
      ldB(m, stride, kt, nt, g, t, b0, b1);
      mma16816(acc[nt], a[kt], b0, b1);
    }
  }
}

// ReLU + pack an accumulator [16 x N] into A fragments for the next layer.
template <int N>
__device__ __forceinline__ void relu_pack(const float (&acc)[N / 8][4], uint32_t (&a)[N / 16][4]) {
#pragma unroll
  for (int kt = 0; kt < N / 16; ++kt) {
    a[kt][0] = pack_bf16(fmaxf(acc[2 * kt][0], 0.f), fmaxf(acc[2 * kt][1], 0.f));
    a[kt][1] = pack_bf16(fmaxf(acc[2 * kt][2], 0.f), fmaxf(acc[2 * kt][3], 0.f));
    a[kt][2] = pack_bf16(fmaxf(acc[2 * kt + 1][0], 0.f), fmaxf(acc[2 * kt + 1][1], 0.f));
    a[kt][3] = pack_bf16(fmaxf(acc[2 * kt + 1][2], 0.f), fmaxf(acc[2 * kt + 1][3], 0.f));
  }
}

// Masked pack: keep g where the forward activation (packed BF16) is > 0.
__device__ __forceinline__ uint32_t mask_pack(float g0, float g1, uint32_t act) {
  __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&act);
  float m0 = __low2float(a) > 0.f ? g0 : 0.f;
  float m1 = __high2float(a) > 0.f ? g1 : 0.f;
  return pack_bf16(m0, m1);
}
template <int N>
__device__ __forceinline__ void mask_relu_pack(const float (&acc)[N / 8][4],
                                               const uint32_t (&act)[N / 16][4],
                                               uint32_t (&a)[N / 16][4]) {
#pragma unroll
  for (int kt = 0; kt < N / 16; ++kt) {
    a[kt][0] = mask_pack(acc[2 * kt][0], acc[2 * kt][1], act[kt][0]);
    a[kt][1] = mask_pack(acc[2 * kt][2], acc[2 * kt][3], act[kt][1]);
    a[kt][2] = mask_pack(acc[2 * kt + 1][0], acc[2 * kt + 1][1], act[kt][2]);
    a[kt][3] = mask_pack(acc[2 * kt + 1][2], acc[2 * kt + 1][3], act[kt][3]);
  }
}

// Hashed trilinear features of one (sample, level): returns (f0, f1) * Delta.
template <typename TT>
__device__ __forceinline__ float2 level_feature(const FieldDev& f, int l, float3 x, float t) {
  const TT* tl = reinterpret_cast<const TT*>(f.table) + (size_t)l * ((size_t)f.mask + 1) * 2;
  const float s = f.s[l];
  const float gx = s * x.x, gy = s * x.y, gz = s * x.z;
  const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
  const int cx = (int)fx0, cy = (int)fy0, cz = (int)fz0;
  const float rx = gx - fx0, ry = gy - fy0, rz = gz - fz0;
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
  return make_float2(dw * ax, dw * ay);
}


}  // namespace nexel
