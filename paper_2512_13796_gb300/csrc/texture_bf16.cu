// BF16 mma.sync form of the texturing backward for a step without cached
// features: input-gradient backward with a fresh gather (the hash-table
// scatter follows in hash_bwd.cu) and the MLP weight-gradient GEMMs.  The
// forward and the cached-feature backward run on tcgen05 (texture_tc.cu).
// FP32 accumulation everywhere; the table is read as FP16 or FP32.
#include "texture_bf16.cuh"

#include <type_traits>

namespace nexel {

constexpr int kWarps = 4;  // warps per CTA, one 16-row tile each

struct RowInfo {
  long long p;   // pixel
  long long s;   // sample index p * K + j
  bool valid;    // a textured sample (slot holds a surfel)
  bool in_pix;   // p < P and j < K (slot exists)
  float D, w;
  float3 x, d;
};

__device__ __forceinline__ RowInfo row_info(const DevCam& c, long long P, int K, int KP,
                                            long long r, const int* __restrict__ ids,
                                            const float* __restrict__ weights,
                                            const float* __restrict__ depths) {
  RowInfo ri;
  ri.p = r / KP;
  const int j = (int)(r % KP);
  ri.in_pix = ri.p < P && j < K;
  ri.s = ri.p * K + j;
  ri.valid = false;
  ri.D = 0.f;
  ri.w = 0.f;
  ri.x = ri.d = make_float3(0.f, 0.f, 0.f);
  if (ri.in_pix && ids[ri.s] >= 0) {
    ri.valid = true;
    ri.D = depths[ri.s];
    ri.w = weights[ri.s];
    ri.d = pixel_dir(c, (int)(ri.p % c.W), (int)(ri.p / c.W));
    ri.x = make_float3(c.o[0] + ri.D * ri.d.x, c.o[1] + ri.D * ri.d.y, c.o[2] + ri.D * ri.d.z);
  }
  return ri;
}

// Gathers the A fragments of the first layer for rows A (g) and B (g + 8).
template <int IN, typename TT>
__device__ __forceinline__ void gather_frags(const FieldDev& f, const RowInfo& A, const RowInfo& B,
                                             int t, uint32_t (&a)[IN / 16][4]) {
#pragma unroll
  for (int kt = 0; kt < IN / 16; ++kt) {
    const int l0 = 8 * kt + t, l1 = 8 * kt + t + 4;
    float2 fa0 = A.valid ? level_feature<TT>(f, l0, A.x, A.D) : make_float2(0.f, 0.f);
    float2 fb0 = B.valid ? level_feature<TT>(f, l0, B.x, B.D) : make_float2(0.f, 0.f);
    float2 fa1 = A.valid ? level_feature<TT>(f, l1, A.x, A.D) : make_float2(0.f, 0.f);
    float2 fb1 = B.valid ? level_feature<TT>(f, l1, B.x, B.D) : make_float2(0.f, 0.f);
    a[kt][0] = pack_bf16(fa0.x, fa0.y);
    a[kt][1] = pack_bf16(fb0.x, fb0.y);
    a[kt][2] = pack_bf16(fa1.x, fa1.y);
    a[kt][3] = pack_bf16(fb1.x, fb1.y);
  }
}

// Forward MLP from first-layer fragments; keeps hidden activations.
template <int IN, int H1, int H2>
__device__ __forceinline__ void mlp_fwd_bf16(const __nv_bfloat16* sw, int g, int t,
                                             const uint32_t (&a1)[IN / 16][4],
                                             uint32_t (&a2)[H1 / 16][4],
                                             uint32_t (&a3)[(H2 > 0 ? H2 : 16) / 16][4],
                                             float (&out)[1][4]) {
  using B = Bf16W<IN, H1, H2>;
  {
    float acc[H1 / 8][4];
    layer<IN, H1>(a1, sw + B::o1, B::s1, g, t, acc);
    relu_pack<H1>(acc, a2);
  }
  if constexpr (H2 > 0) {
    float acc[H2 / 8][4];
    layer<H1, H2>(a2, sw + B::o2, B::s2, g, t, acc);
    relu_pack<H2>(acc, a3);
    layer<H2, 8>(a3, sw + B::o3, B::s3, g, t, out);
  } else {
    layer<H1, 8>(a2, sw + B::o3, B::s3, g, t, out);
  }
}

// Backward, per 16-row tile: recompute (or read the cached features), input
// gradient through the MLP on tensor cores, dL/dW; saves the feature
// gradient (level-major, for hash_bwd.cu), the BF16 features and the FP32
// texture gradient (by row) for the weight-gradient kernel.
template <int IN, int H1, int H2, typename TT>
__global__ void __launch_bounds__(kWarps * 32) k_tex_bwd_bf16(
    DevCam c, FieldDev f, int K, int KP, long long n_tiles, const float* __restrict__ weights,
    const int* __restrict__ ids, const float* __restrict__ depths,
    const float* __restrict__ d_image, const float* __restrict__ d_weights,
    const float* __restrict__ d_textures, float* __restrict__ dweff, float* __restrict__ ddepth,
    uint32_t* __restrict__ feat_out, float4* __restrict__ gtex_out, float* __restrict__ gin_out) {
  using Bw = Bf16W<IN, H1, H2>;
  constexpr int HL = Bw::HL;
  extern __shared__ __align__(16) __nv_bfloat16 sw[];
  load_weights_bf16<IN, H1, H2>(f.w, sw, true);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const long long P = (long long)c.W * c.H;
  for (long long mt = (long long)blockIdx.x * kWarps + warp; mt < n_tiles;
       mt += (long long)gridDim.x * kWarps) {
    const long long rA = mt * 16 + g, rB = rA + 8;
    const RowInfo A = row_info(c, P, K, KP, rA, ids, weights, depths);
    const RowInfo B = row_info(c, P, K, KP, rB, ids, weights, depths);
    uint32_t a1[IN / 16][4];
    if (f.feat_mode == 2) {  // the forward of this step left the features
#pragma unroll
      for (int kt = 0; kt < IN / 16; ++kt) {
        a1[kt][0] = feat_out[(rA * IN + 16 * kt + 2 * t) / 2];
        a1[kt][1] = feat_out[(rB * IN + 16 * kt + 2 * t) / 2];
        a1[kt][2] = feat_out[(rA * IN + 16 * kt + 8 + 2 * t) / 2];
        a1[kt][3] = feat_out[(rB * IN + 16 * kt + 8 + 2 * t) / 2];
      }
    } else {
      gather_frags<IN, TT>(f, A, B, t, a1);
    }
    uint32_t a2[H1 / 16][4], a3[(H2 > 0 ? H2 : 16) / 16][4];
    float out[1][4];
    mlp_fwd_bf16<IN, H1, H2>(sw, g, t, a1, a2, a3, out);
    // texture gradient gT = W dC + dT (rows A, B; all three channels per lane)
    float gA[3] = {0.f, 0.f, 0.f}, gB[3] = {0.f, 0.f, 0.f}, dA[3] = {0.f, 0.f, 0.f},
          dB[3] = {0.f, 0.f, 0.f};
    if (A.valid) {
      for (int k = 0; k < 3; ++k) {
        dA[k] = d_image[3 * A.p + k];
        gA[k] = A.w * dA[k] + (d_textures ? d_textures[3 * A.s + k] : 0.f);
      }
    }
    if (B.valid) {
      for (int k = 0; k < 3; ++k) {
        dB[k] = d_image[3 * B.p + k];
        gB[k] = B.w * dB[k] + (d_textures ? d_textures[3 * B.s + k] : 0.f);
      }
    }
    // dL/dW_j = T_j . dC + dW_ext (reduce the channel partials over t)
    float pwA = 0.f, pwB = 0.f;
    if (t == 0) { pwA = out[0][0] * dA[0] + out[0][1] * dA[1]; pwB = out[0][2] * dB[0] + out[0][3] * dB[1]; }
    if (t == 1) { pwA = out[0][0] * dA[2]; pwB = out[0][2] * dB[2]; }
    pwA += __shfl_xor_sync(0xffffffffu, pwA, 1);
    pwA += __shfl_xor_sync(0xffffffffu, pwA, 2);
    pwB += __shfl_xor_sync(0xffffffffu, pwB, 1);
    pwB += __shfl_xor_sync(0xffffffffu, pwB, 2);
    // delta of the output layer as an A fragment [16 x 16], columns = channel
    uint32_t d3[1][4];
    d3[0][0] = t == 0 ? pack_bf16(gA[0], gA[1]) : (t == 1 ? pack_bf16(gA[2], 0.f) : 0u);
    d3[0][1] = t == 0 ? pack_bf16(gB[0], gB[1]) : (t == 1 ? pack_bf16(gB[2], 0.f) : 0u);
    d3[0][2] = 0u;
    d3[0][3] = 0u;
    uint32_t dl[HL / 16][4];
    {
      float acc[HL / 8][4];
      layer<16, HL>(d3, sw + Bw::p3, Bw::t3, g, t, acc);
      if constexpr (H2 > 0) mask_relu_pack<HL>(acc, a3, dl);
      else mask_relu_pack<HL>(acc, a2, dl);
    }
    float gin[IN / 8][4];
    if constexpr (H2 > 0) {
      uint32_t d1[H1 / 16][4];
      float acc[H1 / 8][4];
      layer<H2, H1>(dl, sw + Bw::p2, Bw::t2, g, t, acc);
      mask_relu_pack<H1>(acc, a2, d1);
      layer<H1, IN>(d1, sw + Bw::p1, Bw::t1, g, t, gin);
    } else {
      layer<H1, IN>(dl, sw + Bw::p1, Bw::t1, g, t, gin);
    }
    // feature gradient by row (FP32): n-tile nt holds columns 8 nt + 2t, +1;
    // the hash-grid backward (k_hash_bwd) scatters it and writes ddepth of
    // textured samples
    // level-major: level 4 nt + t of row r at gin_out[l * R + r]
    {
      float2* g2 = reinterpret_cast<float2*>(gin_out);
      const long long R = gin_stride(n_tiles * 16);
#pragma unroll
      for (int nt = 0; nt < IN / 8; ++nt) {
        const long long l = 4 * nt + t;
        g2[l * R + rA] = make_float2(gin[nt][0], gin[nt][1]);
        g2[l * R + rB] = make_float2(gin[nt][2], gin[nt][3]);
      }
    }
    if (t == 0) {
      if (A.in_pix) {
        if (!A.valid) ddepth[A.s] = 0.f;
        dweff[A.s] = A.valid ? pwA + (d_weights ? d_weights[A.s] : 0.f) : 0.f;
      }
      if (B.in_pix) {
        if (!B.valid) ddepth[B.s] = 0.f;
        dweff[B.s] = B.valid ? pwB + (d_weights ? d_weights[B.s] : 0.f) : 0.f;
      }
      gtex_out[rA] = make_float4(gA[0], gA[1], gA[2], 0.f);
      gtex_out[rB] = make_float4(gB[0], gB[1], gB[2], 0.f);
    }
    // features by row, BF16 pairs (for the weight-gradient kernel)
    if (f.feat_mode != 2) {
#pragma unroll
      for (int kt = 0; kt < IN / 16; ++kt) {
        feat_out[(rA * IN + 16 * kt + 2 * t) / 2] = a1[kt][0];
        feat_out[(rB * IN + 16 * kt + 2 * t) / 2] = a1[kt][1];
        feat_out[(rA * IN + 16 * kt + 8 + 2 * t) / 2] = a1[kt][2];
        feat_out[(rB * IN + 16 * kt + 8 + 2 * t) / 2] = a1[kt][3];
      }
    }
  }
}

// Weight gradients dW_l = sum over samples of delta_{l+1} a_l^T on tensor
// cores.  Per chunk of 64 rows every warp recomputes its 16 rows (forward
// and input-side deltas, all in fragments) and stores activations and deltas
// to shared memory; then each warp accumulates its share of the output tiles
// over the chunk's 64 samples (A = delta^T and B = a, both through
// ldmatrix.trans).  Accumulators stay in registers across chunks.
template <int IN, int H1, int H2>
struct WgSmem {
  static constexpr int HL = H2 > 0 ? H2 : H1;
  static constexpr int R = kWarps * 16;
  static constexpr int sa0 = IN + 8, sa1 = H1 + 8, sa2 = (H2 > 0 ? H2 : 8) + 8, sd3 = 16 + 8,
                       sdl = HL + 8, sd1 = H1 + 8;
  static constexpr int oa0 = Bf16W<IN, H1, H2>::all_elems;
  static constexpr int oa1 = oa0 + R * sa0;
  static constexpr int oa2 = oa1 + R * sa1;
  static constexpr int od3 = oa2 + (H2 > 0 ? R * sa2 : 0);
  static constexpr int odl = od3 + R * sd3;
  static constexpr int od1 = odl + R * sdl;
  static constexpr int total = od1 + (H2 > 0 ? R * sd1 : 0);
};

__device__ __forceinline__ void st_frag(__nv_bfloat16* base, int stride, int g, int t, int kt,
                                        const uint32_t (&a)[4]) {
  *reinterpret_cast<uint32_t*>(base + g * stride + 16 * kt + 2 * t) = a[0];
  *reinterpret_cast<uint32_t*>(base + (g + 8) * stride + 16 * kt + 2 * t) = a[1];
  *reinterpret_cast<uint32_t*>(base + g * stride + 16 * kt + 8 + 2 * t) = a[2];
  *reinterpret_cast<uint32_t*>(base + (g + 8) * stride + 16 * kt + 8 + 2 * t) = a[3];
}

// acc[mt][nt] += delta^T a over 64 rows for output rows [16 m0, ...), columns
// [8 n0, 8 n0 + 8 NT).
template <int NT>
__device__ __forceinline__ void wg_tile(const __nv_bfloat16* dsm, int dstride,
                                        const __nv_bfloat16* asm_, int astride, int m0, int n0,
                                        int lane, float (&acc)[NT][4]) {
#pragma unroll
  for (int ks = 0; ks < kWarps; ++ks) {
    const int s0 = 16 * ks;
    uint32_t a[4];
    {
      const int s = s0 + (lane & 7) + ((lane >> 4) << 3);
      const int o = 16 * m0 + ((lane >> 3) & 1) * 8;
      ldsm_x4_trans(a, dsm + s * dstride + o);
    }
#pragma unroll
    for (int nt = 0; nt < NT; nt += 2) {
      const int s = s0 + (lane & 15);
      if (nt + 1 < NT) {
        uint32_t b[4];
        const int i = 8 * (n0 + nt) + ((lane >> 4) << 3);
        ldsm_x4_trans(b, asm_ + s * astride + i);
        mma16816(acc[nt], a, b[0], b[1]);
        mma16816(acc[nt + 1], a, b[2], b[3]);
      } else {
        uint32_t b0, b1;
        ldsm_x2_trans(b0, b1, asm_ + s * astride + 8 * (n0 + nt));
        mma16816(acc[nt], a, b0, b1);
      }
    }
  }
}

template <int NT>
__device__ __forceinline__ void wg_flush(float* __restrict__ dW, int n_out, int n_in, int m0,
                                         int n0, int g, int t, const float (&acc)[NT][4]) {
#pragma unroll
  for (int nt = 0; nt < NT; ++nt) {
    const int i = 8 * (n0 + nt) + 2 * t;
    const int oA = 16 * m0 + g, oB = oA + 8;
    if (oA < n_out) {
      atomicAdd(dW + oA * n_in + i, acc[nt][0]);
      atomicAdd(dW + oA * n_in + i + 1, acc[nt][1]);
    }
    if (oB < n_out) {
      atomicAdd(dW + oB * n_in + i, acc[nt][2]);
      atomicAdd(dW + oB * n_in + i + 1, acc[nt][3]);
    }
  }
}

template <int IN, int H1, int H2>
__global__ void __launch_bounds__(kWarps * 32) k_mlp_wgrad_bf16(
    long long n_rows, const float* __restrict__ w, const uint32_t* __restrict__ feat,
    const float4* __restrict__ gtex, float* __restrict__ d_mlp) {
  using Bw = Bf16W<IN, H1, H2>;
  using S = WgSmem<IN, H1, H2>;
  constexpr int HL = Bw::HL;
  static_assert(H1 % 16 == 0 && HL % 16 == 0 && IN % 16 == 0, "BF16 MLP widths");
  extern __shared__ __align__(16) __nv_bfloat16 sm[];
  load_weights_bf16<IN, H1, H2>(w, sm, true);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  // output tiles owned by this warp
  constexpr int M1 = H1 / 16;                    // layer-1 rows (o) tiles
  constexpr int M2 = H2 > 0 ? H2 / 16 : 0;       // layer-2 rows tiles
  constexpr int NT1 = IN / 8, NT2 = H1 / 8;
  constexpr int NT3 = HL / 8 / kWarps > 0 ? HL / 8 / kWarps : 1;  // output layer columns per warp
  float acc1[(M1 + kWarps - 1) / kWarps][NT1][4];
  float acc2[M2 > 0 ? (M2 + kWarps - 1) / kWarps : 1][NT2][4];
  float acc3[NT3][4];
#pragma unroll
  for (int a = 0; a < (M1 + kWarps - 1) / kWarps; ++a)
#pragma unroll
    for (int b = 0; b < NT1; ++b) acc1[a][b][0] = acc1[a][b][1] = acc1[a][b][2] = acc1[a][b][3] = 0.f;
#pragma unroll
  for (int a = 0; a < (M2 > 0 ? (M2 + kWarps - 1) / kWarps : 1); ++a)
#pragma unroll
    for (int b = 0; b < NT2; ++b) acc2[a][b][0] = acc2[a][b][1] = acc2[a][b][2] = acc2[a][b][3] = 0.f;
#pragma unroll
  for (int b = 0; b < NT3; ++b) acc3[b][0] = acc3[b][1] = acc3[b][2] = acc3[b][3] = 0.f;
  __nv_bfloat16* sA0 = sm + S::oa0;
  __nv_bfloat16* sA1 = sm + S::oa1;
  __nv_bfloat16* sA2 = sm + S::oa2;
  __nv_bfloat16* sD3 = sm + S::od3;
  __nv_bfloat16* sDL = sm + S::odl;
  __nv_bfloat16* sD1 = sm + S::od1;
  const long long n_chunks = (n_rows + S::R - 1) / S::R;
  for (long long ch = blockIdx.x; ch < n_chunks; ch += gridDim.x) {
    const long long r0 = ch * S::R + warp * 16;
    const long long rA = r0 + g, rB = rA + 8;
    const bool vA = rA < n_rows, vB = rB < n_rows;
    uint32_t a1[IN / 16][4];
#pragma unroll
    for (int kt = 0; kt < IN / 16; ++kt) {
      a1[kt][0] = vA ? feat[(rA * IN + 16 * kt + 2 * t) / 2] : 0u;
      a1[kt][1] = vB ? feat[(rB * IN + 16 * kt + 2 * t) / 2] : 0u;
      a1[kt][2] = vA ? feat[(rA * IN + 16 * kt + 8 + 2 * t) / 2] : 0u;
      a1[kt][3] = vB ? feat[(rB * IN + 16 * kt + 8 + 2 * t) / 2] : 0u;
    }
    uint32_t a2[H1 / 16][4], a3[(H2 > 0 ? H2 : 16) / 16][4];
    float out[1][4];
    mlp_fwd_bf16<IN, H1, H2>(sm, g, t, a1, a2, a3, out);
    float4 gA4 = vA ? gtex[rA] : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 gB4 = vB ? gtex[rB] : make_float4(0.f, 0.f, 0.f, 0.f);
    uint32_t d3[1][4];
    d3[0][0] = t == 0 ? pack_bf16(gA4.x, gA4.y) : (t == 1 ? pack_bf16(gA4.z, 0.f) : 0u);
    d3[0][1] = t == 0 ? pack_bf16(gB4.x, gB4.y) : (t == 1 ? pack_bf16(gB4.z, 0.f) : 0u);
    d3[0][2] = 0u;
    d3[0][3] = 0u;
    uint32_t dl[HL / 16][4];
    {
      float acc[HL / 8][4];
      layer<16, HL>(d3, sm + Bw::p3, Bw::t3, g, t, acc);
      if constexpr (H2 > 0) mask_relu_pack<HL>(acc, a3, dl);
      else mask_relu_pack<HL>(acc, a2, dl);
    }
    __syncthreads();  // the previous chunk's tiles are consumed
    const int wr = warp * 16;
#pragma unroll
    for (int kt = 0; kt < IN / 16; ++kt) st_frag(sA0 + wr * S::sa0, S::sa0, g, t, kt, a1[kt]);
#pragma unroll
    for (int kt = 0; kt < H1 / 16; ++kt) st_frag(sA1 + wr * S::sa1, S::sa1, g, t, kt, a2[kt]);
    if constexpr (H2 > 0) {
#pragma unroll
      for (int kt = 0; kt < H2 / 16; ++kt) st_frag(sA2 + wr * S::sa2, S::sa2, g, t, kt, a3[kt]);
    }
    st_frag(sD3 + wr * S::sd3, S::sd3, g, t, 0, d3[0]);
#pragma unroll
    for (int kt = 0; kt < HL / 16; ++kt) st_frag(sDL + wr * S::sdl, S::sdl, g, t, kt, dl[kt]);
    if constexpr (H2 > 0) {
      uint32_t d1[H1 / 16][4];
      float acc[H1 / 8][4];
      layer<H2, H1>(dl, sm + Bw::p2, Bw::t2, g, t, acc);
      mask_relu_pack<H1>(acc, a2, d1);
#pragma unroll
      for (int kt = 0; kt < H1 / 16; ++kt) st_frag(sD1 + wr * S::sd1, S::sd1, g, t, kt, d1[kt]);
    }
    __syncthreads();
    // layer 1: dW1 [H1 x IN] = delta1^T a0
    const __nv_bfloat16* d1s = (H2 > 0) ? sD1 : sDL;
    const int d1stride = (H2 > 0) ? S::sd1 : S::sdl;
#pragma unroll
    for (int a = 0; a < (M1 + kWarps - 1) / kWarps; ++a) {
      const int m0 = warp + a * kWarps;
      if (m0 < M1) wg_tile<NT1>(d1s, d1stride, sA0, S::sa0, m0, 0, lane, acc1[a]);
    }
    if constexpr (H2 > 0) {
#pragma unroll
      for (int a = 0; a < (M2 + kWarps - 1) / kWarps; ++a) {
        const int m0 = warp + a * kWarps;
        if (m0 < M2) wg_tile<NT2>(sDL, S::sdl, sA1, S::sa1, m0, 0, lane, acc2[a]);
      }
    }
    // output layer: dW3 [3 x HL] = delta3^T aL, columns split over warps
    {
      const __nv_bfloat16* aL = (H2 > 0) ? sA2 : sA1;
      const int aLs = (H2 > 0) ? S::sa2 : S::sa1;
      const int n0 = warp * NT3;
      if (n0 < HL / 8) wg_tile<NT3>(sD3, S::sd3, aL, aLs, 0, n0, lane, acc3);
    }
  }
  float* dW1 = d_mlp;
  float* dW2 = d_mlp + IN * H1;
  float* dW3 = d_mlp + IN * H1 + (H2 > 0 ? H1 * H2 : 0);
#pragma unroll
  for (int a = 0; a < (M1 + kWarps - 1) / kWarps; ++a) {
    const int m0 = warp + a * kWarps;
    if (m0 < M1) wg_flush<NT1>(dW1, H1, IN, m0, 0, g, t, acc1[a]);
  }
  if constexpr (H2 > 0) {
#pragma unroll
    for (int a = 0; a < (M2 + kWarps - 1) / kWarps; ++a) {
      const int m0 = warp + a * kWarps;
      if (m0 < M2) wg_flush<NT2>(dW2, H2, H1, m0, 0, g, t, acc2[a]);
    }
  }
  {
    const int n0 = warp * NT3;
    if (n0 < HL / 8) wg_flush<NT3>(dW3, 3, HL, 0, n0, g, t, acc3);
  }
}

// ------------------------------------------------------------- dispatch
static int sm_count() {
  int dev = 0, n = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

template <int IN, int H1, int H2, typename TT>
static cudaError_t bwd_bf16(const DevCam& c, const nexel_settings& s, const FieldDev& fd,
                            char* bws, const BwdLayout& B, const float* weights, const int* ids,
                            const float* depths, const float* d_image, const float* d_weights,
                            const float* d_textures, float* d_table, float* d_mlp,
                            cudaStream_t st) {
  int KP = 1;
  while (KP < s.K) KP <<= 1;
  const long long rows = (long long)c.W * c.H * KP;
  const long long n_tiles = (rows + 15) / 16;
  if (fd.feat_mode == 2 && tc_arch_supported(IN, H1, H2)) {
    // the forward cached the features: MLP backward and weight gradients on
    // tcgen05, then the hash-grid backward
    cudaError_t e = launch_texture_bwd_tc(
        c, s.K, KP, n_tiles * 16, IN, H1, H2, fd.w, (const uint32_t*)(bws + B.feat), weights, ids,
        d_image, d_weights, d_textures, (float*)(bws + B.dweff), (float2*)(bws + B.gin), d_mlp,
        (int*)(bws + B.status), st);
    if (e != cudaSuccess) return e;
    return launch_hash_bwd(c, fd, s.K, KP, n_tiles * 16, std::is_same<TT, __half>::value, ids,
                           depths, (const float2*)(bws + B.gin), (float*)(bws + B.ddepth), d_table,
                           st);
  }
  const size_t smem = sizeof(__nv_bfloat16) * Bf16W<IN, H1, H2>::all_elems;
  auto kern = k_tex_bwd_bf16<IN, H1, H2, TT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int nsm = sm_count();
  const long long want = (n_tiles + kWarps - 1) / kWarps;
  unsigned grid = (unsigned)std::min<long long>(want, (long long)nsm * 16);
  {
  NEXEL_PROF("texture_bwd_bf16", st);
  kern<<<grid, kWarps * 32, smem, st>>>(c, fd, s.K, KP, n_tiles, weights, ids, depths, d_image,
                                        d_weights, d_textures, (float*)(bws + B.dweff),
                                        (float*)(bws + B.ddepth), (uint32_t*)(bws + B.feat),
                                        (float4*)(bws + B.gtex), (float*)(bws + B.gin));
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_hash_bwd(c, fd, s.K, KP, n_tiles * 16, std::is_same<TT, __half>::value, ids, depths,
                      (const float2*)(bws + B.gin), (float*)(bws + B.ddepth), d_table, st);
  if (e != cudaSuccess || !d_mlp) return e;
  const size_t smem2 = sizeof(__nv_bfloat16) * WgSmem<IN, H1, H2>::total;
  auto kw = k_mlp_wgrad_bf16<IN, H1, H2>;
  e = cudaFuncSetAttribute(kw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
  if (e != cudaSuccess) return e;
  const long long n_rows = n_tiles * 16;
  const long long chunks = (n_rows + WgSmem<IN, H1, H2>::R - 1) / WgSmem<IN, H1, H2>::R;
  grid = (unsigned)std::min<long long>(chunks, (long long)nsm * 4);
  NEXEL_PROF("mlp_wgrad_bf16", st);
  kw<<<grid, kWarps * 32, smem2, st>>>(n_rows, fd.w, (const uint32_t*)(bws + B.feat),
                                       (const float4*)(bws + B.gtex), d_mlp);
  return cudaGetLastError();
}

#define NEXEL_BF16_ARCHS(X) \
  X(16, 64, 0)              \
  X(32, 64, 64)

static bool match(const nexel_field& f, int in, int h1, int h2) {
  if (h2 == 0) return f.n_layers == 2 && f.widths[0] == in && f.widths[1] == h1 && f.widths[2] == 3;
  return f.n_layers == 3 && f.widths[0] == in && f.widths[1] == h1 && f.widths[2] == h2 &&
         f.widths[3] == 3;
}

bool bf16_arch_supported(const nexel_field& f) {
#define X(a, b, c) if (match(f, a, b, c)) return true;
  NEXEL_BF16_ARCHS(X)
#undef X
  return false;
}

cudaError_t launch_texture_bwd_bf16(const DevCam& c, const nexel_settings& s, const nexel_field& f,
                                    const FieldDev& fd, char* bws, const BwdLayout& B,
                                    const float* weights, const int* ids, const float* depths,
                                    const float* d_image, const float* d_weights,
                                    const float* d_textures, float* d_table, float* d_mlp,
                                    cudaStream_t st) {
  const bool h = s.grid_dtype == NEXEL_F16;
#define X(a, b, cc)                                                                             \
  if (match(f, a, b, cc))                                                                       \
    return h ? bwd_bf16<a, b, cc, __half>(c, s, fd, bws, B, weights, ids, depths, d_image,      \
                                          d_weights, d_textures, d_table, d_mlp, st)            \
             : bwd_bf16<a, b, cc, float>(c, s, fd, bws, B, weights, ids, depths, d_image,       \
                                         d_weights, d_textures, d_table, d_mlp, st);
  NEXEL_BF16_ARCHS(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace nexel
