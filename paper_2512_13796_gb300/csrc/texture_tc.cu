// Texture-MLP backward on the 5th-generation tensor cores (tcgen05, TMEM
// accumulators), for a training step whose forward cached the features:
// Sec. 4.2 / Eq. 4 backward through G (no bias, ReLU hidden layers, linear
// output) for every textured sample, and the MLP weight gradients summed
// over all samples.
//
// One CTA of 128 threads owns 128-row tiles (row = (pixel, slot) pair,
// pixel-major with KP rows per pixel; thread t = row t of the tile = TMEM
// lane t).  Per tile, four rounds of MMAs (M = 128, BF16 operands in shared
// memory, FP32 accumulators in TMEM), each followed by an epilogue in which
// every thread reads its row back (tcgen05.ld), applies ReLU or its mask and
// writes the next operand to shared memory:
//   R1  h1 = X W1^T                      (X = cached features)
//   R2  h2 = h1 W2^T                     (two hidden layers only)
//       T = h_last W3^T, dL/dW_j = T . dL/dC + dL/dW_j (upstream), d3 = the
//       texture gradient, d_last = (d3 W3) * [h_last > 0]   (CUDA cores)
//   R3  d1 = (d2 W2) * [h1 > 0]           (two hidden layers only)
//   R4  feature gradient X' = d1 W1 (to the hash-grid backward), and the
//       weight gradients, accumulated in TMEM over all tiles of the CTA:
//         Da += [h1 | h2]^T [d_last | d3]  -> dW2 (or dummy) and dW3 blocks
//         Db += [X | ...]^T d1             -> dW1 block
//       (the row-major activation tiles are read MN-major, K = rows, so no
//       transposed copies are made).
// SH textures (OUT = 48: the MLP's outputs are the degree-3 SH coefficients
// of the texture, evaluated in the pixel's ray direction, Sec. 3 / Sec. 5):
// the output layer is 48 MMA columns wide; with R1 one more MMA forms each
// row's effective output weights E = Y W3' (Y: the row's 16 SH basis values,
// W3 regrouped per channel), read back in place of W3 by the CUDA-core step;
// the delta tile's output block is Y_k gT_ch; the kernel then needs 512 TMEM
// columns and more shared memory, so it runs one CTA per SM.
// Shared-memory operands use the no-swizzle core-matrix layout (8 rows x
// 16 bytes per core matrix); a descriptor's leading byte offset is the
// stride between core matrices along K and its stride byte offset the stride
// along M/N, for K-major and MN-major operands alike.
#include "tc_common.cuh"

#include <algorithm>

namespace nexel {

namespace {

using namespace tcb;

// Features of levels l0 .. l0 + 3 at x (Eqs. 3-4): all 32 corner loads are
// issued before any is used.  The spatial hash of a corner is the XOR of
// per-axis parts (MapPositive, times the axis's prime), formed once per
// axis value; a row that is not textured reads the entries around the
// origin (valid addresses, harmless) and gets a zero down-weighting.
template <typename TT>
__device__ __forceinline__ void gather4_tc(const FieldDev& f, float focal, int l0, float3 x, float t,
                                           bool valid, float (&v)[8]) {
  using R = RawEntry<TT>;
  typename R::T e[4][8];
  float fr[4][3], dw[4];
  const TT* tab = reinterpret_cast<const TT*>(f.table);
  const uint32_t T2 = 2u * (f.mask + 1u);  // elements per level
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int l = l0 + q;
    const TT* tl = tab + (size_t)((uint32_t)l * T2);
    const float s = f.s[l];
    const float gx = s * x.x, gy = s * x.y, gz = s * x.z;
    const float fx0 = floorf(gx), fy0 = floorf(gy), fz0 = floorf(gz);
    const int cx = (int)fx0, cy = (int)fy0, cz = (int)fz0;
    fr[q][0] = gx - fx0; fr[q][1] = gy - fy0; fr[q][2] = gz - fz0;
    dw[q] = valid ? downweight(focal, s, t) : 0.f;
    const uint32_t hx0 = map_pos(cx), hx1 = map_pos(cx + 1);
    const uint32_t hy0 = map_pos(cy) * 2654435761u, hy1 = map_pos(cy + 1) * 2654435761u;
    const uint32_t hz0 = map_pos(cz) * 805459861u, hz1 = map_pos(cz + 1) * 805459861u;
    const uint32_t yz[4] = {hy0 ^ hz0, hy1 ^ hz0, hy0 ^ hz1, hy1 ^ hz1};
#pragma unroll
    for (int k = 0; k < 8; ++k)
      e[q][k] = R::load(tl, (((k & 1) ? hx1 : hx0) ^ yz[k >> 1]) & f.mask);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float rx = fr[q][0], ry = fr[q][1], rz = fr[q][2];
    const float wx[2] = {1.f - rx, rx};
    const float wyz[4] = {(1.f - ry) * (1.f - rz), ry * (1.f - rz), (1.f - ry) * rz, ry * rz};
    float ax = 0.f, ay = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const float w = wx[k & 1] * wyz[k >> 1];
      const float2 ee = R::to2(e[q][k]);
      ax = fmaf(w, ee.x, ax);
      ay = fmaf(w, ee.y, ay);
    }
    v[2 * q] = dw[q] * ax;
    v[2 * q + 1] = dw[q] * ay;
  }
}

// OUT = 3 (RGB texture, output layer padded to ON = 16 MMA columns) or 48
// (the texture's degree-3 SH coefficients, ON = 48).
template <int IN, int H1, int H2, int OUT = 3>
struct TcLayout {
  static constexpr int HL = H2 > 0 ? H2 : H1;
  static constexpr int ON = OUT == 3 ? 16 : 48;            // output-layer MMA columns
  static constexpr int FA = IN + H1 + H2;                  // activation features per row
  static constexpr int FD = HL + ON + (H2 > 0 ? H1 : 0);  // delta features per row
  static constexpr int SA = FA / 8 * 128, SD = FD / 8 * 128;
  static constexpr int D1 = H2 > 0 ? HL + ON : 0;         // first feature of d1 in the delta tile
  // bytes
  static constexpr int act = 0;
  static constexpr int act_bytes = kTcRows / 8 * SA + 2048;  // MN-major reads run up to 128 features
  static constexpr int del = act + act_bytes;
  static constexpr int del_bytes = kTcRows / 8 * SD + 2048;
  static constexpr int w1 = del + del_bytes;                 // [H1][IN]   K-major, B of R1
  static constexpr int w2 = w1 + H1 * IN * 2;                // [H2][H1]   B of R2
  static constexpr int w2t = w2 + H2 * H1 * 2;               // [H1][H2]   B of R3
  static constexpr int w1t = w2t + H2 * H1 * 2;              // [IN][H1]   B of the feature gradient
  static constexpr int w3 = w1t + IN * H1 * 2;               // FP32 [OUT][HL]
  // SH outputs: the rows' SH bases Y [128][16] (A of RE) and W3 regrouped
  // as [3 HL][16] (B of RE: row ch HL + i, column k = W3[3k + ch][i])
  static constexpr int ytile = w3 + OUT * HL * 4;
  static constexpr int w3p = ytile + (OUT == 48 ? kTcRows * 16 * 2 : 0);
  static constexpr int total = w3p + (OUT == 48 ? 3 * HL * 16 * 2 : 0);
  // TMEM columns: feature gradient / activations, then Da, then Db; SH
  // outputs add the rows' effective output weights E = Y W3' (3 HL columns)
  static constexpr int t_da = 64, t_db = 64 + HL + ON;
  static constexpr int t_e = 256;
  static constexpr int cols = OUT == 48 ? 512 : 256;
  static_assert(t_db + 64 <= 256, "TMEM columns");
  static_assert(OUT == 3 || t_e + 3 * HL <= cols, "TMEM columns of E");
  static_assert(IN % 16 == 0 && H1 == 64 && (H2 == 0 || H2 == 64), "supported MLP shapes");
  static_assert(HL + ON <= 256 && FA <= 256, "MMA N limits");
};

template <int IN, int H1, int H2, typename OP, int OUT, bool MV>
__global__ void __launch_bounds__(kTcThreads, 2) k_tex_bwd_tc(
    const __grid_constant__ ViewBatch<TexBwdView> b, int K, int log2KP,
    const float* __restrict__ wts, float* __restrict__ d_mlp, int fault) {
  using Lt = TcLayout<IN, H1, H2, OUT>;
  const long long n_tiles = b.item0[b.n];
  // fault > 0 (test hook only): no MMA is issued and each completion wait
  // gives up after `fault` polls, which exercises the timeout path
  const int wlim = fault > 0 ? fault : kTcWaitLimit;
  const bool issue = fault == 0;
  constexpr int HL = Lt::HL;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_bar;
  const int tid = threadIdx.x, warp = tid >> 5;
  unsigned char* act = tc_smem + Lt::act;
  unsigned char* del = tc_smem + Lt::del;
  float* w3s = reinterpret_cast<float*>(tc_smem + Lt::w3);

  // weights -> shared: BF16 K-major core-matrix tiles (B operands), W3 FP32
  {
    const float* W1 = wts;               // [H1][IN]
    const float* W2 = wts + H1 * IN;     // [H2][H1]
    const float* W3 = W2 + H2 * H1;      // [3][HL]
    for (int i = tid; i < H1 * IN; i += kTcThreads) {
      const int o = i / IN, k = i % IN;
      *reinterpret_cast<uint16_t*>(tc_smem + Lt::w1 + cm_off(o, k, IN / 8 * 128)) =
          OP::cvt(W1[i]);
      *reinterpret_cast<uint16_t*>(tc_smem + Lt::w1t + cm_off(k, o, H1 / 8 * 128)) =
          OP::cvt(W1[i]);
    }
    for (int i = tid; i < H2 * H1; i += kTcThreads) {
      const int o = i / H1, k = i % H1;
      *reinterpret_cast<uint16_t*>(tc_smem + Lt::w2 + cm_off(o, k, H1 / 8 * 128)) =
          OP::cvt(W2[i]);
      *reinterpret_cast<uint16_t*>(tc_smem + Lt::w2t + cm_off(k, o, (H2 > 0 ? H2 : 8) / 8 * 128)) =
          OP::cvt(W2[i]);
    }
    // the output layer as the forward's MMA reads it (rounded to the operand
    // type), so that the texture formed here for dL/dW_j is the forward's
    for (int i = tid; i < OUT * HL; i += kTcThreads) w3s[i] = OP::round(W3[i]);
    if constexpr (OUT == 48) {
      for (int i = tid; i < 3 * HL * 16; i += kTcThreads) {
        const int n = i / 16, k = i % 16, ch = n / HL, h = n % HL;
        *reinterpret_cast<uint16_t*>(tc_smem + Lt::w3p + cm_off(n, k, 256)) =
            OP::cvt(W3[(3 * k + ch) * HL + h]);
      }
    }
    // zero the delta tile once: the padding columns of d3 stay zero
    for (int i = tid; i < Lt::del_bytes / 16; i += kTcThreads)
      reinterpret_cast<uint4*>(del)[i] = make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_bar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(Lt::cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  sync_to_mma();
  const uint32_t tmem = s_tmem;
  const uint32_t t0 = tmem, t_da = tmem + Lt::t_da, t_db = tmem + Lt::t_db;  // columns
  const uint32_t t_e = tmem + Lt::t_e;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t sb = smem_u32(tc_smem);
  uint32_t phase = 0;
  bool ok = true;
  bool first = true;
  const int KP = 1 << log2KP;

  // per-row inputs of a tile; the next tile's are loaded while this one's
  // MMA rounds run
  struct RowIn {
    uint4 x[IN / 8];
    float w, dC[3], dT[3], dWx;
    long long s, r;  // sample and row within the tile's view
    int vi, id;      // the tile's view, the slot's surfel
    bool in_pix;
  };
  auto load_row = [&](long long tile, RowIn& in) {
    // MV: a batch of views (else one view, at a fixed index)
    in.vi = (MV && tile < n_tiles) ? view_of(b, (int)tile) : 0;
    const TexBwdView& V = b.v[in.vi];
    const long long n_rows = V.n_rows;
    const long long P = (long long)V.c.W * V.c.H;
    const float* __restrict__ weights = V.weights;
    const int* __restrict__ ids = V.ids;
    const float* __restrict__ d_image = V.d_image;
    const float* __restrict__ d_textures = V.d_textures;
    const float* __restrict__ d_weights = V.d_weights;
    const uint32_t* __restrict__ feat = V.feat;
    const long long r = (MV ? tile - b.item0[in.vi] : tile) * kTcRows + tid;
    in.r = r;
    const long long p = r >> log2KP;
    const int j = (int)(r & (KP - 1));
    in.s = p * K + j;
    in.in_pix = tile < n_tiles && r < n_rows && p < P && j < K;
    // every load of the row is issued at once and nothing here waits for
    // them: the values are first used when the tile is staged, a tile later
    in.id = -1;
    in.w = in.dWx = 0.f;
    in.dC[0] = in.dC[1] = in.dC[2] = 0.f;
    in.dT[0] = in.dT[1] = in.dT[2] = 0.f;
    if (in.in_pix) {
      in.id = ids[in.s];
      in.w = weights[in.s];
      in.dC[0] = d_image[3 * p]; in.dC[1] = d_image[3 * p + 1]; in.dC[2] = d_image[3 * p + 2];
      if (d_textures) {
        in.dT[0] = d_textures[3 * in.s]; in.dT[1] = d_textures[3 * in.s + 1];
        in.dT[2] = d_textures[3 * in.s + 2];
      }
      if (d_weights) in.dWx = d_weights[in.s];
    }
    // cached BF16 features of this row; zero beyond the pixels
#pragma unroll
    for (int c8 = 0; c8 < IN / 8; ++c8) {
      in.x[c8] = make_uint4(0u, 0u, 0u, 0u);
      if (tile < n_tiles && r < n_rows && p < P)
        in.x[c8] = reinterpret_cast<const uint4*>(feat + (size_t)r * (IN / 2))[c8];
    }
  };
  RowIn nxt;
  load_row(blockIdx.x, nxt);
  for (long long tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const RowIn cur = nxt;
    const TexBwdView& V = b.v[MV ? cur.vi : 0];
    const DevCam& c = V.c;
    const long long r = cur.r, n_rows = V.n_rows;
    const long long s = cur.s;
    // the row's texture gradient gT = w dL/dC + dL/dT (Eq. 6); nothing for
    // an empty slot or a row beyond the pixels
    const bool in_pix = cur.in_pix, valid = cur.in_pix && cur.id >= 0;
    const float gT[3] = {valid ? fmaf(cur.w, cur.dC[0], cur.dT[0]) : 0.f,
                         valid ? fmaf(cur.w, cur.dC[1], cur.dT[1]) : 0.f,
                         valid ? fmaf(cur.w, cur.dC[2], cur.dT[2]) : 0.f};
    const float dC[3] = {valid ? cur.dC[0] : 0.f, valid ? cur.dC[1] : 0.f, valid ? cur.dC[2] : 0.f};
    const float dWx = valid ? cur.dWx : 0.f;
    // stage X and d3
#pragma unroll
    for (int c8 = 0; c8 < IN / 8; ++c8)
      *reinterpret_cast<uint4*>(act + cm_off(tid, 8 * c8, Lt::SA)) = cur.x[c8];
    if constexpr (OUT == 3) {
      const float d3[8] = {OP::kScale * gT[0], OP::kScale * gT[1], OP::kScale * gT[2], 0.f, 0.f, 0.f, 0.f, 0.f};
      st8<OP>(del, tid, HL, Lt::SD, d3);
    } else {
      // output gradient of SH output 3k + ch: Y_k(ray) gT_ch; and the row's
      // SH basis, the A operand of RE
      const Sh3 Y = pixel_sh3(c, valid ? (r >> log2KP) : 0);
#pragma unroll
      for (int c8 = 0; c8 < 6; ++c8) {
        float d3[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int o = 8 * c8 + i;
          d3[i] = valid ? OP::kScale * Y.y[o / 3] * gT[o % 3] : 0.f;
        }
        st8<OP>(del, tid, HL + 8 * c8, Lt::SD, d3);
      }
      float yv[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) yv[k] = valid ? Y.y[k] : 0.f;
      st8<OP>(tc_smem + Lt::ytile, tid, 0, 256, yv);
      st8<OP>(tc_smem + Lt::ytile, tid, 8, 256, yv + 8);
    }
    sync_to_mma();
    // R1: h1 = X W1^T -> t0 (SH outputs: with RE, E = Y W3'^T -> t_e)
    if (tid == 0 && issue) {
#pragma unroll
      for (int kk = 0; kk < IN / 16; ++kk)
        mma(t0, dadv(sdesc(sb + Lt::act, 128, Lt::SA), kk * 256),
            dadv(sdesc(sb + Lt::w1, 128, IN / 8 * 128), kk * 256), idesc(128, H1, 0, 0, OP::kFmt),
            kk > 0);
      if constexpr (OUT == 48)
        mma(t_e, sdesc(sb + Lt::ytile, 128, 256), sdesc(sb + Lt::w3p, 128, 256),
            idesc(128, 3 * HL, 0, 0, OP::kFmt), false);
      commit(&s_bar);
    }
    load_row(tile + gridDim.x, nxt);
    ok = wait_bar(&s_bar, phase, wlim);
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    uint64_t m1 = 0, m2 = 0;  // ReLU masks of h1, h2
#pragma unroll
    for (int c16 = 0; c16 < H1 / 16; ++c16) {
      float v[16];
      tmem_ld16(t0 + lane_base + 16 * c16, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        if (v[i] > 0.f) m1 |= 1ull << (16 * c16 + i);
        v[i] = fmaxf(v[i], 0.f);
      }
      st8<OP>(act, tid, IN + 16 * c16, Lt::SA, v);
      st8<OP>(act, tid, IN + 16 * c16 + 8, Lt::SA, v + 8);
    }
    if constexpr (H2 > 0) {
      sync_to_mma();
      // R2: h2 = h1 W2^T -> t0
      if (tid == 0 && issue) {
#pragma unroll
        for (int kk = 0; kk < H1 / 16; ++kk)
          mma(t0, dadv(sdesc(sb + Lt::act, 128, Lt::SA), (IN / 8) * 128 + kk * 256),
              dadv(sdesc(sb + Lt::w2, 128, H1 / 8 * 128), kk * 256),
              idesc(128, H2, 0, 0, OP::kFmt), kk > 0);
        commit(&s_bar);
      }
      ok = ok && wait_bar(&s_bar, phase, wlim);
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c16 = 0; c16 < H2 / 16; ++c16) {
        float v[16];
        tmem_ld16(t0 + lane_base + 16 * c16, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (v[i] > 0.f) m2 |= 1ull << (16 * c16 + i);
          v[i] = fmaxf(v[i], 0.f);
        }
        st8<OP>(act, tid, IN + H1 + 16 * c16, Lt::SA, v);
        st8<OP>(act, tid, IN + H1 + 16 * c16 + 8, Lt::SA, v + 8);
      }
    }
    // texture T = W3 h_last, dL/dW_j, and d_last = (W3^T d3) * [h_last > 0]
    {
      const uint64_t ml = H2 > 0 ? m2 : m1;
      const float4* w34 = reinterpret_cast<const float4*>(w3s);
      float T0 = 0.f, T1 = 0.f, T2 = 0.f;
#pragma unroll
      for (int c8 = 0; c8 < HL / 8; ++c8) {
        // the (per-row, for SH) output-layer weights of hidden units 8 c8 ..
        float wr[3][8];
        if constexpr (OUT == 3) {
#pragma unroll
          for (int o = 0; o < 3; ++o) {
            const float4 a = w34[(o * HL + 8 * c8) / 4], b = w34[(o * HL + 8 * c8) / 4 + 1];
            wr[o][0] = a.x; wr[o][1] = a.y; wr[o][2] = a.z; wr[o][3] = a.w;
            wr[o][4] = b.x; wr[o][5] = b.y; wr[o][6] = b.z; wr[o][7] = b.w;
          }
        } else {
          // SH: T_ch = sum_k Y_k (W3 h)_{3k + ch}; the row's effective weight
          // of channel ch, sum_k Y_k W3[3k + ch], came from RE (TMEM
          // columns ch HL + i)
#pragma unroll
          for (int o = 0; o < 3; ++o) tmem_ld8(t_e + lane_base + o * HL + 8 * c8, wr[o]);
        }
        // the last hidden layer of this row, as stored (BF16)
        const uint4 hq = *reinterpret_cast<const uint4*>(act + cm_off(tid, IN + H1 + H2 - HL + 8 * c8, Lt::SA));
        const uint32_t hw[4] = {hq.x, hq.y, hq.z, hq.w};
        float hv[8];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 h2v = OP::unpack2(hw[i]);
          hv[2 * i] = h2v.x;
          hv[2 * i + 1] = h2v.y;
        }
        float v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int q = 8 * c8 + i;
          const float hlq = hv[i];
          T0 = fmaf(wr[0][i], hlq, T0);
          T1 = fmaf(wr[1][i], hlq, T1);
          T2 = fmaf(wr[2][i], hlq, T2);
          const float g = OP::kScale * fmaf(gT[0], wr[0][i], fmaf(gT[1], wr[1][i], gT[2] * wr[2][i]));
          v[i] = ((ml >> q) & 1ull) ? g : 0.f;
        }
        st8<OP>(del, tid, 8 * c8, Lt::SD, v);
      }
      if (in_pix) V.dweff[s] = valid ? T0 * dC[0] + T1 * dC[1] + T2 * dC[2] + dWx : 0.f;
    }
    if constexpr (H2 > 0) {
      sync_to_mma();
      // R3: d1 = (d2 W2) * [h1 > 0]; d2 is the delta tile's first H2 features
      if (tid == 0 && issue) {
#pragma unroll
        for (int kk = 0; kk < H2 / 16; ++kk)
          mma(t0, dadv(sdesc(sb + Lt::del, 128, Lt::SD), kk * 256),
              dadv(sdesc(sb + Lt::w2t, 128, H2 / 8 * 128), kk * 256),
              idesc(128, H1, 0, 0, OP::kFmt), kk > 0);
        commit(&s_bar);
      }
      ok = ok && wait_bar(&s_bar, phase, wlim);
      phase ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c16 = 0; c16 < H1 / 16; ++c16) {
        float v[16];
        tmem_ld16(t0 + lane_base + 16 * c16, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = ((m1 >> (16 * c16 + i)) & 1ull) ? v[i] : 0.f;
        st8<OP>(del, tid, Lt::D1 + 16 * c16, Lt::SD, v);
        st8<OP>(del, tid, Lt::D1 + 16 * c16 + 8, Lt::SD, v + 8);
      }
    }
    sync_to_mma();
    // R4: feature gradient d1 W1 -> t0; weight gradients into Da, Db
    if (tid == 0 && issue) {
#pragma unroll
      for (int kk = 0; kk < H1 / 16; ++kk)
        mma(t0, dadv(sdesc(sb + Lt::del, 128, Lt::SD), (Lt::D1 / 8) * 128 + kk * 256),
            dadv(sdesc(sb + Lt::w1t, 128, H1 / 8 * 128), kk * 256),
            idesc(128, IN, 0, 0, OP::kFmt), kk > 0);
      // K = rows: 16 rows = two 8-row groups per MMA
      const uint64_t aM = sdesc(sb + Lt::act, Lt::SA, 128), dM = sdesc(sb + Lt::del, Lt::SD, 128);
#pragma unroll 1
      for (int kk = 0; kk < kTcRows / 16; ++kk) {
        const bool acc = !(first && kk == 0);
        mma(t_da, dadv(aM, (IN / 8) * 128 + kk * 2 * Lt::SA), dadv(dM, kk * 2 * Lt::SD),
            idesc(128, HL + Lt::ON, 1, 1, OP::kFmt), acc);
        mma(t_db, dadv(aM, kk * 2 * Lt::SA), dadv(dM, (Lt::D1 / 8) * 128 + kk * 2 * Lt::SD),
            idesc(128, H1, 1, 1, OP::kFmt), acc);
      }
      commit(&s_bar);
    }
    ok = ok && wait_bar(&s_bar, phase, wlim);
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    first = false;
    {
      // feature gradient, level-major float2 per level
      const long long R = gin_stride(n_rows);
#pragma unroll
      for (int c16 = 0; c16 < IN / 16; ++c16) {
        float v[16];
        tmem_ld16(t0 + lane_base + 16 * c16, v);
        if (r < n_rows) {
#pragma unroll
          for (int i = 0; i < 8; ++i)  // streamed to the hash backward: evict-first
            __stcs(V.gin + (long long)(8 * c16 + i) * R + r,
                   make_float2(v[2 * i] * (1.f / OP::kScale), v[2 * i + 1] * (1.f / OP::kScale)));
        }
      }
    }
    // the next tile's staging overwrites the operand tiles: the MMAs that
    // read them have completed (the wait above).  A wait that ran out on any
    // thread ends the loop for the whole CTA.
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    ok = __syncthreads_and(ok) != 0;
  }
  // weight gradients of this CTA: Da lane m = activation feature IN + m,
  // column n = delta feature n; Db lane m = activation feature m, column
  // n = d1 feature n
  if (!first && ok && d_mlp) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float* dW1 = d_mlp;
    float* dW2 = d_mlp + H1 * IN;
    float* dW3 = dW2 + H2 * H1;
    for (int c16 = 0; c16 < (HL + Lt::ON) / 16; ++c16) {
      float v[16];
      tmem_ld16(t_da + lane_base + 16 * c16, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int n = 16 * c16 + i, m = tid;
        if (H2 > 0) {
          if (m < H1 && n < H2) atomicAdd(dW2 + n * H1 + m, v[i] * (1.f / OP::kScale));  // dW2[o=n][i=m]
          if (m >= H1 && m < H1 + H2 && n >= HL && n < HL + OUT)
            atomicAdd(dW3 + (n - HL) * HL + (m - H1), v[i] * (1.f / OP::kScale));         // dW3[o][i]
        } else {
          if (m < H1 && n >= HL && n < HL + OUT)
            atomicAdd(dW3 + (n - HL) * HL + m, v[i] * (1.f / OP::kScale));
        }
      }
    }
    for (int c16 = 0; c16 < H1 / 16; ++c16) {
      float v[16];
      tmem_ld16(t_db + lane_base + 16 * c16, v);
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (tid < IN) atomicAdd(dW1 + (16 * c16 + i) * IN + tid, v[i] * (1.f / OP::kScale));  // dW1[o][i]
    }
  }
  if (!ok && tid == 0)  // a wait that ran out marks every view of the launch
    for (int v = 0; v < b.n; ++v)
      if (b.v[v].status) atomicOr(b.v[v].status, kStatusTimeout);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Lt::cols));
}

template <int IN, int H1, int H2, typename OP, int OUT = 3>
cudaError_t tex_bwd_tc(int K, int KP, const float* w, const ViewBatch<TexBwdView>& b, float* d_mlp,
                       cudaStream_t st) {
  using Lt = TcLayout<IN, H1, H2, OUT>;
  int log2KP = 0;
  while ((1 << log2KP) < KP) ++log2KP;
  const long long n_tiles = b.item0[b.n];
  if (n_tiles == 0) return cudaSuccess;
  auto kern = b.n > 1 ? k_tex_bwd_tc<IN, H1, H2, OP, OUT, true> : k_tex_bwd_tc<IN, H1, H2, OP, OUT, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Lt::total);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // two CTAs per SM where their shared memory fits (227 KB per SM)
  const long long per_sm = std::min<long long>(
      current_tuning().tex_bwd_ctas, 2LL * (Lt::total + 1024) <= 227LL * 1024 ? 2 : 1);
  const unsigned grid = (unsigned)std::min<long long>(n_tiles, per_sm * nsm);
  NEXEL_PROF("texture_bwd_tc", st);
  kern<<<grid, kTcThreads, Lt::total, st>>>(b, K, log2KP, w, d_mlp, tc_wait_fault());
  return cudaGetLastError();
}

// ------------------------------------------------------------- forward
// Texturing forward on tcgen05 (Eqs. 3-4 and the composite of Eq. 6), warp
// specialised.  A CTA of 12 warps walks a sequence of 128-row tiles (128 / KP
// pixels x KP slots):
//   warps 0-7 gather: thread t handles half t / 128 of the levels of one row;
//     within a warp the lanes are consecutive pixels of one slot, so at
//     coarse levels neighbouring lanes read the same table entries.  The
//     down-weighted features go, as the A operand, into a ring of kFwStages
//     shared-memory stages (2..kFwStages in use, a tuning knob; and, in a
//     training step, to the feature cache).
//     A stage is handed to the MLP warps through an mbarrier (`full`) and
//     handed back by the completion of the MMA that reads it (`empty`, a
//     tcgen05 commit), so the gather runs up to kFwStages tiles ahead and
//     never waits for the MLP's round trips.
//   warps 8-11 MLP: warp 8 + q owns TMEM lanes 32 q .. 32 q + 31 (= rows); one
//     thread issues X W1^T, h1 W2^T and h_last W3^T with FP32 accumulators in
//     TMEM; the four warps run the ReLU epilogues (TMEM -> the hidden tile in
//     shared memory, h2 overwriting h1) and the last epilogue writes the
//     textures and the composite.
// Every mbarrier wait is bounded: a wait that runs out sets the status word
// and ends the CTA's loops (the TMEM is freed before the kernel returns).
constexpr int kFwGatherWarps = 8;
constexpr int kFwThreads = (kFwGatherWarps + 4) * 32;
constexpr int kFwStages = 4;
constexpr int kTcFwdCols = 128;

template <int IN, int H1, int H2, int OUT = 3>
struct TcFwdLayout {
  static constexpr int HL = H2 > 0 ? H2 : H1;
  static constexpr int ON = OUT == 3 ? 16 : 48;  // output-layer MMA columns
  static constexpr int HM = H1 > H2 ? H1 : H2;   // hidden-tile features
  static constexpr int SX = IN / 8 * 128;        // bytes per 8-row group of a stage
  static constexpr int SHd = HM / 8 * 128;       // ... of the hidden tile
  static constexpr int xstage = kTcRows / 8 * SX;
  static constexpr int xring = 0;
  static constexpr int hid = xring + kFwStages * xstage;
  static constexpr int w1 = hid + kTcRows / 8 * SHd;  // [H1][IN]
  static constexpr int w2 = w1 + H1 * IN * 2;         // [H2][H1]
  static constexpr int w3 = w2 + H2 * H1 * 2;         // [ON][HL], rows OUT.. zero
  static constexpr int total = w3 + ON * HL * 2;
  static_assert(ON <= 64, "the output layer uses TMEM columns 64 .. 127");
  static_assert(HM == 64, "hidden layers of 64 units");
};

// Consumer-group (the four MLP warps) hand-over to the MMA-issuing thread:
// their shared-memory stores and TMEM reads happen before the MMAs issued
// next.
__device__ __forceinline__ void mlp_warps_sync() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  asm volatile("bar.sync 1, 128;" ::: "memory");
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// AND of `v` over the four MLP warps (a named-barrier reduction).
__device__ __forceinline__ bool mlp_warps_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, 1, 128, p;\n"
      "selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}

__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}


template <int IN, int H1, int H2, typename TT, typename OP, int OUT, bool MV>
__global__ void __launch_bounds__(kFwThreads, 2) k_tex_fwd_tc(
    const __grid_constant__ ViewBatch<TexFwdView> b, FieldDev f, int K, int log2KP, float bg0,
    float bg1, float bg2, int fault, int ns) {
  const long long n_tiles = b.item0[b.n];
  using Lt = TcFwdLayout<IN, H1, H2, OUT>;
  constexpr int HL = Lt::HL;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_full[kFwStages];
  __shared__ __align__(8) uint64_t s_empty[kFwStages];
  __shared__ __align__(8) uint64_t s_mma;
  // fault > 0 (test hook only): no MMA is issued and each completion wait
  // gives up after `fault` polls, which exercises the timeout path
  const int wlim = fault > 0 ? fault : kTcWaitLimit;
  const bool issue = fault == 0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  {
    const float* W1 = f.w;
    const float* W2 = f.w + H1 * IN;
    const float* W3 = W2 + H2 * H1;
    for (int i = tid; i < H1 * IN; i += kFwThreads)
      *reinterpret_cast<uint16_t*>(tc_smem + Lt::w1 + cm_off(i / IN, i % IN, IN / 8 * 128)) =
          OP::cvt(W1[i]);
    for (int i = tid; i < H2 * H1; i += kFwThreads)
      *reinterpret_cast<uint16_t*>(tc_smem + Lt::w2 + cm_off(i / H1, i % H1, H1 / 8 * 128)) =
          OP::cvt(W2[i]);
    for (int i = tid; i < Lt::ON * HL; i += kFwThreads) {
      const int o = i / HL, k = i % HL;
      *reinterpret_cast<uint16_t*>(tc_smem + Lt::w3 + cm_off(o, k, HL / 8 * 128)) =
          OP::cvt(o < OUT ? W3[o * HL + k] : 0.f);
    }
  }
  if (tid == 0) {
    for (int s = 0; s < kFwStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&s_full[s])),
                   "r"(kFwGatherWarps * 32));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_empty[s])));
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_mma)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kFwGatherWarps) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(kTcFwdCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  sync_to_mma();
  const uint32_t tmem = s_tmem;
  const uint32_t t0 = tmem, t1 = tmem + 64;
  const uint32_t sb = smem_u32(tc_smem);
  const int KP = 1 << log2KP, PPT = kTcRows >> log2KP;
  // a wait that ran out marks every view of the launch
  auto mark_timeout = [&]() {
    for (int v = 0; v < b.n; ++v)
      if (b.v[v].status) atomicOr(b.v[v].status, kStatusTimeout);
  };

  if (warp < kFwGatherWarps) {
    // ------------------------------------------------------- gather warps
    const int tt = tid & (kTcRows - 1), gh = tid >> 7;
    const int grow = (tt % PPT) * KP + tt / PPT;
    int i = 0;
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
      const int st = i % ns, use = i / ns;  // ns <= kFwStages stages in use
      // the MMA that read this stage kFwStages tiles ago has completed
      if (use > 0 && !wait_bar(&s_empty[st], (uint32_t)((use - 1) & 1), wlim)) {
        if (tid == 0) mark_timeout();
        break;
      }
      unsigned char* xs = tc_smem + Lt::xring + st * Lt::xstage;
      const int vi = MV ? view_of(b, (int)tile) : 0;  // MV: a batch of views
      const TexFwdView& V = b.v[vi];
      const DevCam& c = V.c;
      const long long lt = MV ? tile - b.item0[vi] : tile;  // the view's own tile index
      const long long P = (long long)c.W * c.H;
      const long long p = lt * PPT + tt % PPT;
      const int j = tt / PPT;
      const bool in_pix = p < P && j < K;
      const long long s = p * K + j;
      const bool valid = in_pix && V.ids[s] >= 0;
      float3 x = make_float3(0.f, 0.f, 0.f);
      float D = 1.f;
      if (valid) {
        D = V.depths[s];
        const float3 d = pixel_dir(c, (int)(p % c.W), (int)(p / c.W));
        x = make_float3(c.o[0] + D * d.x, c.o[1] + D * d.y, c.o[2] + D * d.z);
      }
      constexpr int LH = IN / 4;  // levels per half (F = 2)
#pragma unroll
      for (int g8 = 0; g8 < LH / 4; ++g8) {  // 4 levels = 8 features per store
        float v[8];
        gather4_tc<TT>(f, c.fx, gh * LH + 4 * g8, x, D, valid, v);
        const int f0 = gh * (IN / 2) + 8 * g8;
        const uint4 q4 = pack8<OP>(v);
        *reinterpret_cast<uint4*>(xs + cm_off(grow, f0, Lt::SX)) = q4;
        if (V.feat_cache && p < P)
          reinterpret_cast<uint4*>(V.feat_cache + (size_t)(lt * kTcRows + grow) * (IN / 2))[f0 / 8] = q4;
      }
      // the stage's generic stores become visible to the MMA (async proxy)
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bar_arrive(&s_full[st]);
    }
    return;
  }

  // ---------------------------------------------------------- MLP warps
  const int q = warp - kFwGatherWarps;  // TMEM lane quadrant (= warp % 4)
  const int erow = 32 * q + lane;
  const uint32_t elane = (uint32_t)(32 * q) << 16;
  const bool leader = tid == kFwGatherWarps * 32;
  uint32_t mph = 0;
  bool ok = true;
  int i = 0;
  unsigned char* hid = tc_smem + Lt::hid;
  // Completion of the MMAs just issued: the issuing thread polls the
  // mbarrier, a named-barrier reduction releases the other MLP threads (who
  // sleep instead of polling) and tells them whether the wait ran out.
  auto mma_done = [&]() -> bool {
    bool got = true;
    if (leader) got = ok && wait_bar(&s_mma, mph, wlim);
    mph ^= 1u;
    got = mlp_warps_and(got);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return got;
  };
  for (long long tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++i) {
    const int st = i % ns, use = i / ns;  // ns <= kFwStages stages in use
    const int vi = MV ? view_of(b, (int)tile) : 0;
    const TexFwdView& V = b.v[vi];
    const DevCam& c = V.c;
    const long long P = (long long)c.W * c.H;
    // this row's composite inputs, fetched before the MMA waits
    const long long p = (MV ? tile - b.item0[vi] : tile) * PPT + erow / KP;
    const int j = erow & (KP - 1);
    const bool in_pix = p < P && j < K;
    const long long s = p * K + j;
    int id = -1;
    float wj = 0.f, n0 = 0.f, n1 = 0.f, n2 = 0.f, Tf = 0.f;
    if (in_pix) {
      id = V.ids[s];
      wj = V.weights[s];
    }
    if (j == 0 && p < P) {
      n0 = V.notex[3 * p]; n1 = V.notex[3 * p + 1]; n2 = V.notex[3 * p + 2];
      Tf = V.T_final[p];
    }
    // R1: h1 = X W1^T -> t0; its completion also frees the stage
    if (leader) {
      const bool got = wait_bar(&s_full[st], (uint32_t)(use & 1), wlim);
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (got && issue) {
        const uint32_t xa = sb + Lt::xring + st * Lt::xstage;
#pragma unroll
        for (int kk = 0; kk < IN / 16; ++kk)
          mma(t0, sdesc(xa + kk * 256, 128, Lt::SX), sdesc(sb + Lt::w1 + kk * 256, 128, IN / 8 * 128),
              idesc(128, H1, 0, 0, OP::kFmt), kk > 0);
        commit(&s_mma);
        commit(&s_empty[st]);
      }
    }
    ok = mma_done();
#pragma unroll
    for (int c32 = 0; c32 < H1 / 32; ++c32) {
      float v[32];
      tmem_ld32(t0 + elane + 32 * c32, v);
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = fmaxf(v[k], 0.f);
#pragma unroll
      for (int k8 = 0; k8 < 4; ++k8)
        *reinterpret_cast<uint4*>(hid + cm_off(erow, 32 * c32 + 8 * k8, Lt::SHd)) = pack8<OP>(v + 8 * k8);
    }
    mlp_warps_sync();
    if constexpr (H2 > 0) {
      // R2: h2 = h1 W2^T -> t0 (h2 then overwrites h1 in the hidden tile)
      if (leader && ok && issue) {
#pragma unroll
        for (int kk = 0; kk < H1 / 16; ++kk)
          mma(t0, sdesc(sb + Lt::hid + kk * 256, 128, Lt::SHd),
              sdesc(sb + Lt::w2 + kk * 256, 128, H1 / 8 * 128), idesc(128, H2, 0, 0, OP::kFmt), kk > 0);
        commit(&s_mma);
      }
      ok = mma_done() && ok;
#pragma unroll
      for (int c32 = 0; c32 < H2 / 32; ++c32) {
        float v[32];
        tmem_ld32(t0 + elane + 32 * c32, v);
#pragma unroll
        for (int k = 0; k < 32; ++k) v[k] = fmaxf(v[k], 0.f);
#pragma unroll
        for (int k8 = 0; k8 < 4; ++k8)
          *reinterpret_cast<uint4*>(hid + cm_off(erow, 32 * c32 + 8 * k8, Lt::SHd)) = pack8<OP>(v + 8 * k8);
      }
      mlp_warps_sync();
    }
    // R3: outputs h_last W3^T -> t1
    if (leader && ok && issue) {
#pragma unroll
      for (int kk = 0; kk < HL / 16; ++kk)
        mma(t1, sdesc(sb + Lt::hid + kk * 256, 128, Lt::SHd),
            sdesc(sb + Lt::w3 + kk * 256, 128, HL / 8 * 128), idesc(128, Lt::ON, 0, 0, OP::kFmt), kk > 0);
      commit(&s_mma);
    }
    ok = mma_done() && ok;
    {
      float o3[3];
      if constexpr (OUT == 3) {
        float v[16];
        tmem_ld16(t1 + elane, v);
        o3[0] = v[0]; o3[1] = v[1]; o3[2] = v[2];
      } else {
        // SH coefficients o[3k + ch], evaluated in the ray direction
        const Sh3 Y = pixel_sh3(c, in_pix ? p : 0);
        o3[0] = o3[1] = o3[2] = 0.f;
#pragma unroll
        for (int c16 = 0; c16 < 3; ++c16) {
          float v[16];
          tmem_ld16(t1 + elane + 16 * c16, v);
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int o = 16 * c16 + k;
            o3[o % 3] = fmaf(Y.y[o / 3], v[k], o3[o % 3]);
          }
        }
      }
      float T0 = 0.f, T1 = 0.f, T2 = 0.f;
      if (in_pix) {
        if (id >= 0) {
          T0 = o3[0]; T1 = o3[1]; T2 = o3[2];
        } else {
          wj = 0.f;
        }
        V.textures[3 * s] = T0; V.textures[3 * s + 1] = T1; V.textures[3 * s + 2] = T2;
      }
      float c0 = wj * T0, c1 = wj * T1, c2 = wj * T2;
      for (int dd = 1; dd < KP; dd <<= 1) {
        c0 += __shfl_xor_sync(0xffffffffu, c0, dd);
        c1 += __shfl_xor_sync(0xffffffffu, c1, dd);
        c2 += __shfl_xor_sync(0xffffffffu, c2, dd);
      }
      if (j == 0 && p < P) {
        V.image[3 * p] = n0 + c0 + Tf * bg0;
        V.image[3 * p + 1] = n1 + c1 + Tf * bg1;
        V.image[3 * p + 2] = n2 + c2 + Tf * bg2;
      }
    }
    // a wait that ran out on any MLP thread ends the loop for all four warps
    ok = mlp_warps_and(ok);
  }
  if (!ok && q == 0 && lane == 0) mark_timeout();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  asm volatile("bar.sync 1, 128;" ::: "memory");
  if (warp == kFwGatherWarps)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcFwdCols));
}

template <int IN, int H1, int H2, typename TT, typename OP, int OUT = 3>
cudaError_t tex_fwd_tc(const nexel_settings& s, const FieldDev& fd, const ViewBatch<TexFwdView>& b,
                       cudaStream_t st) {
  using Lt = TcFwdLayout<IN, H1, H2, OUT>;
  int log2KP = 0;
  while ((1 << log2KP) < s.K) ++log2KP;
  const long long n_tiles = b.item0[b.n];
  if (n_tiles == 0) return cudaSuccess;
  auto kern = b.n > 1 ? k_tex_fwd_tc<IN, H1, H2, TT, OP, OUT, true>
                      : k_tex_fwd_tc<IN, H1, H2, TT, OP, OUT, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Lt::total);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid =
      (unsigned)std::min<long long>(n_tiles, (long long)current_tuning().tex_fwd_ctas * nsm);
  NEXEL_PROF("texture_fwd_tc", st);
  kern<<<grid, kFwThreads, Lt::total, st>>>(
      b, fd, s.K, log2KP, s.bg[0], s.bg[1], s.bg[2], tc_wait_fault(),
      std::min(std::max(current_tuning().tex_fwd_stages, 2), kFwStages));
  return cudaGetLastError();
}

constexpr int kGatherThreads = 256;

// Feature pass of a backward without cached features: the gather of the
// forward (same lane layout and arithmetic), written to the feature buffer.
template <int IN, typename TT, typename OP>
__global__ void __launch_bounds__(kGatherThreads) k_gather_tc(DevCam c, FieldDev f, int K, int log2KP,
                                                           long long n_tiles, const int* __restrict__ ids,
                                                           const float* __restrict__ depths,
                                                           uint32_t* __restrict__ feat) {
  const long long tile = blockIdx.x;
  const int tid = threadIdx.x, tt = tid & (kTcRows - 1), gh = tid >> 7;
  const int KP = 1 << log2KP, PPT = kTcRows >> log2KP;
  const long long P = (long long)c.W * c.H;
  const long long p = tile * PPT + tt % PPT;
  const int j = tt / PPT;
  if (tile >= n_tiles || p >= P) return;
  const long long s = p * K + j;
  const bool valid = j < K && ids[s] >= 0;
  float3 x = make_float3(0.f, 0.f, 0.f);
  float D = 1.f;
  if (valid) {
    D = depths[s];
    const float3 d = pixel_dir(c, (int)(p % c.W), (int)(p / c.W));
    x = make_float3(c.o[0] + D * d.x, c.o[1] + D * d.y, c.o[2] + D * d.z);
  }
  const size_t row = (size_t)p * KP + j;
  constexpr int LH = IN / 4;
#pragma unroll
  for (int g8 = 0; g8 < LH / 4; ++g8) {
    float v[8];
    gather4_tc<TT>(f, f.focal, gh * LH + 4 * g8, x, D, valid, v);
    const int f0 = gh * (IN / 2) + 8 * g8;
    reinterpret_cast<uint4*>(feat + row * (IN / 2))[f0 / 8] =
        make_uint4(OP::pack2(v[0], v[1]), OP::pack2(v[2], v[3]), OP::pack2(v[4], v[5]),
                   OP::pack2(v[6], v[7]));
  }
}

template <int IN, typename TT, typename OP>
cudaError_t gather_tc(const DevCam& c, const nexel_settings& s, const FieldDev& fd, const int* ids,
                      const float* depths, uint32_t* feat, cudaStream_t st) {
  int log2KP = 0;
  while ((1 << log2KP) < s.K) ++log2KP;
  const long long rows = (long long)c.W * c.H << log2KP;
  const long long n_tiles = (rows + kTcRows - 1) / kTcRows;
  if (n_tiles == 0) return cudaSuccess;
  NEXEL_PROF("texture_gather_tc", st);
  k_gather_tc<IN, TT, OP><<<(unsigned)n_tiles, kGatherThreads, 0, st>>>(c, fd, s.K, log2KP, n_tiles,
                                                                      ids, depths, feat);
  return cudaGetLastError();
}

}  // namespace

bool tc_arch_supported(int in, int h1, int h2, int out, bool half_table) {
  const bool hidden = (in == 16 && h1 == 64 && h2 == 0) || (in == 32 && h1 == 64 && h2 == 64);
  // the 48-output (SH texture) kernels are built for the FP16 table
  return hidden && (out == 3 || (out == 48 && half_table));
}

cudaError_t launch_texture_bwd_tc_batch(int K, int KP, int in, int h1, int h2, int out, bool f16,
                                        const float* w, const ViewBatch<TexBwdView>& b,
                                        float* d_mlp, cudaStream_t st) {
  // three tiles in flight per SM where the shape allows (texture_tc_bwd3.cu)
  if (current_tuning().tex_bwd_ctas >= 3 && tex_bwd_tc3_supported(in, h1, h2, out))
    return launch_texture_bwd_tc3(K, KP, in, f16, w, b, d_mlp, st);
#define NEXEL_TCB(A, B, C, OPT, O) return tex_bwd_tc<A, B, C, OPT, O>(K, KP, w, b, d_mlp, st)
#define NEXEL_TCB2(A, B, C, O)           \
  if (out == O) {                        \
    if (f16) NEXEL_TCB(A, B, C, OpF16, O); \
    NEXEL_TCB(A, B, C, OpBf16, O);       \
  }
  if (in == 16 && h1 == 64 && h2 == 0) {
    NEXEL_TCB2(16, 64, 0, 3)
    NEXEL_TCB2(16, 64, 0, 48)
  }
  if (in == 32 && h1 == 64 && h2 == 64) {
    NEXEL_TCB2(32, 64, 64, 3)
    NEXEL_TCB2(32, 64, 64, 48)
  }
#undef NEXEL_TCB2
#undef NEXEL_TCB
  return cudaErrorInvalidValue;
}

cudaError_t launch_texture_bwd_tc(const DevCam& c, int K, int KP, long long n_rows, int in, int h1,
                                  int h2, int out, bool f16, const float* w, const uint32_t* feat,
                                  const float* weights, const int* ids, const float* d_image,
                                  const float* d_weights, const float* d_textures, float* dweff,
                                  float2* gin, float* d_mlp, int* status, cudaStream_t st) {
  ViewBatch<TexBwdView> b;
  b.n = 1;
  b.item0[0] = 0;
  b.item0[1] = (int)((n_rows + kTcRows - 1) / kTcRows);
  b.v[0] = TexBwdView{c, feat, weights, ids, d_image, d_weights, d_textures, dweff, gin, n_rows,
                      status};
  return launch_texture_bwd_tc_batch(K, KP, in, h1, h2, out, f16, w, b, d_mlp, st);
}

cudaError_t launch_texture_fwd_tc_batch(const nexel_settings& s, const nexel_field& f,
                                        const FieldDev& fd, const ViewBatch<TexFwdView>& b,
                                        cudaStream_t st) {
  const bool h = s.grid_dtype == NEXEL_F16, f16 = s.mlp_dtype == NEXEL_F16;
  const int in = f.widths[0], h1 = f.widths[1], h2 = f.n_layers == 3 ? f.widths[2] : 0;
  const int out = f.widths[f.n_layers];
#define NEXEL_TCF(A, B, C, TT, OPT, O) return tex_fwd_tc<A, B, C, TT, OPT, O>(s, fd, b, st)
#define NEXEL_TCF2(A, B, C)                                \
  if (h && out == 48) {                                    \
    if (f16) NEXEL_TCF(A, B, C, __half, OpF16, 48);        \
    NEXEL_TCF(A, B, C, __half, OpBf16, 48);                \
  }                                                        \
  if (out != 3) return cudaErrorInvalidValue;              \
  if (h) {                                                 \
    if (f16) NEXEL_TCF(A, B, C, __half, OpF16, 3);         \
    NEXEL_TCF(A, B, C, __half, OpBf16, 3);                 \
  }                                                        \
  if (f16) NEXEL_TCF(A, B, C, float, OpF16, 3);            \
  NEXEL_TCF(A, B, C, float, OpBf16, 3);
  if (in == 16 && h1 == 64 && h2 == 0) { NEXEL_TCF2(16, 64, 0) }
  if (in == 32 && h1 == 64 && h2 == 64) { NEXEL_TCF2(32, 64, 64) }
#undef NEXEL_TCF2
#undef NEXEL_TCF
  return cudaErrorInvalidValue;
}

cudaError_t launch_texture_fwd_tc(const DevCam& c, const nexel_settings& s, const nexel_field& f,
                                  const FieldDev& fd, const float* notex, const float* weights,
                                  const int* ids, const float* depths, const float* T_final,
                                  float* image, float* textures, int* status, cudaStream_t st) {
  int log2KP = 0;
  while ((1 << log2KP) < s.K) ++log2KP;
  const long long rows = (long long)c.W * c.H << log2KP;
  ViewBatch<TexFwdView> b;
  b.n = 1;
  b.item0[0] = 0;
  b.item0[1] = (int)((rows + kTcRows - 1) / kTcRows);
  b.v[0] = TexFwdView{c, notex, weights, ids, depths, T_final, image, textures,
                      fd.feat_mode == 1 ? (uint32_t*)fd.feat : nullptr, status};
  return launch_texture_fwd_tc_batch(s, f, fd, b, st);
}

cudaError_t launch_texture_gather_tc(const DevCam& c, const nexel_settings& s,
                                     const nexel_field& f, const FieldDev& fd, const int* ids,
                                     const float* depths, uint32_t* feat, cudaStream_t st) {
  const bool h = s.grid_dtype == NEXEL_F16, f16 = s.mlp_dtype == NEXEL_F16;
  const int in = f.widths[0];
#define NEXEL_TCG(A, TT, OPT) return gather_tc<A, TT, OPT>(c, s, fd, ids, depths, feat, st)
#define NEXEL_TCG2(A)                                              \
  if (h) {                                                         \
    if (f16) NEXEL_TCG(A, __half, OpF16);                          \
    NEXEL_TCG(A, __half, OpBf16);                                  \
  }                                                                \
  if (f16) NEXEL_TCG(A, float, OpF16);                             \
  NEXEL_TCG(A, float, OpBf16);
  if (in == 16) { NEXEL_TCG2(16) }
  if (in == 32) { NEXEL_TCG2(32) }
#undef NEXEL_TCG2
#undef NEXEL_TCG
  return cudaErrorInvalidValue;
}

}  // namespace nexel
