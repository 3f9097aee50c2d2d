// Texture-MLP backward on tcgen05 with three tiles in flight per CTA (RGB
// textures, two hidden layers of 64 units): the same per-sample arithmetic
// as k_tex_bwd_tc in texture_tc.cu (Sec. 4.2 / Eq. 4 backward through G, no
// bias, ReLU hidden layers, linear output; the MLP weight gradients summed
// over all samples), arranged so that the MMA round trips of one tile
// overlap the epilogues of two others.
//
// A CTA of 13 warps:
//   warps 4 g .. 4 g + 3 (g = 0, 1, 2): tile group g.  Thread t of the group
//     owns row t of the group's current 128-row tile (TMEM lane t; the warp
//     index modulo 4 is the TMEM lane quadrant).  Per tile the group stages
//     X and d3, then runs four MMA rounds, each followed by an epilogue:
//       R1  h1 = X W1^T
//       R2  h2 = h1 W2^T;  then on CUDA cores d2 = (W3^T d3) * [h2 > 0]
//       R3  d1 = (d2 W2) * [h1 > 0] and the texture T = h2 W3^T (N = 16),
//           then dL/dW_j = T . dL/dC; with R3, Da += [h1 | h2]^T [d2 | d3]
//       R4  feature gradient d1 W1;  with it Db += [X | ...]^T d1
//     The group's thread 0 issues its own rounds once the group's named
//     barrier shows all 128 rows in place, and the group waits for the
//     round's tcgen05 commit on its `done` mbarrier.  A single thread issues
//     about one MMA per 44 cycles whatever its width up to N = 128, so one
//     issuer for the CTA would serialise the groups.
//   warp 12: one thread issues the weight-gradient products Da and Db, which
//     the groups share (one issuer per accumulator), in the order the groups
//     hand their tiles over (`wready` / `wdone` mbarriers).
// A row's inputs for the next tile are loaded while the current tile runs
// and used only when it is staged.
// Shared memory per group: the activation tile [X | h1 | h2] and the delta
// tile [d2 | d3]; d1 overwrites d2 once R3 and Da (the only readers of d2)
// have completed, which keeps a group at 60 KB and three groups plus the
// weights under the 227 KB of an SM.  TMEM: 96 columns per group (its round
// accumulator and T), then Da (80 columns) and Db (64).
// Every wait is bounded; a wait that runs out ends the CTA's loops, the MMA
// thread waits (bounded) for the MMAs it issued, the TMEM is freed and the
// status word of every view of the launch gets NEXEL_ERR_TIMEOUT.
#include "tc_common.cuh"

#include <algorithm>

namespace nexel {

namespace {

using namespace tcb;

constexpr int kB3Groups = 3;
constexpr int kB3Threads = (4 * kB3Groups + 1) * 32;
constexpr int kB3MmaWarp = 4 * kB3Groups;  // the weight-gradient MMA warp

template <int IN, int H1, int H2>
struct TcBwd3Layout {
  static constexpr int FA = IN + H1 + H2;  // activation features: X | h1 | h2
  static constexpr int FD = H2 + 16;       // delta features: d2 (then d1) | d3 padded to 16
  static constexpr int SA = FA / 8 * 128, SD = FD / 8 * 128;  // bytes per 8-row group
  static constexpr int act_bytes = kTcRows / 8 * SA;
  static constexpr int del_bytes = kTcRows / 8 * SD;
  static constexpr int group_bytes = act_bytes + del_bytes;
  static constexpr int w1 = kB3Groups * group_bytes;  // [H1][IN]  B of R1
  static constexpr int w2 = w1 + H1 * IN * 2;         // [H2][H1]  B of R2
  static constexpr int w2t = w2 + H2 * H1 * 2;        // [H1][H2]  B of R3
  static constexpr int w1t = w2t + H2 * H1 * 2;       // [IN][H1]  B of R4
  static constexpr int w3b = w1t + IN * H1 * 2;       // [16][H2]  B of T (rows 3.. zero)
  static constexpr int w3 = w3b + 16 * H2 * 2;        // FP32 [3][H2]
  static constexpr int total = w3 + 3 * H2 * 4;
  // TMEM columns
  // TMEM columns: per group its round accumulator (64) and T (16), 96
  // apart; then Da and Db
  static constexpr int t_grp = 96, t_T = 64;
  static constexpr int t_da = t_grp * kB3Groups, t_db = t_da + H2 + 16;
  static constexpr int cols = 512;
  static_assert(IN % 16 == 0 && IN <= 32 && H1 == 64 && H2 == 64, "supported MLP shapes");
  static_assert(FA >= IN + 128, "Da reads 128 activation features from IN");
  static_assert(t_db + H1 <= cols, "TMEM columns");
  static_assert(total <= 220 * 1024, "shared memory");
};

__device__ __forceinline__ bool bar_test(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// A plain arrival on a hand-over barrier (the caller has ordered its
// shared-memory writes for the async proxy before).
__device__ __forceinline__ void bar_arrive_only(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// AND of `v` over the 128 threads of group g (named barrier 1 + g).
__device__ __forceinline__ bool group_and(int g, bool v) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.and.pred q, %2, 128, p;\n"
      "selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "r"(1 + g)
      : "memory");
  return r != 0;
}

template <int IN, int H1, int H2, typename OP, bool MV>
__global__ void __launch_bounds__(kB3Threads, 1) k_tex_bwd_tc3(
    const __grid_constant__ ViewBatch<TexBwdView> b, int K, int log2KP,
    const float* __restrict__ wts, float* __restrict__ d_mlp, int fault) {
  using Lt = TcBwd3Layout<IN, H1, H2>;
  const long long n_tiles = b.item0[b.n];
  // fault > 0 (test hook only): no MMA is issued and every wait gives up
  // after `fault` polls, which exercises the timeout path
  const int wlim = fault > 0 ? fault : kTcWaitLimit;
  const bool issue = fault == 0;
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  __shared__ uint32_t s_tmem;
  __shared__ __align__(8) uint64_t s_done[kB3Groups];    // a group's own rounds complete
  __shared__ __align__(8) uint64_t s_wready[kB3Groups];  // group -> weight-gradient issuer
  __shared__ __align__(8) uint64_t s_wdone[kB3Groups];   // weight-gradient issuer -> group
  __shared__ __align__(8) uint64_t s_fin[kB3Groups + 1];  // all MMAs of an issuer complete
  __shared__ int s_bad, s_acc;
  const int tid = threadIdx.x, warp = tid >> 5;
  float* w3s = reinterpret_cast<float*>(tc_smem + Lt::w3);

  // weights -> shared: BF16/FP16 K-major core-matrix tiles (B operands),
  // the output layer in FP32 rounded to the operand type (the forward's)
  {
    const float* W1 = wts;            // [H1][IN]
    const float* W2 = wts + H1 * IN;  // [H2][H1]
    const float* W3 = W2 + H2 * H1;   // [3][H2]
    for (int i = tid; i < H1 * IN; i += kB3Threads) {
      const int o = i / IN, k = i % IN;
      const uint16_t v = OP::cvt(W1[i]);
      *reinterpret_cast<uint16_t*>(tc_smem + Lt::w1 + cm_off(o, k, IN / 8 * 128)) = v;
      *reinterpret_cast<uint16_t*>(tc_smem + Lt::w1t + cm_off(k, o, H1 / 8 * 128)) = v;
    }
    for (int i = tid; i < H2 * H1; i += kB3Threads) {
      const int o = i / H1, k = i % H1;
      const uint16_t v = OP::cvt(W2[i]);
      *reinterpret_cast<uint16_t*>(tc_smem + Lt::w2 + cm_off(o, k, H1 / 8 * 128)) = v;
      *reinterpret_cast<uint16_t*>(tc_smem + Lt::w2t + cm_off(k, o, H2 / 8 * 128)) = v;
    }
    for (int i = tid; i < 3 * H2; i += kB3Threads) w3s[i] = OP::round(W3[i]);
    for (int i = tid; i < 16 * H2; i += kB3Threads) {
      const int o = i / H2, k = i % H2;
      *reinterpret_cast<uint16_t*>(tc_smem + Lt::w3b + cm_off(o, k, H2 / 8 * 128)) =
          OP::cvt(o < 3 ? W3[o * H2 + k] : 0.f);
    }
    // the delta tiles start at zero: the padding of d3 (features H2 + 8 ..)
    // stays zero
    for (int g = 0; g < kB3Groups; ++g)
      for (int i = tid; i < Lt::del_bytes / 16; i += kB3Threads)
        reinterpret_cast<uint4*>(tc_smem + g * Lt::group_bytes + Lt::act_bytes)[i] =
            make_uint4(0u, 0u, 0u, 0u);
  }
  if (tid == 0) {
    for (int g = 0; g < kB3Groups; ++g) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_done[g])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&s_wready[g])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_wdone[g])));
    }
    for (int r = 0; r <= kB3Groups; ++r)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&s_fin[r])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_bad = 0;
    s_acc = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(Lt::cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  sync_to_mma();
  const uint32_t tmem = s_tmem;
  const uint32_t sb = smem_u32(tc_smem);
  const long long stride = (long long)gridDim.x * kB3Groups;

  if (warp < kB3MmaWarp) {
    // ------------------------------------------------------ tile group g
    const int g = warp >> 2, gt = tid & 127;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    const uint32_t tg = tmem + Lt::t_grp * g;  // the group's round accumulator
    unsigned char* act = tc_smem + g * Lt::group_bytes;
    unsigned char* del = act + Lt::act_bytes;
    const int KP = 1 << log2KP;
    bool ok = true;
    uint32_t dph = 0, wph = 0;  // phases of the group's `done` and `wdone` barriers

    // per-row inputs of a tile; the group's next tile's are loaded while
    // this one's rounds run
    struct RowIn {
      uint4 x[IN / 8];
      float w, dC[3], dT[3], dWx;
      long long s, r;  // sample and row within the tile's view
      int vi, id;      // the tile's view, the slot's surfel
      bool in_pix;
    };
    // issues the loads of a row's inputs and nothing that waits for them:
    // the values are first used when the tile is staged, a tile later
    auto load_row = [&](long long tile, RowIn& in) {
      in.vi = (MV && tile < n_tiles) ? view_of(b, (int)tile) : 0;
      const TexBwdView& V = b.v[in.vi];
      const long long n_rows = V.n_rows;
      const long long P = (long long)V.c.W * V.c.H;
      const long long r = (MV ? tile - b.item0[in.vi] : tile) * kTcRows + gt;
      in.r = r;
      const long long p = r >> log2KP;
      const int j = (int)(r & (KP - 1));
      in.s = p * K + j;
      in.in_pix = tile < n_tiles && r < n_rows && p < P && j < K;
      in.id = -1;
      in.w = in.dWx = 0.f;
      in.dC[0] = in.dC[1] = in.dC[2] = 0.f;
      in.dT[0] = in.dT[1] = in.dT[2] = 0.f;
      if (in.in_pix) {
        in.id = V.ids[in.s];
        in.w = V.weights[in.s];
        in.dC[0] = V.d_image[3 * p];
        in.dC[1] = V.d_image[3 * p + 1];
        in.dC[2] = V.d_image[3 * p + 2];
        if (V.d_textures) {
          in.dT[0] = V.d_textures[3 * in.s];
          in.dT[1] = V.d_textures[3 * in.s + 1];
          in.dT[2] = V.d_textures[3 * in.s + 2];
        }
        if (V.d_weights) in.dWx = V.d_weights[in.s];
      }
#pragma unroll
      for (int c8 = 0; c8 < IN / 8; ++c8) {
        in.x[c8] = make_uint4(0u, 0u, 0u, 0u);
        if (tile < n_tiles && r < n_rows && p < P)
          in.x[c8] = reinterpret_cast<const uint4*>(V.feat + (size_t)r * (IN / 2))[c8];
      }
    };
    // BF16 has FP32's exponent range: a positive FP32 value stays positive
    // (all but FP32 subnormals below 2^-134), so the d1 epilogue reads the
    // ReLU mask of h1 back from the stored activations; FP16 rounds values
    // below 2^-25 to zero, so there the mask is kept from the FP32 values
    constexpr bool kMaskFromTile = OP::kFmt == 1;
    // the ReLU epilogue of h1: the round's accumulator -> the activation
    // tile; returns the FP32 ReLU mask where the tile cannot give it
    auto relu_h1 = [&]() {
      uint32_t m[2] = {0u, 0u};
#pragma unroll
      for (int c16 = 0; c16 < H1 / 16; ++c16) {
        float v[16];
        tmem_ld16(tg + lane_base + 16 * c16, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          if (!kMaskFromTile && v[i] > 0.f) m[c16 >> 1] |= 1u << (16 * (c16 & 1) + i);
          v[i] = fmaxf(v[i], 0.f);
        }
        st8<OP>(act, gt, IN + 16 * c16, Lt::SA, v);
        st8<OP>(act, gt, IN + 16 * c16 + 8, Lt::SA, v + 8);
      }
      return make_uint2(m[0], m[1]);
    };
    // round r of the group's tile, issued by the group's own thread 0 once
    // all 128 rows are in place (rounds 2, 3 also go to the weight-gradient
    // thread, for Da and Db)
    const uint32_t sgrp = sb + g * Lt::group_bytes;
    auto issue_round = [&](int r) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      if (r >= 2) bar_arrive_only(&s_wready[g]);
      asm volatile("bar.sync %0, 128;" ::"r"(1 + g) : "memory");
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (gt == 0 && issue) {
        constexpr uint32_t fmt = OP::kFmt;
        const uint64_t aK = sdesc(sgrp, 128, Lt::SA), dK = sdesc(sgrp + Lt::act_bytes, 128, Lt::SD);
        if (r == 0) {  // R1: h1 = X W1^T
          const uint64_t wd = sdesc(sb + Lt::w1, 128, IN / 8 * 128);
#pragma unroll
          for (int kk = 0; kk < IN / 16; ++kk)
            mma(tg, dadv(aK, kk * 256), dadv(wd, kk * 256), idesc(128, H1, 0, 0, fmt), kk > 0);
        } else if (r == 1) {  // R2: h2 = h1 W2^T
          const uint64_t wd = sdesc(sb + Lt::w2, 128, H1 / 8 * 128);
#pragma unroll
          for (int kk = 0; kk < H1 / 16; ++kk)
            mma(tg, dadv(aK, (IN / 8) * 128 + kk * 256), dadv(wd, kk * 256),
                idesc(128, H2, 0, 0, fmt), kk > 0);
        } else if (r == 2) {  // R3: d2 W2; and the texture T = h2 W3^T (N = 16)
          const uint64_t wd = sdesc(sb + Lt::w2t, 128, H2 / 8 * 128);
#pragma unroll
          for (int kk = 0; kk < H2 / 16; ++kk)
            mma(tg, dadv(dK, kk * 256), dadv(wd, kk * 256), idesc(128, H1, 0, 0, fmt), kk > 0);
          const uint64_t w3d = sdesc(sb + Lt::w3b, 128, H2 / 8 * 128);
#pragma unroll
          for (int kk = 0; kk < H2 / 16; ++kk)
            mma(tg + Lt::t_T, dadv(aK, ((IN + H1) / 8) * 128 + kk * 256), dadv(w3d, kk * 256),
                idesc(128, 16, 0, 0, fmt), kk > 0);
        } else {  // R4: feature gradient d1 W1
          const uint64_t wd = sdesc(sb + Lt::w1t, 128, H1 / 8 * 128);
#pragma unroll
          for (int kk = 0; kk < H1 / 16; ++kk)
            mma(tg, dadv(dK, kk * 256), dadv(wd, kk * 256), idesc(128, IN, 0, 0, fmt), kk > 0);
        }
        commit(&s_done[g]);
      }
    };
    auto weights_done = [&]() {
      ok = ok && wait_bar(&s_wdone[g], wph, wlim);
      wph ^= 1u;
    };
    auto round_done = [&]() {
      ok = ok && wait_bar(&s_done[g], dph, wlim);
      dph ^= 1u;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    };

    long long tile = (long long)blockIdx.x * kB3Groups + g;
    RowIn nxt;
    load_row(tile, nxt);
    for (; tile < n_tiles && ok; tile += stride) {
      const RowIn cur = nxt;
      const TexBwdView& V = b.v[MV ? cur.vi : 0];
      // the row's texture gradient gT = w dL/dC + dL/dT (Eq. 6); nothing
      // for an empty slot or a row beyond the pixels
      const bool valid = cur.in_pix && cur.id >= 0;
      const float gT[3] = {valid ? fmaf(cur.w, cur.dC[0], cur.dT[0]) : 0.f,
                           valid ? fmaf(cur.w, cur.dC[1], cur.dT[1]) : 0.f,
                           valid ? fmaf(cur.w, cur.dC[2], cur.dT[2]) : 0.f};
      // stage X and d3 (the previous tile's R4 and Db have completed)
#pragma unroll
      for (int c8 = 0; c8 < IN / 8; ++c8)
        *reinterpret_cast<uint4*>(act + cm_off(gt, 8 * c8, Lt::SA)) = cur.x[c8];
      {
        const float d3[8] = {OP::kScale * gT[0], OP::kScale * gT[1],
                             OP::kScale * gT[2], 0.f, 0.f, 0.f, 0.f, 0.f};
        st8<OP>(del, gt, H2, Lt::SD, d3);
      }
      issue_round(0);
      load_row(tile + stride, nxt);
      round_done();
      const uint2 m1 = relu_h1();
      issue_round(1);
      round_done();
      // h2 = ReLU of the round's accumulator, and with it (CUDA cores)
      // d2 = (W3^T d3) * [h2 > 0]
      {
        const float4* w34 = reinterpret_cast<const float4*>(w3s);
#pragma unroll
        for (int c16 = 0; c16 < H2 / 16; ++c16) {
          float v[16], d2[16];
          tmem_ld16(tg + lane_base + 16 * c16, v);
#pragma unroll
          for (int c4 = 0; c4 < 4; ++c4) {
            const int q0 = 16 * c16 + 4 * c4;
            const float4 a0 = w34[q0 / 4], a1 = w34[(H2 + q0) / 4], a2 = w34[(2 * H2 + q0) / 4];
            const float wr[3][4] = {{a0.x, a0.y, a0.z, a0.w}, {a1.x, a1.y, a1.z, a1.w},
                                    {a2.x, a2.y, a2.z, a2.w}};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int i = 4 * c4 + e;
              const bool pos = v[i] > 0.f;
              v[i] = fmaxf(v[i], 0.f);
              const float gsum = OP::kScale * fmaf(gT[0], wr[0][e],
                                                   fmaf(gT[1], wr[1][e], gT[2] * wr[2][e]));
              d2[i] = pos ? gsum : 0.f;
            }
          }
          st8<OP>(act, gt, IN + H1 + 16 * c16, Lt::SA, v);
          st8<OP>(act, gt, IN + H1 + 16 * c16 + 8, Lt::SA, v + 8);
          st8<OP>(del, gt, 16 * c16, Lt::SD, d2);
          st8<OP>(del, gt, 16 * c16 + 8, Lt::SD, d2 + 8);
        }
      }
      issue_round(2);  // and Da
      round_done();
      {
        // dL/dW_j = T . dL/dC + dL/dW_j (upstream), T from the R3 round
        float T[8];
        tmem_ld8(tg + Lt::t_T + lane_base, T);
        if (cur.in_pix)
          V.dweff[cur.s] =
              valid ? T[0] * cur.dC[0] + T[1] * cur.dC[1] + T[2] * cur.dC[2] + cur.dWx : 0.f;
      }
      weights_done();  // Da has read d2
      // d1 = (d2 W2) * [h1 > 0], over d2 (R3 and Da, its readers, are done)
#pragma unroll
      for (int c16 = 0; c16 < H1 / 16; ++c16) {
        float v[16];
        tmem_ld16(tg + lane_base + 16 * c16, v);
        if constexpr (kMaskFromTile) {
          // a stored BF16 value is positive exactly when it is as a signed
          // 16-bit integer
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int f0 = 16 * c16 + 8 * h;
            const uint4 hq = *reinterpret_cast<const uint4*>(act + cm_off(gt, IN + f0, Lt::SA));
            const uint4 dq = pack8<OP>(v + 8 * h);
            *reinterpret_cast<uint4*>(del + cm_off(gt, f0, Lt::SD)) =
                make_uint4(dq.x & __vcmpgts2(hq.x, 0u), dq.y & __vcmpgts2(hq.y, 0u),
                           dq.z & __vcmpgts2(hq.z, 0u), dq.w & __vcmpgts2(hq.w, 0u));
          }
        } else {
          const uint32_t mw = (c16 >> 1) ? m1.y : m1.x;
#pragma unroll
          for (int i = 0; i < 16; ++i) v[i] = ((mw >> (16 * (c16 & 1) + i)) & 1u) ? v[i] : 0.f;
          st8<OP>(del, gt, 16 * c16, Lt::SD, v);
          st8<OP>(del, gt, 16 * c16 + 8, Lt::SD, v + 8);
        }
      }
      issue_round(3);  // and Db
      round_done();
      {
        // feature gradient, level-major float2 per level, streamed to the
        // hash backward (evict-first)
        const long long R = gin_stride(V.n_rows);
#pragma unroll
        for (int c16 = 0; c16 < IN / 16; ++c16) {
          float v[16];
          tmem_ld16(tg + lane_base + 16 * c16, v);
          if (cur.r < V.n_rows) {
#pragma unroll
            for (int i = 0; i < 8; ++i)
              __stcs(V.gin + (long long)(8 * c16 + i) * R + cur.r,
                     make_float2(v[2 * i] * (1.f / OP::kScale), v[2 * i + 1] * (1.f / OP::kScale)));
          }
        }
      }
      // Db has read X, h1 and d1 before the next tile overwrites them
      weights_done();
      // the next R1 overwrites the group's accumulator: these TMEM reads
      // come first; a wait that ran out on any thread ends the group's loop
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      ok = group_and(g, ok);
    }
    // the group's MMAs have completed before the TMEM is read or freed
    if (gt == 0 && issue) {
      commit(&s_fin[g]);
      if (!wait_bar(&s_fin[g], 0, kTcWaitLimit)) ok = false;
    }
    if (!ok) s_bad = 1;
  } else if (tid == kB3MmaWarp * 32) {
    // ------------------------------------------- weight-gradient MMA thread
    // Da and Db, shared by the groups, have this one issuer; it serves the
    // groups in the order they hand their tiles over (two events per tile).
    constexpr uint32_t fmt = OP::kFmt;
    int left[kB3Groups], ev[kB3Groups];
    uint32_t rph[kB3Groups];
    uint64_t aM[kB3Groups], dM[kB3Groups];  // MN-major base descriptors
    for (int g = 0; g < kB3Groups; ++g) {
      const long long t0 = (long long)blockIdx.x * kB3Groups + g;
      left[g] = t0 < n_tiles ? (int)((n_tiles - 1 - t0) / stride + 1) : 0;
      ev[g] = 0;
      rph[g] = 0;
      const uint32_t act = sb + g * Lt::group_bytes;
      aM[g] = sdesc(act, Lt::SA, 128);
      dM[g] = sdesc(act + Lt::act_bytes, Lt::SD, 128);
    }
    bool da_acc = false, db_acc = false, ok = true;
    int idle = 0;
    while (left[0] + left[1] + left[2] > 0) {
      bool any = false;
#pragma unroll
      for (int g = 0; g < kB3Groups; ++g) {
        if (left[g] == 0 || !bar_test(&s_wready[g], rph[g])) continue;
        rph[g] ^= 1u;
        any = true;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (issue) {
          // K = rows: 16 rows = two 8-row groups per MMA, operands MN-major
          if (ev[g] == 0) {  // Da += [h1 | h2]^T [d2 | d3]
#pragma unroll
            for (int kk = 0; kk < kTcRows / 16; ++kk)
              mma(tmem + Lt::t_da, dadv(aM[g], (IN / 8) * 128 + kk * 2 * Lt::SA),
                  dadv(dM[g], kk * 2 * Lt::SD), idesc(128, H2 + 16, 1, 1, fmt), da_acc || kk > 0);
            da_acc = true;
          } else {  // Db += [X | ...]^T d1
#pragma unroll
            for (int kk = 0; kk < kTcRows / 16; ++kk)
              mma(tmem + Lt::t_db, dadv(aM[g], kk * 2 * Lt::SA), dadv(dM[g], kk * 2 * Lt::SD),
                  idesc(128, H1, 1, 1, fmt), db_acc || kk > 0);
            db_acc = true;
          }
          commit(&s_wdone[g]);
        }
        if (++ev[g] == 2) {
          ev[g] = 0;
          --left[g];
        }
      }
      if (any) {
        idle = 0;
      } else if (++idle > wlim) {  // a group stopped handing tiles over
        ok = false;
        break;
      }
    }
    // every MMA issued here has completed before the TMEM is read or freed
    if (issue) {
      commit(&s_fin[kB3Groups]);
      if (!wait_bar(&s_fin[kB3Groups], 0, kTcWaitLimit)) ok = false;
    }
    if (!ok) s_bad = 1;
    s_acc = (da_acc && db_acc) ? 1 : 0;
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // weight gradients of this CTA (group 0's warps cover the four TMEM lane
  // quadrants): Da lane m = activation feature IN + m, column n = delta
  // feature n; Db lane m = activation feature m, column n = d1 feature n
  if (tid < 128 && !s_bad && s_acc && d_mlp) {
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    float* dW1 = d_mlp;
    float* dW2 = d_mlp + H1 * IN;
    float* dW3 = dW2 + H2 * H1;
    const int m = tid;
    for (int c16 = 0; c16 < (H2 + 16) / 16; ++c16) {
      float v[16];
      tmem_ld16(tmem + Lt::t_da + lane_base + 16 * c16, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int n = 16 * c16 + i;
        if (m < H1 && n < H2) atomicAdd(dW2 + n * H1 + m, v[i] * (1.f / OP::kScale));
        if (m >= H1 && m < H1 + H2 && n >= H2 && n < H2 + 3)
          atomicAdd(dW3 + (n - H2) * H2 + (m - H1), v[i] * (1.f / OP::kScale));
      }
    }
    for (int c16 = 0; c16 < H1 / 16; ++c16) {
      float v[16];
      tmem_ld16(tmem + Lt::t_db + lane_base + 16 * c16, v);
#pragma unroll
      for (int i = 0; i < 16; ++i)
        if (m < IN) atomicAdd(dW1 + (16 * c16 + i) * IN + m, v[i] * (1.f / OP::kScale));
    }
  }
  if (s_bad && tid == 0)  // a wait that ran out marks every view of the launch
    for (int v = 0; v < b.n; ++v)
      if (b.v[v].status) atomicOr(b.v[v].status, kStatusTimeout);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Lt::cols));
}

template <int IN, typename OP>
cudaError_t tex_bwd_tc3(int K, int KP, const float* w, const ViewBatch<TexBwdView>& b,
                        float* d_mlp, cudaStream_t st) {
  using Lt = TcBwd3Layout<IN, 64, 64>;
  int log2KP = 0;
  while ((1 << log2KP) < KP) ++log2KP;
  const long long n_tiles = b.item0[b.n];
  if (n_tiles == 0) return cudaSuccess;
  auto kern = b.n > 1 ? k_tex_bwd_tc3<IN, 64, 64, OP, true> : k_tex_bwd_tc3<IN, 64, 64, OP, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Lt::total);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // one CTA per SM (its shared memory and TMEM), three tiles in flight
  const unsigned grid =
      (unsigned)std::min<long long>((n_tiles + kB3Groups - 1) / kB3Groups, nsm);
  NEXEL_PROF("texture_bwd_tc", st);
  kern<<<grid, kB3Threads, Lt::total, st>>>(b, K, log2KP, w, d_mlp, tc_wait_fault());
  return cudaGetLastError();
}

}  // namespace

bool tex_bwd_tc3_supported(int in, int h1, int h2, int out) {
  return (in == 16 || in == 32) && h1 == 64 && h2 == 64 && out == 3;
}

cudaError_t launch_texture_bwd_tc3(int K, int KP, int in, bool f16, const float* w,
                                   const ViewBatch<TexBwdView>& b, float* d_mlp, cudaStream_t st) {
  if (in == 32)
    return f16 ? tex_bwd_tc3<32, OpF16>(K, KP, w, b, d_mlp, st)
               : tex_bwd_tc3<32, OpBf16>(K, KP, w, b, d_mlp, st);
  if (in == 16)
    return f16 ? tex_bwd_tc3<16, OpF16>(K, KP, w, b, d_mlp, st)
               : tex_bwd_tc3<16, OpBf16>(K, KP, w, b, d_mlp, st);
  return cudaErrorInvalidValue;
}

}  // namespace nexel
