// Building blocks of the tcgen05 texturing kernels (texture_tc.cu,
// texture_tc_bwd3.cu): shared-memory and instruction descriptors for
// tcgen05.mma kind::f16 (no swizzle, core-matrix layout), the MMA issue and
// its completion (tcgen05.commit to an mbarrier, bounded waits), TMEM
// read-back, and the BF16 / FP16 operand types.
#pragma once

#include "texture_common.cuh"

namespace nexel {
namespace tcb {

constexpr int kTcRows = 128;
constexpr int kTcThreads = 128;
constexpr int kTcWaitLimit = 1 << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor, no swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// A shared-memory descriptor moved `bytes` (a multiple of 16) further along
// its start address.  The address field holds the byte address / 16 in 14
// bits, which no address inside the 228 KB of an SM overflows, so the move
// is one add.
__device__ __forceinline__ uint64_t dadv(uint64_t d, uint32_t bytes) { return d + (bytes >> 4); }

// instruction descriptor, kind::f16: A and B of format fmt (0 = F16,
// 1 = BF16), F32 accumulator, M x N
__host__ __device__ constexpr uint32_t idesc(int m, int n, int a_mn, int b_mn, uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                    bool acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(id), "r"((uint32_t)acc));
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_u32(bar)));
}

// Bounded wait for the mbarrier phase `parity`; false when `limit` polls ran
// out.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, int limit) {
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity));
    if (done) return true;
  }
  return false;
}

// 16 consecutive FP32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
      "[%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive FP32 columns of this thread's TMEM lane (one wait)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Thread-to-MMA hand-over: generic-proxy shared stores and TMEM reads of all
// threads happen before the MMAs thread 0 issues next.
__device__ __forceinline__ void sync_to_mma() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// MMA operand type.  BF16; or FP16, where the backward scales the gradient
// entering the MLP by 128 and unscales the feature and weight gradients (the
// paper trains the MLP in FP16 with a loss scale of 128).
struct OpBf16 {
  static constexpr uint32_t kFmt = 1;
  static constexpr float kScale = 1.f;
  __device__ static uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
  }
  __device__ static float2 unpack2(uint32_t w) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w));
  }
  __device__ static uint16_t cvt(float x) {
    __nv_bfloat16 b = __float2bfloat16_rn(x);
    return *reinterpret_cast<uint16_t*>(&b);
  }
  __device__ static float round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
};
struct OpF16 {
  static constexpr uint32_t kFmt = 0;
  static constexpr float kScale = 128.f;
  __device__ static uint32_t pack2(float lo, float hi) {
    __half2 v = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
  }
  __device__ static float2 unpack2(uint32_t w) {
    return __half22float2(*reinterpret_cast<const __half2*>(&w));
  }
  __device__ static uint16_t cvt(float x) {
    __half h = __float2half_rn(x);
    return *reinterpret_cast<uint16_t*>(&h);
  }
  __device__ static float round(float x) { return __half2float(__float2half_rn(x)); }
};

// byte offset of element (row r, feature f) in a core-matrix tile whose
// 8-row groups are sg bytes apart
__host__ __device__ constexpr uint32_t cm_off(int r, int f, int sg) {
  return (uint32_t)((r >> 3) * sg + (f >> 3) * 128 + (r & 7) * 16 + (f & 7) * 2);
}

// 8 consecutive values packed to the operand type (16 bytes)
template <typename OP>
__device__ __forceinline__ uint4 pack8(const float* v) {
  return make_uint4(OP::pack2(v[0], v[1]), OP::pack2(v[2], v[3]), OP::pack2(v[4], v[5]),
                    OP::pack2(v[6], v[7]));
}

// Stores 8 consecutive features f0..f0+7 (f0 % 8 == 0) of row r.
template <typename OP>
__device__ __forceinline__ void st8(unsigned char* base, int r, int f0, int sg, const float* v) {
  uint4 q = make_uint4(OP::pack2(v[0], v[1]), OP::pack2(v[2], v[3]), OP::pack2(v[4], v[5]),
                       OP::pack2(v[6], v[7]));
  *reinterpret_cast<uint4*>(base + cm_off(r, f0, sg)) = q;
}

}  // namespace tcb
}  // namespace nexel
