// Surfel preprocess, tile binning (the stable radix sort of the centre
// depths, then the per-tile lists), plus the preprocess backward.
//
// Ordering (Sec. 3, "Preliminaries"): surfels are sorted by the view depth of
// their centres and composited per tile.  Instead of sorting 64-bit
// (tile, depth) keys of every (tile, surfel) instance, the N surfels are
// first sorted by depth (32-bit float keys, index order on ties).  The
// instances are then placed directly at their slots in the per-tile lists
// (at most kPlaceMaxTiles tiles), or emitted in depth-rank order and stably
// sorted on the tile bits alone.  Either way the per-tile lists are
// identical, bit for bit, to a stable sort of (tile << 32 | depth bits)
// keys.  A key is (tile << rank_bits | rank), in 32 bits whenever
// tile_bits + rank_bits <= 32; otherwise a placed key holds the rank alone
// (32 bits; its slot gives the tile) and a sorted one is 64-bit.
#include "common.cuh"

#include <algorithm>
#include <cmath>

namespace nexel {

// ----------------------------------------------------------- float-float
struct ff { float hi, lo; };
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ ff two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ ff two_prod(float a, float b) {
  float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
  ff s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff ff_mul_f(ff a, float b) {
  ff p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, fmaf(a.lo, b, p.lo));
}
__device__ __forceinline__ ff ff_div(ff a, ff b) {
  float q1 = a.hi / b.hi;
  ff qb = ff_mul_f(b, q1);
  ff r = ff_add(a, {-qb.hi, -qb.lo});
  float q2 = r.hi / b.hi;
  return fast_two_sum(q1, q2);
}

__device__ __forceinline__ float3 rot(const float* R, float3 v) {
  return make_float3(R[0] * v.x + R[1] * v.y + R[2] * v.z, R[3] * v.x + R[4] * v.y + R[5] * v.z,
                     R[6] * v.x + R[7] * v.y + R[8] * v.z);
}
__device__ __forceinline__ float3 rotT(const float* R, float3 v) {
  return make_float3(R[0] * v.x + R[3] * v.y + R[6] * v.z, R[1] * v.x + R[4] * v.y + R[7] * v.z,
                     R[2] * v.x + R[5] * v.y + R[8] * v.z);
}

// ------------------------------------------------------------ preprocess
// One thread per surfel.  Builds the packed record (see common.cuh), the
// depth key and the tile rectangle of the region where alpha >= alpha_min:
// |u| <= (2 ln(o / alpha_min))^(1 / (2 gamma_1)) and likewise for v, i.e. a
// rectangle on the surfel plane, clipped to view depth >= near (hits at
// t* <= near are dropped) and projected; its image is the convex hull of the
// projected vertices.
// Conservative tile test.  With the conic of the support written by
// k_preprocess, Q(delta) = delta^T M delta + 2 b . delta - 1 <= 0 holds at
// every pixel where alpha >= alpha_min.  The tile is kept unless Q > 0 on
// the whole rectangle of its pixel centres grown by one pixel (and a small
// tolerance), so dropping it removes only (pixel, surfel) pairs that the
// collection pass would skip anyway.
//
// Minimum of Q over the rectangle.  When M is positive definite (the
// common case: the support is an ellipse) Q is convex with its minimum at
// delta*: if delta* lies in the rectangle the tile is kept; otherwise the
// constrained minimum lies on an edge that faces delta* (from the minimiser
// Q decreases towards delta*, which must leave the rectangle), so only the
// one or two facing edges are searched.  Otherwise (an oblique surfel whose
// support reaches the horizon) the minimum lies at a corner, at the
// critical point of an edge or at the interior critical point.
//
// Every operation is explicitly rounded (no contraction left to the
// compiler), so the counting and the emitting kernels take identical
// decisions.
struct TileConic {
  float m00, m01, m11, bx, by, cpx, cpy, inv00, inv11, dsx, dsy, pd;
};

__device__ __forceinline__ TileConic load_conic(const float4* __restrict__ conic, uint32_t i) {
  const float4 a = conic[3 * i], b = conic[3 * i + 1], c = conic[3 * i + 2];
  return {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
}

__device__ __forceinline__ float conic_q(const TileConic& k, float x, float y) {
  // x (m00 x + 2 (m01 y + bx)) + y (m11 y + 2 by) - 1
  const float lx = __fmaf_rn(k.m00, x, __fmul_rn(2.f, __fmaf_rn(k.m01, y, k.bx)));
  const float ly = __fmaf_rn(k.m11, y, __fmul_rn(2.f, k.by));
  return __fadd_rn(__fmaf_rn(x, lx, __fmul_rn(y, ly)), -1.f);
}

// min of Q on the edge x = xe, y in [y0, y1] (m11 > 0)
__device__ __forceinline__ float edge_min_x(const TileConic& k, float xe, float y0, float y1) {
  const float y = fminf(fmaxf(__fmul_rn(-__fmaf_rn(k.m01, xe, k.by), k.inv11), y0), y1);
  return conic_q(k, xe, y);
}
// min of Q on the edge y = ye, x in [x0, x1] (m00 > 0)
__device__ __forceinline__ float edge_min_y(const TileConic& k, float ye, float x0, float x1) {
  const float x = fminf(fmaxf(__fmul_rn(-__fmaf_rn(k.m01, ye, k.bx), k.inv00), x0), x1);
  return conic_q(k, x, ye);
}

__device__ __forceinline__ bool tile_may_hit(const TileConic& k, int tx, int ty, int W, int H) {
  const float X0 = __fadd_rn((float)(tx * kTile) - 0.5f, -k.cpx);
  const float X1 = __fadd_rn((float)min(tx * kTile + kTile - 1, W - 1) + 1.5f, -k.cpx);
  const float Y0 = __fadd_rn((float)(ty * kTile) - 0.5f, -k.cpy);
  const float Y1 = __fadd_rn((float)min(ty * kTile + kTile - 1, H - 1) + 1.5f, -k.cpy);
  float q = 3.0e38f;
  if (k.pd != 0.f) {
    const bool in_x = k.dsx >= X0 && k.dsx <= X1, in_y = k.dsy >= Y0 && k.dsy <= Y1;
    if (in_x && in_y) return true;
    if (!in_x) q = edge_min_x(k, k.dsx < X0 ? X0 : X1, Y0, Y1);
    if (!in_y) q = fminf(q, edge_min_y(k, k.dsy < Y0 ? Y0 : Y1, X0, X1));
  } else {
    q = fminf(fminf(conic_q(k, X0, Y0), conic_q(k, X1, Y0)),
              fminf(conic_q(k, X0, Y1), conic_q(k, X1, Y1)));
    if (k.m00 > 0.f) q = fminf(q, fminf(edge_min_y(k, Y0, X0, X1), edge_min_y(k, Y1, X0, X1)));
    if (k.m11 > 0.f) q = fminf(q, fminf(edge_min_x(k, X0, Y0, Y1), edge_min_x(k, X1, Y0, Y1)));
  }
  return !(q > 1e-3f);  // NaN keeps the tile
}

__global__ void k_preprocess(DevCam c, float alpha_min, int sh_degree, int N,
                             const float* __restrict__ mu,
                             const float* __restrict__ quat, const float* __restrict__ scale,
                             const float* __restrict__ opac, const float* __restrict__ gam,
                             const float* __restrict__ color, float4* __restrict__ geom,
                             float4* __restrict__ aux, uint32_t* __restrict__ dkey,
                             uint32_t* __restrict__ did, uint2* __restrict__ rect,
                             float4* __restrict__ conic, uint32_t* __restrict__ count,
                             float* __restrict__ shj, uint32_t* __restrict__ n_nonfinite,
                             int* __restrict__ status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  did[i] = (uint32_t)i;
  float m[3] = {mu[3 * i], mu[3 * i + 1], mu[3 * i + 2]};
  float qw = quat[4 * i], qx = quat[4 * i + 1], qy = quat[4 * i + 2], qz = quat[4 * i + 3];
  float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  // A surfel with a NaN or infinite parameter (or a zero quaternion) has no
  // defined footprint: it is culled like one behind the camera, counted, and
  // the status word reports it (NEXEL_ERR_NUMERIC from nexel_read_status).
  bool finite = isfinite(m[0]) && isfinite(m[1]) && isfinite(m[2]) && isfinite(qn) &&
                isfinite(qw) && isfinite(qx) && isfinite(qy) && isfinite(qz) &&
                isfinite(scale[2 * i]) && isfinite(scale[2 * i + 1]) && isfinite(opac[i]) &&
                isfinite(gam[2 * i]) && isfinite(gam[2 * i + 1]);
  {
    const int nc = sh_degree == 3 ? 48 : 3;
    for (int k = 0; k < nc; ++k) finite = finite && isfinite(color[(size_t)nc * i + k]);
  }
  if (!finite) {
    atomicAdd(n_nonfinite, 1u);
    atomicOr(status, kStatusNumeric);
  }
  qw *= qn; qx *= qn; qy *= qn; qz *= qn;
  float3 v1, v2, n;
  quat_cols(qw, qx, qy, qz, v1, v2, n);
  float s1 = scale[2 * i], s2 = scale[2 * i + 1];
  float o = opac[i];
  float g1 = gam[2 * i], g2 = gam[2 * i + 1];
  // camera-space centre in float-float (the projected centre is the one
  // quantity whose absolute error enters every pixel's offset)
  ff mc[3];
  for (int a = 0; a < 3; ++a) {
    ff acc = two_prod(c.R[3 * a], m[0]);
    acc = ff_add(acc, two_prod(c.R[3 * a + 1], m[1]));
    acc = ff_add(acc, two_prod(c.R[3 * a + 2], m[2]));
    mc[a] = ff_add(acc, {c.t[a], 0.f});
  }
  float z = mc[2].hi;
  float3 v1c = rot(c.R, v1), v2c = rot(c.R, v2), nc = rot(c.R, n);
  bool ok = finite && (z > c.near_) && (o >= alpha_min) && (s1 > 0.f) && (s2 > 0.f) &&
            (g1 >= 1.f) && (g2 >= 1.f);
  float dmx = 0.f, dmy = 0.f, dn0 = 0.f;
  if (ok) {
    dmx = mc[0].hi / z;
    dmy = mc[1].hi / z;
    dn0 = dmx * nc.x + dmy * nc.y + nc.z;
    ok = fabsf(dn0) >= 1e-7f;  // edge-on to its own centre ray: a line, dropped
  }
  uint2 rc = make_uint2(0, 0);
  uint32_t cnt = 0;
  if (ok) {
    // support rectangle, slightly inflated
    float lr = 2.f * logf(o / alpha_min);
    float ru = (lr > 0.f ? powf(lr, 0.5f / g1) : 0.f) * 1.001f + 1e-6f;
    float rv = (lr > 0.f ? powf(lr, 0.5f / g2) : 0.f) * 1.001f + 1e-6f;
    float3 eu = make_float3(ru * s1 * v1c.x, ru * s1 * v1c.y, ru * s1 * v1c.z);
    float3 ev = make_float3(rv * s2 * v2c.x, rv * s2 * v2c.y, rv * s2 * v2c.z);
    float3 ctr = make_float3(mc[0].hi, mc[1].hi, z);
    float3 P[4];
    const float su[4] = {-1.f, 1.f, 1.f, -1.f}, sv[4] = {-1.f, -1.f, 1.f, 1.f};
    for (int k = 0; k < 4; ++k)
      P[k] = make_float3(ctr.x + su[k] * eu.x + sv[k] * ev.x, ctr.y + su[k] * eu.y + sv[k] * ev.y,
                         ctr.z + su[k] * eu.z + sv[k] * ev.z);
    float xmin = 3e38f, xmax = -3e38f, ymin = 3e38f, ymax = -3e38f;
    int nv = 0;
    auto take = [&](float3 p) {
      float iz = 1.f / p.z;
      float px = c.fx * p.x * iz + c.cx, py = c.fy * p.y * iz + c.cy;
      xmin = fminf(xmin, px); xmax = fmaxf(xmax, px);
      ymin = fminf(ymin, py); ymax = fmaxf(ymax, py);
      ++nv;
    };
    for (int k = 0; k < 4; ++k) {
      float3 A = P[k], B = P[(k + 1) & 3];
      bool ia = A.z >= c.near_, ib = B.z >= c.near_;
      if (ia) take(A);
      if (ia != ib) {
        float s = (c.near_ - A.z) / (B.z - A.z);
        float3 X = make_float3(A.x + s * (B.x - A.x), A.y + s * (B.y - A.y), c.near_);
        take(X);
      }
    }
    if (nv > 0) {
      // pixel centres (x + .5) inside [xmin, xmax], one pixel of margin
      float fx0 = fmaxf(xmin - 1.5f, -1e7f), fx1 = fminf(xmax + 0.5f, 1e7f);
      float fy0 = fmaxf(ymin - 1.5f, -1e7f), fy1 = fminf(ymax + 0.5f, 1e7f);
      int px0 = max((int)ceilf(fx0), 0), px1 = min((int)floorf(fx1), c.W - 1);
      int py0 = max((int)ceilf(fy0), 0), py1 = min((int)floorf(fy1), c.H - 1);
      if (px0 <= px1 && py0 <= py1) {
        int tx0 = px0 / kTile, tx1 = px1 / kTile, ty0 = py0 / kTile, ty1 = py1 / kTile;
        rc = make_uint2((uint32_t)tx0 | ((uint32_t)tx1 << 16), (uint32_t)ty0 | ((uint32_t)ty1 << 16));
        cnt = (uint32_t)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
      }
    }
  }
  if (cnt == 0) ok = false;
  rect[i] = rc;
  count[i] = cnt;
  dkey[i] = ok ? __float_as_uint(z) : 0xFFFFFFFFu;
  float4* g = geom + (size_t)i * kRecF4;
  if (!ok) {
    for (int k = 0; k < kRecF4; ++k) g[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < kAuxF4; ++k) aux[(size_t)i * kAuxF4 + k] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  // projected centre in float-float: cp = f * (mc / z) + c
  ff zz = mc[2];
  ff dx = ff_div(mc[0], zz), dy = ff_div(mc[1], zz);
  ff cpx = ff_add(ff_mul_f(dx, c.fx), {c.cx, 0.f});
  ff cpy = ff_add(ff_mul_f(dy, c.fy), {c.cy, 0.f});
  // u and v numerators (common.cuh): Cu = -z (d_mu x v2) / s1 and
  // Cv = z (d_mu x v1) / s2, x and y components, with z d_mu = mu_c
  const float mx = mc[0].hi, my = mc[1].hi;
  const float Cux = -(my * v2c.z - z * v2c.y) / s1, Cuy = -(z * v2c.x - mx * v2c.z) / s1;
  const float Cvx = (my * v1c.z - z * v1c.y) / s2, Cvy = (z * v1c.x - mx * v1c.z) / s2;
  {
    // support conic for the tile test (tile_may_hit): with delta the pixel
    // offset from the projected centre and den = dn0 + delta . n', the
    // support |u|^(2 g1) + |v|^(2 g2) <= 2 ln(o / alpha_min) lies inside
    // (u / ru)^2 + (v / rv)^2 <= kappa (kappa = 1 when g1 = g2 = 1, else 2),
    // i.e. Q(delta) = (delta . A)^2 + (delta . B)^2 - kappa den^2 <= 0 with
    // A = Cu' / ru, B = Cv' / rv; stored divided by kappa dn0^2, so that
    // Q = delta^T M delta + 2 b . delta - 1.
    const float lr = 2.f * logf(o / alpha_min);
    const float ru = powf(lr, 0.5f / g1) * 1.001f + 1e-6f, rv = powf(lr, 0.5f / g2) * 1.001f + 1e-6f;
    const float kap = (g1 == 1.f && g2 == 1.f) ? 1.f : 2.f;
    const float Ax = Cux / (c.fx * ru), Ay = Cuy / (c.fy * ru);
    const float Bx = Cvx / (c.fx * rv), By = Cvy / (c.fy * rv);
    const float nx = nc.x / c.fx, ny = nc.y / c.fy;
    const float is = 1.f / (kap * dn0 * dn0), in2 = 1.f / (dn0 * dn0);
    const float m00 = (Ax * Ax + Bx * Bx) * is - nx * nx * in2;
    const float m01 = (Ax * Ay + Bx * By) * is - nx * ny * in2;
    const float m11 = (Ay * Ay + By * By) * is - ny * ny * in2;
    const float bx = -nx / dn0, by = -ny / dn0;
    const float det = m00 * m11 - m01 * m01;
    const bool pd = m00 > 0.f && m11 > 0.f && det > 0.f;
    // minimiser delta* = -M^-1 b of the convex case
    const float dsx = pd ? (m01 * by - m11 * bx) / det : 0.f;
    const float dsy = pd ? (m01 * bx - m00 * by) / det : 0.f;
    conic[3 * i] = make_float4(m00, m01, m11, bx);
    conic[3 * i + 1] = make_float4(by, cpx.hi, cpy.hi, m00 > 0.f ? 1.f / m00 : 0.f);
    conic[3 * i + 2] = make_float4(m11 > 0.f ? 1.f / m11 : 0.f, dsx, dsy, pd ? 1.f : 0.f);
  }
  g[0] = make_float4(cpx.hi, cpy.hi, cpx.lo, cpy.lo);
  g[1] = make_float4(z, o, g1, g2);
  g[2] = make_float4(nc.x / c.fx, nc.y / c.fy, Cux / c.fx, Cuy / c.fy);
  g[3] = make_float4(Cvx / c.fx, Cvy / c.fy, dn0, 0.f);
  float3 rgb;
  if (sh_degree == 3) {
    // degree-3 SH coefficients [16][3], evaluated in the direction from the
    // camera centre to the surfel centre, plus one half
    float dx = m[0] - c.o[0], dy = m[1] - c.o[1], dz = m[2] - c.o[2];
    const float inv = rsqrtf(fmaxf(dx * dx + dy * dy + dz * dz, 1e-30f));
    const Sh3 Y = sh3_eval(dx * inv, dy * inv, dz * inv);
    const float* cf = color + (size_t)48 * i;
    rgb = make_float3(0.5f, 0.5f, 0.5f);
    float w[3][16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      w[0][k] = cf[3 * k]; w[1][k] = cf[3 * k + 1]; w[2][k] = cf[3 * k + 2];
      rgb.x = fmaf(Y.y[k], w[0][k], rgb.x);
      rgb.y = fmaf(Y.y[k], w[1][k], rgb.y);
      rgb.z = fmaf(Y.y[k], w[2][k], rgb.z);
    }
    // d colour_ch / d dir (for the backward, which has no coefficients)
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float3 gd = sh3_grad_dot(dx * inv, dy * inv, dz * inv, w[ch]);
      shj[9 * (size_t)i + 3 * ch] = gd.x;
      shj[9 * (size_t)i + 3 * ch + 1] = gd.y;
      shj[9 * (size_t)i + 3 * ch + 2] = gd.z;
    }
  } else {
    rgb = make_float3(color[3 * i], color[3 * i + 1], color[3 * i + 2]);
  }
  g[4] = make_float4(rgb.x, rgb.y, rgb.z, __uint_as_float((uint32_t)i));
  float4* a = aux + (size_t)i * kAuxF4;
  a[0] = make_float4(mx, my, z, s1);
  a[1] = make_float4(v1c.x, v1c.y, v1c.z, s2);
  a[2] = make_float4(v2c.x, v2c.y, v2c.z, 1.f / s1);
  a[3] = make_float4(nc.x, nc.y, nc.z, 1.f / s2);
}

// ------------------------------------------------------- scan (exclusive)
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_w, uint32_t& total) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) s_w[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int nw = blockDim.x >> 5;
    uint32_t y = lane < nw ? s_w[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t z = __shfl_up_sync(0xffffffffu, y, d);
      if (lane >= d) y += z;
    }
    if (lane < nw) s_w[lane] = y;
  }
  __syncthreads();
  uint32_t pre = warp > 0 ? s_w[warp - 1] : 0;
  total = s_w[(blockDim.x >> 5) - 1];
  __syncthreads();
  return pre + x - v;
}

// Exclusive scan in two launches: the block sums of kScanTile-element
// tiles, then every block adds the sum of the tiles before it (a block
// reduction over at most a few thousand sums) to its own in-place scan.
__global__ void __launch_bounds__(256) k_scan_reduce(const uint32_t* __restrict__ a, long long n,
                                                     uint32_t* __restrict__ sums) {
  __shared__ uint32_t s_w[8];
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  uint32_t loc = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) loc += (base + k < n) ? a[base + k] : 0u;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) loc += __shfl_xor_sync(0xffffffffu, loc, d);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = loc;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += s_w[w];
    sums[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(256) k_scan_final(uint32_t* __restrict__ a, long long n,
                                                    const uint32_t* __restrict__ sums,
                                                    uint32_t* __restrict__ total_out) {
  __shared__ uint32_t s_w[8];
  __shared__ uint32_t s_carry;
  // carry = sum of the sums of the tiles before this one
  uint32_t c = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += 256) c += sums[b];
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) c += __shfl_xor_sync(0xffffffffu, c, d);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < 8; ++w) t += s_w[w];
    s_carry = t;
  }
  __syncthreads();
  const uint32_t carry = s_carry;
  const long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t loc = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = (base + k < n) ? a[base + k] : 0u;
    loc += v[k];
  }
  uint32_t tot;
  uint32_t pre = block_excl_scan(loc, s_w, tot) + carry;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (base + k < n) a[base + k] = pre;
    pre += v[k];
  }
  if (total_out && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total_out = carry + tot;
}

static cudaError_t excl_scan(uint32_t* a, long long n, uint32_t* sums, uint32_t* total,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int nb = (int)((n + kScanTile - 1) / kScanTile);
  {
    NEXEL_PROF("scan_reduce", st);
    k_scan_reduce<<<nb, 256, 0, st>>>(a, n, sums);
  }
  {
    NEXEL_PROF("scan_final", st);
    k_scan_final<<<nb, 256, 0, st>>>(a, n, sums, total);
  }
  return cudaGetLastError();
}

// ----------------------------------------------------------- radix sort
// Stable LSD radix sort, reduce-then-scan: per pass a per-block digit
// histogram, one exclusive scan over (digit, block), and a scatter that ranks
// keys stably inside the block (warp match + per-warp digit counts), stages
// them in shared memory in digit order and writes runs out coalesced.
template <typename KeyT, int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const KeyT* __restrict__ keys,
                                                             long long n, int shift, int bits,
                                                             uint32_t* __restrict__ hist,
                                                             int nblocks,
                                                             const uint32_t* __restrict__ n_dev) {
  // n is the key count, or, with n_dev, the capacity the grid was sized for
  // and *n_dev (clamped to it) the count the device produced
  if (n_dev) n = min(n, (long long)*n_dev);
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  uint32_t mask = (1u << bits) - 1u;
  long long base = (long long)blockIdx.x * (kSortThreads * ITEMS);
#pragma unroll 4
  for (int k = 0; k < ITEMS; ++k) {
    long long i = base + (long long)k * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & mask], 1u);
  }
  __syncthreads();
  if (threadIdx.x < (1 << bits)) hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

template <typename KeyT, bool kVal, int ITEMS>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const KeyT* __restrict__ kin, KeyT* __restrict__ kout, const uint32_t* __restrict__ vin,
    uint32_t* __restrict__ vout, long long n, int shift, int bits,
    const uint32_t* __restrict__ offs, int nblocks, const uint32_t* __restrict__ n_dev) {
  // Warp w ranks the block's keys [512 w, 512 w + 512) in order (item k,
  // lane l -> key 512 w + 32 k + l) with warp-private digit counters (match
  // + leader update, no block barrier per item); one block-wide scan over
  // (digit, warp) then gives every key its place in digit order.
  extern __shared__ __align__(16) unsigned char smem[];
  KeyT* s_key = reinterpret_cast<KeyT*>(smem);
  uint32_t* s_val = reinterpret_cast<uint32_t*>(s_key + (kSortThreads * ITEMS));
  constexpr int kW = kSortThreads / 32;
  __shared__ uint32_t s_start[256], s_w[8];
  __shared__ uint32_t s_wc[kW][256];
  const int nbins = 1 << bits;
  const uint32_t mask = (uint32_t)nbins - 1u;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (n_dev) n = min(n, (long long)*n_dev);
  const long long base = (long long)blockIdx.x * (kSortThreads * ITEMS);
  const int nloc = (int)max(0LL, min((long long)(kSortThreads * ITEMS), n - base));
  for (int b = threadIdx.x; b < 256 * kW; b += kSortThreads) (&s_wc[0][0])[b] = 0;
  __syncthreads();
  KeyT key[ITEMS];
  uint32_t val[ITEMS], rank[ITEMS];
  const unsigned lt = (1u << lane) - 1u;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int li = warp * (32 * ITEMS) + k * 32 + lane;
    const bool valid = li < nloc;
    if (valid) {
      key[k] = kin[base + li];
      if (kVal) val[k] = vin[base + li];
    }
    const uint32_t d = valid ? ((uint32_t)(key[k] >> shift) & mask) : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = 0;
    if (valid) before = s_wc[warp][d];
    __syncwarp();
    rank[k] = before + __popc(peers & lt);
    if (valid && (peers & lt) == 0) s_wc[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over warps (in place) and the block total
  uint32_t tot_d = 0;
  if (threadIdx.x < 256) {
#pragma unroll
    for (int w = 0; w < kW; ++w) {
      const uint32_t c = s_wc[w][threadIdx.x];
      s_wc[w][threadIdx.x] = tot_d;
      tot_d += c;
    }
  }
  uint32_t tot;
  const uint32_t st0 = block_excl_scan(tot_d, s_w, tot);
  s_start[threadIdx.x] = st0;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int li = warp * (32 * ITEMS) + k * 32 + lane;
    if (li < nloc) {
      const uint32_t d = (uint32_t)(key[k] >> shift) & mask;
      const uint32_t pos = s_start[d] + s_wc[warp][d] + rank[k];
      s_key[pos] = key[k];
      if (kVal) s_val[pos] = val[k];
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < nloc; j += kSortThreads) {
    KeyT kk = s_key[j];
    uint32_t d = (uint32_t)(kk >> shift) & mask;
    size_t g = (size_t)offs[(size_t)d * nblocks + blockIdx.x] + (j - s_start[d]);
    kout[g] = kk;
    if (kVal) vout[g] = s_val[j];
  }
}

// Sorts n keys (and values when vin != nullptr) on bits [lo, lo + nbits).
// Returns the index (0 or 1) of the buffer pair that holds the result.  With
// n_dev the key count is read on the device (clamped to n, the capacity the
// launches are sized for), so no host synchronisation is needed.
template <typename KeyT, int ITEMS>
static cudaError_t radix_sort(KeyT* k0, KeyT* k1, uint32_t* v0, uint32_t* v1, long long n, int lo,
                              int nbits, uint32_t* hist, uint32_t* sums, cudaStream_t st,
                              int* which, const uint32_t* n_dev = nullptr) {
  *which = 0;
  if (n <= 1 || nbits <= 0) return cudaSuccess;
  int nblocks = (int)((n + (kSortThreads * ITEMS) - 1) / (kSortThreads * ITEMS));
  KeyT* kin = k0; KeyT* kout = k1;
  uint32_t* vin = v0; uint32_t* vout = v1;
  size_t smem = (size_t)(kSortThreads * ITEMS) * (sizeof(KeyT) + (v0 ? sizeof(uint32_t) : 0));
  for (int b = 0; b < nbits; b += 8) {
    int bits = std::min(8, nbits - b);
    int shift = lo + b;
    {
      NEXEL_PROF("radix_hist", st);
      k_radix_hist<KeyT, ITEMS><<<nblocks, kSortThreads, 0, st>>>(kin, n, shift, bits, hist, nblocks,
                                                                   n_dev);
    }
    cudaError_t e = excl_scan(hist, (long long)(1 << bits) * nblocks, sums, nullptr, st);
    if (e != cudaSuccess) return e;
    if (v0) {
      {
        NEXEL_PROF("radix_scatter", st);
        k_radix_scatter<KeyT, true, ITEMS><<<nblocks, kSortThreads, smem, st>>>(
            kin, kout, vin, vout, n, shift, bits, hist, nblocks, n_dev);
      }
    } else {
      {
        NEXEL_PROF("radix_scatter", st);
        k_radix_scatter<KeyT, false, ITEMS><<<nblocks, kSortThreads, smem, st>>>(
            kin, kout, nullptr, nullptr, n, shift, bits, hist, nblocks, n_dev);
      }
    }
    std::swap(kin, kout);
    std::swap(vin, vout);
    *which ^= 1;
  }
  return cudaGetLastError();
}

// ------------------------------------------- permutation, duplicate, ranges
__global__ void k_permute(int N, const uint32_t* __restrict__ did, const float4* __restrict__ geom,
                          float4* __restrict__ geom_sorted, const float4* __restrict__ aux,
                          float4* __restrict__ aux_sorted, const uint32_t* __restrict__ count,
                          uint32_t* __restrict__ offs, uint32_t* __restrict__ rank_of) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  uint32_t id = did[r];
  rank_of[id] = (uint32_t)r;  // the inverse permutation, for the backward
  const float4* s = geom + (size_t)id * kRecF4;
  float4* d = geom_sorted + (size_t)r * kRecF4;
#pragma unroll
  for (int k = 0; k < kRecF4; ++k) d[k] = s[k];
  const float4* sa = aux + (size_t)id * kAuxF4;
  float4* da = aux_sorted + (size_t)r * kAuxF4;
#pragma unroll
  for (int k = 0; k < kAuxF4; ++k) da[k] = sa[k];
  offs[r] = count[id];
}

// (k / nx, k % nx) for the small tile counts of one rectangle (k < 2^22),
// exact through the float reciprocal: (k + 1/2) / nx stays at least
// 1 / (2 nx) from an integer.
__device__ __forceinline__ int2 rect_tile(int k, int nx, float inv_nx) {
  const int q = __float2int_rz(((float)k + 0.5f) * inv_nx);
  return make_int2(k - q * nx, q);
}

template <typename KeyT>
__global__ void __launch_bounds__(256) k_duplicate(const DevCam c, int N, int rank_bits,
                                                   const uint32_t* __restrict__ did,
                                                   const uint2* __restrict__ rect,
                                                   const float4* __restrict__ conic,
                                                   const uint4* __restrict__ tmask,
                                                   const uint32_t* __restrict__ offs,
                                                   const uint32_t* __restrict__ count,
                                                   KeyT* __restrict__ keys, uint32_t cap) {
  // one warp per surfel (rank order): the lanes take 32 tiles of the
  // rectangle at a time and the passing ones are written in tile order; the
  // decisions come from the counting pass's mask when the rectangle has at
  // most 128 tiles, else the test runs again.  Instances at or beyond the
  // key buffer's capacity are dropped (the device-count path flags that).
  const int lane = threadIdx.x & 31;
  const int r = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (r >= N) return;
  const uint32_t id = did[r];
  if (count[id] == 0) return;
  const uint2 rc = rect[id];
  const int tx0 = rc.x & 0xFFFF, tx1 = rc.x >> 16, ty0 = rc.y & 0xFFFF, ty1 = rc.y >> 16;
  const int nx = tx1 - tx0 + 1, nt = nx * (ty1 - ty0 + 1);
  const float inv_nx = 1.f / (float)nx;
  size_t o = offs[r];
  if (nt <= 128) {
    const uint4 mq = tmask[id];
    const uint32_t mw[4] = {mq.x, mq.y, mq.z, mq.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (32 * i >= nt) break;
      const unsigned m = mw[i];
      if ((m >> lane) & 1u) {
        const int2 t2 = rect_tile(32 * i + lane, nx, inv_nx);
        const KeyT tile = (KeyT)((ty0 + t2.y) * c.tiles_x + tx0 + t2.x);
        const size_t at = o + __popc(m & ((1u << lane) - 1u));
        if (at < cap) keys[at] = (tile << rank_bits) | (KeyT)r;
      }
      o += __popc(m);
    }
    return;
  }
  const TileConic kc = load_conic(conic, id);
  for (int b = 0; b < nt; b += 32) {
    const int k = b + lane;
    const int2 t2 = rect_tile(k, nx, inv_nx);
    const int tx = tx0 + t2.x, ty = ty0 + t2.y;
    const bool hit = k < nt && tile_may_hit(kc, tx, ty, c.W, c.H);
    const unsigned m = __ballot_sync(0xffffffffu, hit);
    if (hit) {
      const KeyT tile = (KeyT)(ty * c.tiles_x + tx);
      const size_t at = o + __popc(m & ((1u << lane) - 1u));
      if (at < cap) keys[at] = (tile << rank_bits) | (KeyT)r;
    }
    o += __popc(m);
  }
}

// Exact instance count of each surfel: the tiles of its rectangle that pass
// tile_may_hit (original order), and, for rectangles of at most 128 tiles,
// the pass/fail bits in rectangle order for k_duplicate.  With mwords, the
// pass/fail bits of every rectangle are also stored, one word per 32 tiles
// of rectangle order, at the surfel's offset moff[i] (an exclusive scan of
// the word counts), when they fit below cap_words.
// One warp per 32 consecutive surfels: lane i loads surfel i's visibility,
// rectangle, support conic and word offset (coalesced, all at once), then
// the warp walks its visible surfels one by one (their data broadcast by
// shuffles), lane b testing tile b of each 32-tile word; the surfel's own
// lane keeps its count and mask for one coalesced store at the end.
__global__ void __launch_bounds__(256) k_tile_count(const DevCam c, int N,
                                                    const uint2* __restrict__ rect,
                                                    const float4* __restrict__ conic,
                                                    uint4* __restrict__ tmask,
                                                    uint32_t* __restrict__ count,
                                                    const uint32_t* __restrict__ moff,
                                                    uint32_t* __restrict__ mwords,
                                                    uint32_t cap_words) {
  const int lane = threadIdx.x & 31;
  const long long i0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) & ~31LL;
  if (i0 >= N) return;  // warp-uniform
  const long long i = i0 + lane;
  const bool vis = i < N && count[i] != 0;
  uint2 rc_own = make_uint2(0u, 0u);
  uint32_t off_own = 0u;
  float4 ka = make_float4(0.f, 0.f, 0.f, 0.f), kb = ka, kcc = ka;
  if (vis) {
    rc_own = rect[i];
    ka = conic[3 * i];
    kb = conic[3 * i + 1];
    kcc = conic[3 * i + 2];
    if (mwords) off_own = moff[i];
  }
  uint32_t my_n = 0u;
  uint4 my_mask = make_uint4(0u, 0u, 0u, 0u);
  for (unsigned todo = __ballot_sync(0xffffffffu, vis); todo; todo &= todo - 1u) {
    const int sl = __ffs(todo) - 1;  // the surfel's lane (warp-uniform)
    const uint32_t rx = __shfl_sync(0xffffffffu, rc_own.x, sl);
    const uint32_t ry = __shfl_sync(0xffffffffu, rc_own.y, sl);
    const TileConic kc = {__shfl_sync(0xffffffffu, ka.x, sl),  __shfl_sync(0xffffffffu, ka.y, sl),
                          __shfl_sync(0xffffffffu, ka.z, sl),  __shfl_sync(0xffffffffu, ka.w, sl),
                          __shfl_sync(0xffffffffu, kb.x, sl),  __shfl_sync(0xffffffffu, kb.y, sl),
                          __shfl_sync(0xffffffffu, kb.z, sl),  __shfl_sync(0xffffffffu, kb.w, sl),
                          __shfl_sync(0xffffffffu, kcc.x, sl), __shfl_sync(0xffffffffu, kcc.y, sl),
                          __shfl_sync(0xffffffffu, kcc.z, sl), __shfl_sync(0xffffffffu, kcc.w, sl)};
    const int tx0 = rx & 0xFFFF, tx1 = rx >> 16, ty0 = ry & 0xFFFF, ty1 = ry >> 16;
    const int nx = tx1 - tx0 + 1, nt = nx * (ty1 - ty0 + 1);
    const float inv_nx = 1.f / (float)nx;
    const uint32_t words = (uint32_t)(nt + 31) / 32;
    uint32_t* mw_out = nullptr;
    if (mwords) {
      const uint32_t off = __shfl_sync(0xffffffffu, off_own, sl);
      if (off <= cap_words && words <= cap_words - off) mw_out = mwords + off;
    }
    uint32_t n = 0;
    if (nt <= 128) {
      uint32_t mw[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        if (32 * w >= nt) break;  // warp-uniform
        const int k = 32 * w + lane;
        const int2 t2 = rect_tile(k, nx, inv_nx);
        const bool hit = k < nt && tile_may_hit(kc, tx0 + t2.x, ty0 + t2.y, c.W, c.H);
        mw[w] = __ballot_sync(0xffffffffu, hit);
        n += __popc(mw[w]);
      }
      if (lane == sl) my_mask = make_uint4(mw[0], mw[1], mw[2], mw[3]);
      if (mw_out && lane < (int)words)
        mw_out[lane] = lane == 0 ? mw[0] : lane == 1 ? mw[1] : lane == 2 ? mw[2] : mw[3];
    } else {
      for (int b = 0; b < nt; b += 32) {  // warp-uniform
        const int k = b + lane;
        const int2 t2 = rect_tile(k, nx, inv_nx);
        const bool hit = k < nt && tile_may_hit(kc, tx0 + t2.x, ty0 + t2.y, c.W, c.H);
        const uint32_t m = __ballot_sync(0xffffffffu, hit);
        n += __popc(m);
        if (mw_out && lane == 0) mw_out[b >> 5] = m;
      }
    }
    if (lane == sl) my_n = n;
  }
  if (vis) {
    const uint32_t nt = ((rc_own.x >> 16) - (rc_own.x & 0xFFFF) + 1) *
                        ((rc_own.y >> 16) - (rc_own.y & 0xFFFF) + 1);
    if (nt <= 128) tmask[i] = my_mask;
    count[i] = my_n;
  }
}

// Word count of each surfel's rectangle decisions (one per 32 tiles; none
// for a culled surfel), to be scanned into the offsets of k_tile_count.
__global__ void k_mask_words(int N, const uint2* __restrict__ rect,
                             const uint32_t* __restrict__ count, uint32_t* __restrict__ words) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint2 rc = rect[i];
  const uint32_t nt = ((rc.x >> 16) - (rc.x & 0xFFFF) + 1) * ((rc.y >> 16) - (rc.y & 0xFFFF) + 1);
  words[i] = count[i] == 0 ? 0u : (nt + 31) / 32;
}

// ------------------------------------------------ direct placement by tile
// The per-tile lists are the instances of the depth-rank-ordered surfels,
// split by tile and kept in rank order.  Instead of sorting the rank-ordered
// instance sequence on its tile bits, every instance is written straight to
// its final slot:
//   slot(r, t) = start(t) + #{instances of tile t from surfels of rank < r}.
// Ranks come in blocks of kPlaceRanks: k_place_count counts each block's
// instances per tile (shared-memory counters), k_place_colscan turns the
// [block][tile] counts into per-tile exclusive prefixes over the blocks and
// per-tile totals, whose exclusive scan gives start(t).  k_place_write then
// walks its block in groups of 64 ranks: two 32-bit masks per tile record
// which ranks of the group cover the tile, so an instance's place within
// the group is a popcount of the lower bits, and the group's counts advance
// the tile's running base.  The result is the same sequence as the stable
// sort, bit for bit.  Both kernels read the tile decisions k_tile_count
// stored (one word per 32 rectangle tiles), so the tile test runs once.

// The block's kPlaceRanks ranks staged in shared memory (tile rectangle,
// surfel id or ~0 when the surfel has no instance, offset of its decision
// words), loaded with all threads at once so that the walks below read no
// per-rank data from global memory.
struct PlaceRanks {
  uint2* rect;
  uint32_t* id;
  uint32_t* off;
};
constexpr size_t kPlaceStageBytes = (size_t)kPlaceRanks * (8 + 4 + 4);
constexpr int kPlaceStageWords = 8192;  // decision words the write kernel stages
static_assert(kPlaceThreads == kPlaceRanks, "the count kernel scans one rank per thread");

__device__ __forceinline__ PlaceRanks stage_ranks(unsigned char* smem, long long r0, int N,
                                                  const uint32_t* __restrict__ did,
                                                  const uint2* __restrict__ rect,
                                                  const uint32_t* __restrict__ count,
                                                  const uint32_t* __restrict__ moff) {
  PlaceRanks pr;
  pr.rect = reinterpret_cast<uint2*>(smem);
  pr.id = reinterpret_cast<uint32_t*>(smem + (size_t)kPlaceRanks * 8);
  pr.off = reinterpret_cast<uint32_t*>(smem + (size_t)kPlaceRanks * 12);
  for (int i = threadIdx.x; i < kPlaceRanks; i += blockDim.x) {
    const long long r = r0 + i;
    uint32_t id = ~0u;
    if (r < N) {
      id = did[r];
      pr.rect[i] = rect[id];
      pr.off[i] = moff[id];
      if (count[id] == 0) id = ~0u;
    }
    pr.id[i] = id;
  }
  return pr;
}

__device__ __forceinline__ uint32_t rect_words(uint2 rc) {
  const uint32_t nt = ((rc.x >> 16) - (rc.x & 0xFFFF) + 1) * ((rc.y >> 16) - (rc.y & 0xFFFF) + 1);
  return (nt + 31) / 32;
}

// Decision word w (rectangle tiles 32 w .. 32 w + 31) of a staged surfel,
// from one thread: stored by k_tile_count when it fitted, else the same
// tests again.
__device__ __forceinline__ uint32_t rect_word(const DevCam& c, uint32_t id, uint2 rc,
                                              uint32_t off, const uint32_t* __restrict__ mwords,
                                              uint32_t cap_words,
                                              const float4* __restrict__ conic, int w) {
  const int tx0 = rc.x & 0xFFFF, tx1 = rc.x >> 16, ty0 = rc.y & 0xFFFF, ty1 = rc.y >> 16;
  const int nx = tx1 - tx0 + 1, nt = nx * (ty1 - ty0 + 1);
  const uint32_t words = (uint32_t)(nt + 31) / 32;
  if (off <= cap_words && words <= cap_words - off) return mwords[off + w];
  const float inv_nx = 1.f / (float)nx;
  const TileConic kc = load_conic(conic, id);
  uint32_t m = 0u;
  for (int b = 0; b < 32; ++b) {
    const int k = 32 * w + b;
    if (k >= nt) break;
    const int2 t2 = rect_tile(k, nx, inv_nx);
    if (tile_may_hit(kc, tx0 + t2.x, ty0 + t2.y, c.W, c.H)) m |= 1u << b;
  }
  return m;
}

// Calls f(t) for every passing tile of decision word w of a rectangle.
template <typename F>
__device__ __forceinline__ void for_word_tiles(const DevCam& c, uint2 rc, uint32_t m, int w,
                                               F&& f) {
  const int tx0 = rc.x & 0xFFFF, ty0 = rc.y & 0xFFFF;
  const int nx = (rc.x >> 16) - tx0 + 1;
  const float inv_nx = 1.f / (float)nx;
  while (m) {
    const int b = __ffs(m) - 1;
    m &= m - 1u;
    const int2 t2 = rect_tile(32 * w + b, nx, inv_nx);
    f((ty0 + t2.y) * c.tiles_x + tx0 + t2.x);
  }
}

// Block-wide exclusive prefix of the staged ranks' decision-word counts into
// pre[0 .. kPlaceRanks] (one rank per thread; wsum: kPlaceThreads / 32 words).
__device__ __forceinline__ void rank_word_prefix(const PlaceRanks& pr, uint32_t* pre,
                                                 uint32_t* wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t v = pr.id[threadIdx.x] == ~0u ? 0u : rect_words(pr.rect[threadIdx.x]);
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  if (lane == 31) wsum[warp] = v;
  __syncthreads();
  uint32_t carry = 0;
  for (int w = 0; w < warp; ++w) carry += wsum[w];
  pre[threadIdx.x + 1] = carry + v;
  if (threadIdx.x == 0) pre[0] = 0u;
  __syncthreads();
}

// The rank i of word k of the block: pre[i] <= k < pre[i + 1].
__device__ __forceinline__ int word_rank(const uint32_t* pre, uint32_t k) {
  int i = 0;
#pragma unroll
  for (int step = kPlaceRanks / 2; step > 0; step >>= 1)
    if (pre[i + step] <= k) i += step;
  return i;
}

// Decision word w (rectangle tiles 32 w .. 32 w + 31) of a staged surfel,
// called by a whole warp with the same arguments: the word k_tile_count
// stored when it fitted, else the same tests again (lane b tests tile
// 32 w + b).  Lane b also gets the index of its tile in *tile.
__device__ __forceinline__ uint32_t rect_word_warp(const DevCam& c, uint32_t id, uint2 rc,
                                                   uint32_t off,
                                                   const uint32_t* __restrict__ mwords,
                                                   uint32_t cap_words,
                                                   const float4* __restrict__ conic, int w,
                                                   int lane, int* tile) {
  const int tx0 = rc.x & 0xFFFF, tx1 = rc.x >> 16, ty0 = rc.y & 0xFFFF, ty1 = rc.y >> 16;
  const int nx = tx1 - tx0 + 1, nt = nx * (ty1 - ty0 + 1);
  const int k = 32 * w + lane;
  const int2 t2 = rect_tile(k, nx, 1.f / (float)nx);
  *tile = (ty0 + t2.y) * c.tiles_x + tx0 + t2.x;
  const uint32_t words = (uint32_t)(nt + 31) / 32;
  if (off <= cap_words && words <= cap_words - off) return mwords[off + w];
  const bool hit = k < nt && tile_may_hit(load_conic(conic, id), tx0 + t2.x, ty0 + t2.y, c.W, c.H);
  return __ballot_sync(0xffffffffu, hit);
}

__global__ void __launch_bounds__(kPlaceThreads) k_place_count(
    const DevCam c, int N, int n_tiles, const uint32_t* __restrict__ did,
    const uint2* __restrict__ rect, const float4* __restrict__ conic,
    const uint32_t* __restrict__ count, const uint32_t* __restrict__ moff,
    const uint32_t* __restrict__ mwords, uint32_t cap_words, uint32_t* __restrict__ M) {
  extern __shared__ __align__(16) unsigned char s_count_smem[];
  __shared__ uint32_t s_pre[kPlaceRanks + 1];  // decision words per rank, exclusive prefix
  __shared__ uint32_t s_wsum[kPlaceThreads / 32];
  const long long r0 = (long long)blockIdx.x * kPlaceRanks;
  const PlaceRanks pr = stage_ranks(s_count_smem, r0, N, did, rect, count, moff);
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(s_count_smem + kPlaceStageBytes);
  for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) s_cnt[t] = 0u;
  __syncthreads();
  rank_word_prefix(pr, s_pre, s_wsum);
  // every (rank, decision word) pair of the block, spread over the threads
  const uint32_t n_items = s_pre[kPlaceRanks];
  for (uint32_t k = threadIdx.x; k < n_items; k += blockDim.x) {
    const int i = word_rank(s_pre, k);
    const int w = (int)(k - s_pre[i]);
    const uint2 rc = pr.rect[i];
    const uint32_t m = rect_word(c, pr.id[i], rc, pr.off[i], mwords, cap_words, conic, w);
    for_word_tiles(c, rc, m, w, [&](int t) { atomicAdd(&s_cnt[t], 1u); });
  }
  __syncthreads();
  uint32_t* row = M + (size_t)blockIdx.x * n_tiles;
  for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) row[t] = s_cnt[t];
}

// Per tile: exclusive prefix of the counts over the rank blocks, in place,
// and the tile's total.  A CTA takes 32 tiles (lane = tile, so every load
// is one 128-byte row piece) and splits the rank blocks into 32 chunks, one
// per warp: each warp sums its chunk, the chunk sums are scanned through
// shared memory, and each warp then rewrites its chunk from its own base.
constexpr int kColscanWarps = 32;
__global__ void __launch_bounds__(kColscanWarps * 32) k_place_colscan(uint32_t* __restrict__ M,
                                                                     int nb, int n_tiles,
                                                                     uint32_t* __restrict__ tot) {
  __shared__ uint32_t s_part[kColscanWarps][33];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = blockIdx.x * 32 + lane;
  const int chunk = (nb + kColscanWarps - 1) / kColscanWarps;
  const int b0 = min(nb, warp * chunk), b1 = min(nb, b0 + chunk);
  uint32_t sum = 0;
  if (t < n_tiles) {
    int b = b0;
    for (; b + 8 <= b1; b += 8) {  // eight independent loads in flight
      uint32_t v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = M[(size_t)(b + k) * n_tiles + t];
#pragma unroll
      for (int k = 0; k < 8; ++k) sum += v[k];
    }
    for (; b < b1; ++b) sum += M[(size_t)b * n_tiles + t];
  }
  s_part[warp][lane] = sum;
  __syncthreads();
  if (t >= n_tiles) return;
  uint32_t run = 0;
  for (int w = 0; w < warp; ++w) run += s_part[w][lane];
  if (warp == kColscanWarps - 1) tot[t] = run + sum;
  int b = b0;
  for (; b + 8 <= b1; b += 8) {
    uint32_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = M[(size_t)(b + k) * n_tiles + t];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      M[(size_t)(b + k) * n_tiles + t] = run;
      run += v[k];
    }
  }
  for (; b < b1; ++b) {
    const uint32_t v = M[(size_t)b * n_tiles + t];
    M[(size_t)b * n_tiles + t] = run;
    run += v;
  }
}

// Tile ranges from the exclusive starts; a total above the key buffer's
// capacity (instances dropped) is flagged and the ranges are clamped to it.
__global__ void k_place_ranges(int n_tiles, const uint32_t* __restrict__ start,
                               const uint32_t* __restrict__ total, uint32_t cap,
                               uint2* __restrict__ ranges, int* __restrict__ status) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tiles) return;
  const uint32_t all = *total;
  if (t == 0 && all > cap && status) atomicOr(status, kStatusCapacity);
  const uint32_t a = start[t], e = t + 1 < n_tiles ? start[t + 1] : all;
  ranges[t] = make_uint2(min(a, cap), min(e, cap));
}

template <typename KeyT>
__global__ void __launch_bounds__(kPlaceThreads) k_place_write(
    const DevCam c, int N, int n_tiles, int tile_shift, const uint32_t* __restrict__ did,
    const uint2* __restrict__ rect, const float4* __restrict__ conic,
    const uint32_t* __restrict__ count, const uint32_t* __restrict__ moff,
    const uint32_t* __restrict__ mwords, uint32_t cap_words, const uint32_t* __restrict__ M,
    const uint32_t* __restrict__ start, KeyT* __restrict__ keys, uint32_t cap) {
  extern __shared__ __align__(16) unsigned char s_write_smem[];
  __shared__ uint32_t s_pre[kPlaceRanks + 1];  // decision words per rank, exclusive prefix
  __shared__ uint32_t s_wsum[kPlaceThreads / 32];
  const long long r0 = (long long)blockIdx.x * kPlaceRanks;
  const PlaceRanks pr = stage_ranks(s_write_smem, r0, N, did, rect, count, moff);
  // the block's first kPlaceStageWords decision words and their ranks
  uint32_t* s_word = reinterpret_cast<uint32_t*>(s_write_smem + kPlaceStageBytes);
  uint16_t* s_wrank = reinterpret_cast<uint16_t*>(s_word + kPlaceStageWords);
  // ranks 0-31 and 32-63 of the current group covering each tile, and each
  // tile's next slot
  uint32_t* s_lo = reinterpret_cast<uint32_t*>(s_wrank + kPlaceStageWords);
  uint32_t* s_hi = s_lo + n_tiles;
  uint32_t* s_base = s_hi + n_tiles;
  const uint32_t* row = M + (size_t)blockIdx.x * n_tiles;
  for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) {
    s_base[t] = start[t] + row[t];
    s_lo[t] = 0u;
    s_hi[t] = 0u;
  }
  __syncthreads();
  rank_word_prefix(pr, s_pre, s_wsum);
  const uint32_t n_items = s_pre[kPlaceRanks];
  for (uint32_t k = threadIdx.x; k < min(n_items, (uint32_t)kPlaceStageWords); k += blockDim.x) {
    const int i = word_rank(s_pre, k);
    s_word[k] = rect_word(c, pr.id[i], pr.rect[i], pr.off[i], mwords, cap_words, conic,
                          (int)(k - s_pre[i]));
    s_wrank[k] = (uint16_t)i;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int g = 0; g < kPlaceRanks; g += 64) {
    if (r0 + g >= N) break;  // block-uniform
    // the group's decision words, one warp per word and one lane per tile:
    // first which ranks cover each tile, then every instance's slot (the
    // tile's base plus the group's lower ranks that cover it)
    const uint32_t k0 = s_pre[g], k1 = s_pre[g + 64];
    for (int pass = 0; pass < 2; ++pass) {
      for (uint32_t k = k0 + warp; k < k1; k += kPlaceThreads / 32) {  // warp-uniform
        int i, t;
        uint32_t m;
        if (k < (uint32_t)kPlaceStageWords) {
          i = s_wrank[k];
          const uint2 rc = pr.rect[i];
          const int tx0 = rc.x & 0xFFFF, ty0 = rc.y & 0xFFFF, nx = (rc.x >> 16) - tx0 + 1;
          const int2 t2 = rect_tile(32 * (int)(k - s_pre[i]) + lane, nx, 1.f / (float)nx);
          t = (ty0 + t2.y) * c.tiles_x + tx0 + t2.x;
          m = s_word[k];
        } else {
          i = word_rank(s_pre, k);
          m = rect_word_warp(c, pr.id[i], pr.rect[i], pr.off[i], mwords, cap_words, conic,
                             (int)(k - s_pre[i]), lane, &t);
        }
        if (((m >> lane) & 1u) == 0u) continue;
        const int gi = i - g;  // rank within the group, 0 .. 63
        if (pass == 0) {
          if (gi < 32) atomicOr(&s_lo[t], 1u << gi);
          else atomicOr(&s_hi[t], 1u << (gi - 32));
        } else {
          const uint32_t lower = gi < 32 ? (uint32_t)__popc(s_lo[t] & ((1u << gi) - 1u))
                                         : (uint32_t)__popc(s_lo[t]) +
                                               (uint32_t)__popc(s_hi[t] & ((1u << (gi - 32)) - 1u));
          const uint32_t at = s_base[t] + lower;
          // (tile << rank bits | rank), or the rank alone (tile_shift 32)
          if (at < cap)
            keys[at] = (tile_shift < 32 ? (KeyT)t << tile_shift : (KeyT)0) | (KeyT)(r0 + i);
        }
      }
      __syncthreads();
    }
    for (int t = threadIdx.x; t < n_tiles; t += blockDim.x) {
      s_base[t] += (uint32_t)(__popc(s_lo[t]) + __popc(s_hi[t]));
      s_lo[t] = 0u;
      s_hi[t] = 0u;
    }
    __syncthreads();
  }
}

template <typename KeyT>
__global__ void k_ranges(long long n, int rank_bits, const KeyT* __restrict__ keys,
                         uint2* __restrict__ ranges, const uint32_t* __restrict__ n_dev,
                         int* __restrict__ status) {
  // with n_dev: n is the capacity and *n_dev the instance count; a count
  // above the capacity (instances dropped by k_duplicate) is flagged
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n_dev) {
    const long long want = (long long)*n_dev;
    if (i == 0 && want > n && status) atomicOr(status, kStatusCapacity);
    n = min(n, want);
  }
  if (i >= n) return;
  uint32_t t = (uint32_t)(keys[i] >> rank_bits);
  if (i == 0 || (uint32_t)(keys[i - 1] >> rank_bits) != t) ranges[t].x = (uint32_t)i;
  if (i == n - 1 || (uint32_t)(keys[i + 1] >> rank_bits) != t) ranges[t].y = (uint32_t)(i + 1);
}

// ------------------------------------------------------ shared primitives
cudaError_t sort_pairs_u32(uint32_t* k0, uint32_t* k1, uint32_t* v0, uint32_t* v1, long long n,
                           uint32_t* hist, uint32_t* sums, cudaStream_t st, int* which) {
  return radix_sort<uint32_t, kSortItemsDepth>(k0, k1, v0, v1, n, 0, 32, hist, sums, st, which);
}

cudaError_t exclusive_scan_u32(uint32_t* a, long long n, uint32_t* sums, uint32_t* total,
                               cudaStream_t st) {
  return excl_scan(a, n, sums, total, st);
}

// ------------------------------------------------------------- launchers
cudaError_t launch_preprocess(const DevCam& c, const nexel_settings& s, int N, const float* mu,
                              const float* quat, const float* scale, const float* opacity,
                              const float* gamma, const float* color, char* ws,
                              const WsLayout& L, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  {
    NEXEL_PROF("preprocess", st);
    k_preprocess<<<(N + 255) / 256, 256, 0, st>>>(
        c, s.alpha_min, s.sh_degree, N, mu, quat, scale, opacity, gamma, color,
        (float4*)(ws + L.geom_orig),
        (float4*)(ws + L.aux_orig), (uint32_t*)(ws + L.dkey0), (uint32_t*)(ws + L.did0),
        (uint2*)(ws + L.rect), (float4*)(ws + L.conic), (uint32_t*)(ws + L.count),
        (float*)(ws + L.shj), (uint32_t*)(ws + L.counters + kCountersNonFinite),
        (int*)(ws + L.counters + kStatusOffset));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  uint32_t* moff = nullptr;
  if (L.place_ok) {
    // offsets of the stored tile decisions (one word per 32 rectangle tiles)
    moff = (uint32_t*)(ws + L.mword_off);
    {
      NEXEL_PROF("mask_words", st);
      k_mask_words<<<(N + 255) / 256, 256, 0, st>>>(N, (const uint2*)(ws + L.rect),
                                                    (const uint32_t*)(ws + L.count), moff);
    }
    e = cudaGetLastError();
    if (e == cudaSuccess)
      e = excl_scan(moff, N, (uint32_t*)(ws + L.scan_sums),
                    (uint32_t*)(ws + L.counters + kCountersMaskWords), st);
    if (e != cudaSuccess) return e;
  }
  {
    NEXEL_PROF("tile_count", st);
    k_tile_count<<<(unsigned)(((long long)N + 255) / 256), 256, 0, st>>>(
        c, N, (uint2*)(ws + L.rect), (float4*)(ws + L.conic), (uint4*)(ws + L.tmask),
        (uint32_t*)(ws + L.count), moff, moff ? (uint32_t*)(ws + L.mwords) : nullptr,
        (uint32_t)L.mword_cap);
  }
  return cudaGetLastError();
}

cudaError_t launch_depth_sort(int N, char* ws, const WsLayout& L, cudaStream_t st) {
  int which = 0;
  // the depth sort (N keys) uses 1024-key tiles, for parallelism at a few
  // hundred thousand surfels
  cudaError_t e = radix_sort<uint32_t, kSortItemsDepth>((uint32_t*)(ws + L.dkey0), (uint32_t*)(ws + L.dkey1),
                                       (uint32_t*)(ws + L.did0), (uint32_t*)(ws + L.did1), N, 0,
                                       32, (uint32_t*)(ws + L.hist), (uint32_t*)(ws + L.scan_sums),
                                       st, &which);
  // 4 passes: the result is back in buffer 0
  (void)which;
  return e;
}

cudaError_t launch_count_scan(int N, char* ws, const WsLayout& L, cudaStream_t st) {
  if (N <= 0) return cudaSuccess;
  {
    NEXEL_PROF("permute", st);
    k_permute<<<(N + 255) / 256, 256, 0, st>>>(N, (uint32_t*)(ws + L.did0),
                                               (float4*)(ws + L.geom_orig),
                                               (float4*)(ws + L.geom_sorted),
                                               (float4*)(ws + L.aux_orig),
                                               (float4*)(ws + L.aux_sorted),
                                               (uint32_t*)(ws + L.count), (uint32_t*)(ws + L.offs),
                                               (uint32_t*)(ws + L.did1));
  }
  uint32_t* counters = (uint32_t*)(ws + L.counters);
  return excl_scan((uint32_t*)(ws + L.offs), N, (uint32_t*)(ws + L.scan_sums), counters + 1, st);
}

// Direct placement (32-bit keys, at most kPlaceMaxTiles tiles): the
// instances land in inst0 in their final order; no sort passes.
static cudaError_t binning_place(const DevCam& c, int N, char* ws, const WsLayout& L,
                                 cudaStream_t st) {
  const int n_tiles = L.n_tiles;
  uint32_t* M = (uint32_t*)(ws + L.place);
  uint32_t* tstart = (uint32_t*)(ws + L.place_tiles);
  uint32_t* total = (uint32_t*)(ws + L.counters + kCountersPlaced);
  const unsigned nb = (unsigned)((N + kPlaceRanks - 1) / kPlaceRanks);
  const uint32_t cap = (uint32_t)std::min<long long>(L.cap, 0xFFFFFFFFLL);
  const uint32_t* did = (const uint32_t*)(ws + L.did0);
  const uint2* rect = (const uint2*)(ws + L.rect);
  const float4* conic = (const float4*)(ws + L.conic);
  const uint32_t* count = (const uint32_t*)(ws + L.count);
  const uint32_t* moff = (const uint32_t*)(ws + L.mword_off);
  const uint32_t* mwords = (const uint32_t*)(ws + L.mwords);
  const uint32_t cap_words = (uint32_t)L.mword_cap;
  cudaError_t e = cudaSuccess;
  const size_t smem_count = kPlaceStageBytes + (size_t)n_tiles * 4;
  const size_t smem_write =
      kPlaceStageBytes + (size_t)kPlaceStageWords * 6 + (size_t)n_tiles * 12;
  if (N > 0) e = cudaFuncSetAttribute(k_place_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem_count);
  if (e == cudaSuccess && N > 0) {
    NEXEL_PROF("place_count", st);
    k_place_count<<<nb, kPlaceThreads, smem_count, st>>>(c, N, n_tiles, did, rect, conic, count,
                                                         moff, mwords, cap_words, M);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && N > 0) {
    NEXEL_PROF("place_colscan", st);
    k_place_colscan<<<(n_tiles + 31) / 32, kColscanWarps * 32, 0, st>>>(M, (int)nb, n_tiles,
                                                                        tstart);
    e = cudaGetLastError();
  } else if (e == cudaSuccess) {
    e = cudaMemsetAsync(tstart, 0, (size_t)n_tiles * 4, st);
  }
  if (e == cudaSuccess) e = excl_scan(tstart, n_tiles, (uint32_t*)(ws + L.scan_sums), total, st);
  if (e == cudaSuccess) {
    NEXEL_PROF("tile_ranges", st);
    k_place_ranges<<<(n_tiles + 255) / 256, 256, 0, st>>>(
        n_tiles, tstart, total, cap, (uint2*)(ws + L.ranges),
        (int*)(ws + L.counters + kStatusOffset));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && N > 0)
    e = cudaFuncSetAttribute(k_place_write<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_write);
  if (e == cudaSuccess && N > 0) {
    NEXEL_PROF("place_write", st);
    k_place_write<uint32_t><<<nb, kPlaceThreads, smem_write, st>>>(
        c, N, n_tiles, L.rank_only ? 32 : L.rank_bits, did, rect, conic, count, moff, mwords,
        cap_words, M, tstart, (uint32_t*)(ws + L.inst0), cap);
    e = cudaGetLastError();
  }
  return e;
}

template <typename KeyT>
static cudaError_t binning_t(const DevCam& c, int N, long long n_inst, char* ws, const WsLayout& L,
                             cudaStream_t st) {
  // n_inst < 0: the count stays on the device; every launch is sized for the
  // capacity and reads the count the scan wrote.
  const bool dev_count = n_inst < 0;
  const uint32_t* n_dev = dev_count ? (const uint32_t*)(ws + L.counters + kCountersInst) : nullptr;
  const long long n_launch = dev_count ? L.cap : n_inst;
  // The duplicate step writes into the buffer that makes the last sort pass
  // land in inst0, which is where the collection kernels read.
  int passes = (n_launch > 1 && L.tile_bits > 0) ? L.tile_passes : 0;
  KeyT* k0 = (KeyT*)(ws + ((passes & 1) ? L.inst1 : L.inst0));
  KeyT* k1 = (KeyT*)(ws + ((passes & 1) ? L.inst0 : L.inst1));
  int rb = L.key64 ? 32 : L.rank_bits;
  if (N > 0) {
    NEXEL_PROF("duplicate", st);
    k_duplicate<KeyT><<<(unsigned)(((long long)N * 32 + 255) / 256), 256, 0, st>>>(
        c, N, rb, (uint32_t*)(ws + L.did0), (uint2*)(ws + L.rect), (float4*)(ws + L.conic),
        (const uint4*)(ws + L.tmask), (uint32_t*)(ws + L.offs), (uint32_t*)(ws + L.count), k0,
        (uint32_t)std::min<long long>(L.cap, 0xFFFFFFFFLL));
  }
  int which = 0;
  cudaError_t e = radix_sort<KeyT, kSortItems>(k0, k1, nullptr, nullptr, n_launch, rb, L.tile_bits,
                                   (uint32_t*)(ws + L.hist), (uint32_t*)(ws + L.scan_sums), st,
                                   &which, n_dev);
  if (e != cudaSuccess) return e;
  KeyT* res = which ? k1 : k0;
  if ((char*)res != ws + L.inst0) return cudaErrorUnknown;
  e = cudaMemsetAsync(ws + L.ranges, 0, sizeof(uint2) * (size_t)L.n_tiles, st);
  if (e != cudaSuccess) return e;
  if (n_launch > 0)
    {
      NEXEL_PROF("tile_ranges", st);
      k_ranges<KeyT><<<(unsigned)((n_launch + 255) / 256), 256, 0, st>>>(
          n_launch, rb, res, (uint2*)(ws + L.ranges), n_dev,
          (int*)(ws + L.counters + kStatusOffset));
    }
  return cudaGetLastError();
}

cudaError_t launch_binning(const DevCam& c, int N, long long n_inst, char* ws, const WsLayout& L,
                           cudaStream_t st) {
  if (L.place_ok) return binning_place(c, N, ws, L, st);
  if (L.key64) return binning_t<unsigned long long>(c, N, n_inst, ws, L, st);
  return binning_t<uint32_t>(c, N, n_inst, ws, L, st);
}

// ------------------------------------------------------ preprocess backward
// The collection backward accumulates, per surfel (rank order), the
// gradient with respect to its camera-space frame: mu_c, v1_c, v2_c, n_c,
// sigma, opacity, gamma and colour.  Here those are rotated back to world
// space (x_c = R x + t, so dL/dx = R^T dL/dx_c) and the three frame columns
// are taken through the rotation of the normalised quaternion and the
// normalisation itself.
template <bool kAtomic>
__device__ __forceinline__ void acc(float* p, float v) {
  if (kAtomic) atomicAdd(p, v);
  else *p += v;
}

// One thread per surfel in original order (its parameters and gradients
// are read and written coalesced); its rank, from the inverse permutation
// the forward left, locates its 64-byte gradient record and frame record.
// kAtomic: views rendered concurrently add into the same gradients.
template <bool kAtomic>
__global__ void k_preprocess_bwd(DevCam c, int N, int sh_degree, const float* __restrict__ mu,
                                 const float* __restrict__ shj, const float* __restrict__ quat,
                                 const uint32_t* __restrict__ rank_of,
                                 const uint32_t* __restrict__ dkey,
                                 const float* __restrict__ gs, const float4* __restrict__ aux,
                                 float* __restrict__ d_mu,
                                 float* __restrict__ d_quat, float* __restrict__ d_scale,
                                 float* __restrict__ d_opac, float* __restrict__ d_gamma,
                                 float* __restrict__ d_color) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint32_t r = rank_of[i];
  if (dkey[r] == 0xFFFFFFFFu) return;  // culled: no gradient
  // the collection backward's sums over the surfel's pixels, turned into
  // camera-space gradients with the surfel's frame (aux: v1, v2, n and the
  // reciprocal scales; the hit offset in the plane is u s1 v1 + v s2 v2)
  const float4* g4 = reinterpret_cast<const float4*>(gs + (size_t)r * kGradStride);
  const float4 ga = g4[0], gb = g4[1], gc = g4[2], gd = g4[3];
  const float g[15] = {ga.x, ga.y, ga.z, ga.w, gb.x, gb.y, gb.z, gb.w,
                       gc.x, gc.y, gc.z, gc.w, gd.x, gd.y, gd.z};
  const float4 a1 = aux[(size_t)r * kAuxF4 + 1], a2 = aux[(size_t)r * kAuxF4 + 2],
               a3 = aux[(size_t)r * kAuxF4 + 3];
  const float3 v1 = make_float3(a1.x, a1.y, a1.z), v2 = make_float3(a2.x, a2.y, a2.z),
               nc = make_float3(a3.x, a3.y, a3.z);
  auto comb = [](float3 p, float a, float3 q, float b) {
    return make_float3(fmaf(p.x, a, q.x * b), fmaf(p.y, a, q.y * b), fmaf(p.z, a, q.z * b));
  };
  const float3 gmc = comb(v1, -g[0], v2, -g[1]);
  const float3 g_m = rotT(c.R, make_float3(fmaf(nc.x, g[2], gmc.x), fmaf(nc.y, g[2], gmc.y),
                                           fmaf(nc.z, g[2], gmc.z)));
  const float3 g_v1 = rotT(c.R, comb(v1, g[3], v2, g[4]));
  const float3 g_v2 = rotT(c.R, comb(v1, g[5], v2, g[6]));
  const float3 g_n = rotT(c.R, comb(v1, -g[7], v2, -g[8]));
  float q0 = quat[4 * i], q1 = quat[4 * i + 1], q2 = quat[4 * i + 2], q3 = quat[4 * i + 3];
  float qn = rsqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
  float w = q0 * qn, x = q1 * qn, y = q2 * qn, zq = q3 * qn;
  // dL/dR with R = [v1 v2 n] (row-major: G[row][col])
  float G[9] = {g_v1.x, g_v2.x, g_n.x, g_v1.y, g_v2.y, g_n.y, g_v1.z, g_v2.z, g_n.z};
  float gw = G[1] * (-2 * zq) + G[2] * (2 * y) + G[3] * (2 * zq) + G[5] * (-2 * x) +
             G[6] * (-2 * y) + G[7] * (2 * x);
  float gx = G[1] * (2 * y) + G[2] * (2 * zq) + G[3] * (2 * y) + G[4] * (-4 * x) +
             G[5] * (-2 * w) + G[6] * (2 * zq) + G[7] * (2 * w) + G[8] * (-4 * x);
  float gy = G[0] * (-4 * y) + G[1] * (2 * x) + G[2] * (2 * w) + G[3] * (2 * x) + G[5] * (2 * zq) +
             G[6] * (-2 * w) + G[7] * (2 * zq) + G[8] * (-4 * y);
  float gz = G[0] * (-4 * zq) + G[1] * (-2 * w) + G[2] * (2 * x) + G[3] * (2 * w) +
             G[4] * (-4 * zq) + G[5] * (2 * y) + G[6] * (2 * x) + G[7] * (2 * y);
  float dot = w * gw + x * gx + y * gy + zq * gz;
  float3 gm = g_m;
  if (sh_degree == 3) {
    // colour = 1/2 + sum_k Y_k(dir) c_k with dir = (mu - o) / |mu - o|:
    // dL/dc_k = Y_k dL/dcolour; dL/dmu through the direction
    const float vx = mu[3 * i] - c.o[0], vy = mu[3 * i + 1] - c.o[1], vz = mu[3 * i + 2] - c.o[2];
    const float inv = rsqrtf(fmaxf(vx * vx + vy * vy + vz * vz, 1e-30f));
    const float x = vx * inv, y = vy * inv, zd = vz * inv;
    const float* J = shj + 9 * (size_t)i;  // d colour_ch / d dir, from the forward
    const float3 q = make_float3(g[12] * J[0] + g[13] * J[3] + g[14] * J[6],
                                 g[12] * J[1] + g[13] * J[4] + g[14] * J[7],
                                 g[12] * J[2] + g[13] * J[5] + g[14] * J[8]);
    const float qd = q.x * x + q.y * y + q.z * zd;
    gm.x += (q.x - x * qd) * inv;
    gm.y += (q.y - y * qd) * inv;
    gm.z += (q.z - zd * qd) * inv;
    if (d_color) {
      const Sh3 Y = sh3_eval(x, y, zd);
      float dc[48];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        dc[3 * k] = Y.y[k] * g[12];
        dc[3 * k + 1] = Y.y[k] * g[13];
        dc[3 * k + 2] = Y.y[k] * g[14];
      }
      if (kAtomic) {
#pragma unroll
        for (int k = 0; k < 48; ++k) atomicAdd(d_color + 48 * (size_t)i + k, dc[k]);
      } else {
        // the surfel's 48 coefficients are 192 contiguous bytes: 16-byte
        // read-modify-writes
        float4* dst = reinterpret_cast<float4*>(d_color + 48 * (size_t)i);
#pragma unroll
        for (int q = 0; q < 12; ++q) {
          float4 v = dst[q];
          v.x += dc[4 * q]; v.y += dc[4 * q + 1]; v.z += dc[4 * q + 2]; v.w += dc[4 * q + 3];
          dst[q] = v;
        }
      }
    }
  }
  if (d_mu) {
    acc<kAtomic>(d_mu + 3 * i, gm.x);
    acc<kAtomic>(d_mu + 3 * i + 1, gm.y);
    acc<kAtomic>(d_mu + 3 * i + 2, gm.z);
  }
  if (d_quat) {
    acc<kAtomic>(d_quat + 4 * i, (gw - w * dot) * qn);
    acc<kAtomic>(d_quat + 4 * i + 1, (gx - x * dot) * qn);
    acc<kAtomic>(d_quat + 4 * i + 2, (gy - y * dot) * qn);
    acc<kAtomic>(d_quat + 4 * i + 3, (gz - zq * dot) * qn);
  }
  if (d_scale) {  // sigma1 = -sum(du / s1 . u s1) / s1, sigma2 likewise
    acc<kAtomic>(d_scale + 2 * i, -g[3] * a2.w);
    acc<kAtomic>(d_scale + 2 * i + 1, -g[6] * a3.w);
  }
  if (d_opac) acc<kAtomic>(d_opac + i, g[9]);
  if (d_gamma) {
    acc<kAtomic>(d_gamma + 2 * i, g[10]);
    acc<kAtomic>(d_gamma + 2 * i + 1, g[11]);
  }
  if (d_color && sh_degree != 3) {
    acc<kAtomic>(d_color + 3 * i, g[12]);
    acc<kAtomic>(d_color + 3 * i + 1, g[13]);
    acc<kAtomic>(d_color + 3 * i + 2, g[14]);
  }
}

cudaError_t launch_preprocess_bwd(const DevCam& c, const nexel_settings& s, int N, const float* mu,
                                  const float* quat, const float* scale, const float* opacity,
                                  const float* gamma, char* ws, const WsLayout& L, int accumulate,
                                  float* d_mu, float* d_quat, float* d_scale, float* d_opacity,
                                  float* d_gamma, float* d_color, bool atomic, cudaStream_t st) {
  (void)s;
  if (N <= 0) return cudaSuccess;
  if (!accumulate) {
    cudaError_t e = cudaSuccess;
    if (d_mu) e = cudaMemsetAsync(d_mu, 0, sizeof(float) * 3 * (size_t)N, st);
    if (e == cudaSuccess && d_quat) e = cudaMemsetAsync(d_quat, 0, sizeof(float) * 4 * (size_t)N, st);
    if (e == cudaSuccess && d_scale) e = cudaMemsetAsync(d_scale, 0, sizeof(float) * 2 * (size_t)N, st);
    if (e == cudaSuccess && d_opacity) e = cudaMemsetAsync(d_opacity, 0, sizeof(float) * (size_t)N, st);
    if (e == cudaSuccess && d_gamma) e = cudaMemsetAsync(d_gamma, 0, sizeof(float) * 2 * (size_t)N, st);
    if (e == cudaSuccess && d_color)
      e = cudaMemsetAsync(d_color, 0, sizeof(float) * (s.sh_degree == 3 ? 48 : 3) * (size_t)N, st);
    if (e != cudaSuccess) return e;
  }
  {
    NEXEL_PROF("preprocess_bwd", st);
    auto kern = atomic ? k_preprocess_bwd<true> : k_preprocess_bwd<false>;
    kern<<<(N + 255) / 256, 256, 0, st>>>(
        c, N, s.sh_degree, mu, (const float*)(ws + L.shj), quat, (uint32_t*)(ws + L.did1),
        (uint32_t*)(ws + L.dkey0),
        (float*)(ws + L.grad_sorted), (const float4*)(ws + L.aux_sorted), d_mu, d_quat, d_scale,
        d_opacity, d_gamma, d_color);
  }
  return cudaGetLastError();
}

}  // namespace nexel
