// FP64 CPU oracle for the Nexels image formation (forward and backward).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
// calls this file; only tests, the smoke check and the benchmark's CPU
// baseline leg do.  It shares no source with the CUDA path.
//
// It is the plain definition evaluated by brute force: for every requested
// pixel it walks ALL surfels in the global order of their centre depth
// (Sec. 3 "Preliminaries": surfels are sorted by the depth of their centres),
// intersects the pixel ray with each surfel plane, evaluates the generalised
// Gaussian kernel (Sec. 4.1, the alpha equation), composites front to back
// (Eq. 1, with the product over j < i of (1 - alpha_j)), keeps the K largest
// blending weights (Sec. 4.2, collection pass), forms the non-textured image
// (Eq. 5), queries the neural field at the K intersections (Eqs. 3-4:
// down-weighted hash-grid features through the MLP; supplementary Sec. 7.1
// for MapPositive and the trilinear interpolation) and composites the result
// (Eq. 6).  The backward is the analytic derivative of that result with the
// discrete choices (order, skips, early stop, top-K selection) held fixed.
//
// Readings where the paper is silent (shared as explicit parameters):
//   alpha_min / alpha_max / T_min, near plane, grazing threshold 1e-9 |d|,
//   unnormalised ray direction d = R^T ((x+.5-cx)/fx, (y+.5-cy)/fy, 1) so the
//   ray parameter equals view depth, focal length f = fx in Delta, the
//   Instant-NGP spatial hash (primes 1, 2654435761, 805459861, XOR, mod T),
//   MLP without bias, ReLU on hidden layers, linear output.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

extern "C" {

struct OCam {
  int W, H;
  double fx, fy, cx, cy;
  double Rt[12];  // row-major [R | t], x_cam = R x_world + t
  double near_;
};

struct OSet {
  int K;
  double alpha_min, alpha_max, T_min;
  double bg[3];
  double tie_tol;    // relative width used to flag threshold / top-K ties
  double order_tol;  // relative width used to flag centre-depth order ties
  double cell_tol;   // world-space distance to a hash-cell face flagged as a kink
  double relu_tol;   // relative width used to flag hidden pre-activations near 0
  double edge_tol;   // width of the band above the edge-on threshold flagged as a tie
};

struct OField {
  int L, T, F;
  const double* scale;    // [L]
  const double* table;    // [L][T][F]
  int n_layers;           // number of weight matrices
  const int* widths;      // [n_layers + 1]
  const double* weights;  // packed, layer l is [widths[l+1]][widths[l]]
};

}  // extern "C"

namespace {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- hash grid
// Supplementary Sec. 7.1: MapPositive(x) = 2x - 1 for x > 0, -2x otherwise.
inline uint64_t map_positive(int64_t k) {
  return k > 0 ? (uint64_t)(2 * k - 1) : (uint64_t)(-2 * k);
}

// Instant-NGP spatial hash on the MapPositive'd integer coordinates,
// computed modulo 2^32, then reduced modulo T.
inline uint32_t spatial_hash(int64_t kx, int64_t ky, int64_t kz, uint32_t T) {
  uint32_t mx = (uint32_t)map_positive(kx);
  uint32_t my = (uint32_t)map_positive(ky);
  uint32_t mz = (uint32_t)map_positive(kz);
  uint32_t h = (mx * 1u) ^ (my * 2654435761u) ^ (mz * 805459861u);
  return h % T;
}

// Eq. 3: Delta_l = 1 - exp(-(1/2pi) (f / (s_l t))^2).
inline double downweight(double f, double s, double t) {
  double r = f / (s * t);
  return 1.0 - std::exp(-(r * r) / (2.0 * kPi));
}
inline double downweight_dt(double f, double s, double t) {
  double r = f / (s * t);
  // d/dt [1 - exp(-r^2/2pi)] with dr/dt = -r/t
  return std::exp(-(r * r) / (2.0 * kPi)) * (-(2.0 * r / (2.0 * kPi)) * (r / t));
}

struct LevelEval {
  double acc[8];   // trilinear interpolation (before Delta), F <= 8
  double delta;    // Delta_l
  double frac[3];
  int64_t c0[3];
};

// Hash-grid features of one point, Sec. 3 (Instant-NGP) and Eq. 4:
// h = Delta_l * trilinear(H_l at s_l x), concatenated level-major.
void field_features(const OField& fd, double focal, const double x[3], double t,
                    double* feat, std::vector<LevelEval>* keep) {
  for (int l = 0; l < fd.L; ++l) {
    LevelEval e;
    double s = fd.scale[l];
    for (int a = 0; a < 3; ++a) {
      double g = s * x[a];
      double fl = std::floor(g);
      e.c0[a] = (int64_t)fl;
      e.frac[a] = g - fl;
    }
    for (int c = 0; c < fd.F; ++c) e.acc[c] = 0.0;
    for (int corner = 0; corner < 8; ++corner) {
      int dx = corner & 1, dy = (corner >> 1) & 1, dz = (corner >> 2) & 1;
      double w = (dx ? e.frac[0] : 1.0 - e.frac[0]) * (dy ? e.frac[1] : 1.0 - e.frac[1]) *
                 (dz ? e.frac[2] : 1.0 - e.frac[2]);
      uint32_t idx = spatial_hash(e.c0[0] + dx, e.c0[1] + dy, e.c0[2] + dz, (uint32_t)fd.T);
      const double* ent = fd.table + ((size_t)l * fd.T + idx) * fd.F;
      for (int c = 0; c < fd.F; ++c) e.acc[c] += w * ent[c];
    }
    e.delta = downweight(focal, s, t);
    for (int c = 0; c < fd.F; ++c) feat[l * fd.F + c] = e.delta * e.acc[c];
    if (keep) keep->push_back(e);
  }
}

// MLP G without bias: ReLU on hidden layers, linear output.  acts[l] holds
// the input of layer l (post-activation), acts[n_layers] the output.
void mlp_forward(const OField& fd, const double* in, std::vector<std::vector<double>>& acts) {
  acts.assign(fd.n_layers + 1, {});
  acts[0].assign(in, in + fd.widths[0]);
  const double* W = fd.weights;
  for (int l = 0; l < fd.n_layers; ++l) {
    int ni = fd.widths[l], no = fd.widths[l + 1];
    acts[l + 1].assign(no, 0.0);
    for (int o = 0; o < no; ++o) {
      double s = 0.0;
      for (int i = 0; i < ni; ++i) s += W[(size_t)o * ni + i] * acts[l][i];
      bool last = (l == fd.n_layers - 1);
      acts[l + 1][o] = last ? s : std::max(s, 0.0);
    }
    W += (size_t)no * ni;
  }
}

// Backward of the MLP: g_out -> g_in, accumulating weight gradients.  With
// `absolute` every product is replaced by the product of magnitudes (the
// ReLU masks kept): g_in and the weight gradients then hold the sums of the
// magnitudes of the terms along every path, the scale of the rounding error
// of an evaluation that rounds each layer's operands.
void mlp_backward(const OField& fd, const std::vector<std::vector<double>>& acts,
                  const double* g_out, double* g_in, double* d_weights, bool absolute = false) {
  std::vector<size_t> off(fd.n_layers + 1, 0);
  for (int l = 0; l < fd.n_layers; ++l)
    off[l + 1] = off[l] + (size_t)fd.widths[l] * fd.widths[l + 1];
  std::vector<double> g(g_out, g_out + fd.widths[fd.n_layers]);
  if (absolute)
    for (double& v : g) v = std::fabs(v);
  for (int l = fd.n_layers - 1; l >= 0; --l) {
    int ni = fd.widths[l], no = fd.widths[l + 1];
    bool last = (l == fd.n_layers - 1);
    if (!last)
      for (int o = 0; o < no; ++o)
        if (acts[l + 1][o] <= 0.0) g[o] = 0.0;  // ReLU derivative
    const double* W = fd.weights + off[l];
    std::vector<double> gi(ni, 0.0);
    for (int o = 0; o < no; ++o) {
      for (int i = 0; i < ni; ++i) {
        if (d_weights) {
          const double c = g[o] * acts[l][i];
          d_weights[off[l] + (size_t)o * ni + i] += absolute ? std::fabs(c) : c;
        }
        const double wv = W[(size_t)o * ni + i];
        gi[i] += (absolute ? std::fabs(wv) : wv) * g[o];
      }
    }
    g.swap(gi);
  }
  for (int i = 0; i < fd.widths[0]; ++i) g_in[i] = g[i];
}

// Real spherical harmonics of degree <= 3 at the unit direction (x, y, z):
// orthonormal on the sphere, ordered by degree l and m = -l .. l, with the
// Condon-Shortley phase.  An MLP with 48 outputs gives the texture as
// channel-wise SH coefficients o[3k + ch] (Sec. 3: "a set of spherical
// harmonics coefficients"; Sec. 5: degree 3), evaluated in the pixel's ray
// direction: T_ch = sum_k Y_k(d / |d|) o[3k + ch].
void sh3_basis(double x, double y, double z, double* Y) {
  const double sp = std::sqrt(3.14159265358979323846);
  const double k0 = 1.0 / (2.0 * sp), k1 = std::sqrt(3.0) / (2.0 * sp);
  const double k2a = std::sqrt(15.0) / (2.0 * sp), k2b = std::sqrt(5.0) / (4.0 * sp),
               k2c = std::sqrt(15.0) / (4.0 * sp);
  const double k3a = std::sqrt(17.5) / (4.0 * sp), k3b = std::sqrt(105.0) / (2.0 * sp),
               k3c = std::sqrt(10.5) / (4.0 * sp), k3d = std::sqrt(7.0) / (4.0 * sp),
               k3e = std::sqrt(105.0) / (4.0 * sp);
  const double xx = x * x, yy = y * y, zz = z * z;
  Y[0] = k0;
  Y[1] = -k1 * y; Y[2] = k1 * z; Y[3] = -k1 * x;
  Y[4] = k2a * x * y; Y[5] = -k2a * y * z; Y[6] = k2b * (2 * zz - xx - yy); Y[7] = -k2a * x * z;
  Y[8] = k2c * (xx - yy);
  Y[9] = -k3a * y * (3 * xx - yy); Y[10] = k3b * x * y * z; Y[11] = -k3c * y * (4 * zz - xx - yy);
  Y[12] = k3d * z * (2 * zz - 3 * xx - 3 * yy); Y[13] = -k3c * x * (4 * zz - xx - yy);
  Y[14] = k3e * z * (xx - yy); Y[15] = -k3a * x * (xx - 3 * yy);
}

// texture of one sample from the MLP output (3 outputs: RGB as is; 48: SH)
void texture_from_output(const OField& fd, const std::vector<double>& out, const double d[3],
                         double tex[3]) {
  const int no = fd.widths[fd.n_layers];
  if (no != 48) {
    for (int ch = 0; ch < 3; ++ch) tex[ch] = out[ch];
    return;
  }
  const double n = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double Y[16];
  sh3_basis(d[0] / n, d[1] / n, d[2] / n, Y);
  for (int ch = 0; ch < 3; ++ch) {
    tex[ch] = 0.0;
    for (int k = 0; k < 16; ++k) tex[ch] += Y[k] * out[3 * k + ch];
  }
}

// gradient with respect to the MLP output from the texture gradient gT
std::vector<double> output_grad(const OField& fd, const double gT[3], const double d[3]) {
  const int no = fd.widths[fd.n_layers];
  std::vector<double> g(no, 0.0);
  if (no != 48) {
    for (int ch = 0; ch < 3; ++ch) g[ch] = gT[ch];
    return g;
  }
  const double n = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double Y[16];
  sh3_basis(d[0] / n, d[1] / n, d[2] / n, Y);
  for (int k = 0; k < 16; ++k)
    for (int ch = 0; ch < 3; ++ch) g[3 * k + ch] = Y[k] * gT[ch];
  return g;
}

// ------------------------------------------------------------- geometry
void quat_to_rot(const double q[4], double R[9]) {
  double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

// dL/dq from dL/dR (R built from q / |q|).
void rot_backward(const double q[4], const double G[9], double dq[4]) {
  double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
  const double dRw[9] = {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0};
  const double dRx[9] = {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
  const double dRy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y};
  const double dRz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0};
  double gh[4] = {0, 0, 0, 0};
  for (int k = 0; k < 9; ++k) {
    gh[0] += G[k] * dRw[k]; gh[1] += G[k] * dRx[k];
    gh[2] += G[k] * dRy[k]; gh[3] += G[k] * dRz[k];
  }
  double qh[4] = {w, x, y, z};
  double dot = qh[0] * gh[0] + qh[1] * gh[1] + qh[2] * gh[2] + qh[3] * gh[3];
  for (int k = 0; k < 4; ++k) dq[k] = (gh[k] - qh[k] * dot) / n;
}

inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// |a|^(2g) with |0|^(2g) = 0
inline double powabs(double a, double g) { return a == 0.0 ? 0.0 : std::pow(std::fabs(a), 2.0 * g); }

// A surfel whose plane contains (to within kEdgeOn) its own centre ray is
// seen edge-on: its footprint on screen degenerates to a line through the
// projected centre.  The paper is silent on this case; the reading culls it.
// The test is |d_mu . n_c| < kEdgeOn with d_mu = mu_c / z_mu the centre ray
// scaled to unit depth and n_c the camera-space normal.
constexpr double kEdgeOn = 1e-7;
enum { EDGE_NONE = 0, EDGE_BAND = 1, EDGE_CULLED = 2 };

struct Scene {
  int N;
  const double *mu, *quat, *scale, *opac, *gamma, *color;
  std::vector<std::array<double, 9>> R;  // per-surfel rotation
  std::vector<int> order;                // sorted by centre depth, culled removed
  std::vector<double> zc;                // centre view depth
  std::vector<unsigned char> edge;       // EDGE_* bits of the edge-on reading
};

void ray_of(const OCam& c, int px, int py, double o[3], double d[3]) {
  const double* M = c.Rt;
  double dc[3] = {(px + 0.5 - c.cx) / c.fx, (py + 0.5 - c.cy) / c.fy, 1.0};
  for (int a = 0; a < 3; ++a) {
    o[a] = -(M[0 * 4 + a] * M[3] + M[1 * 4 + a] * M[7] + M[2 * 4 + a] * M[11]);
    d[a] = M[0 * 4 + a] * dc[0] + M[1 * 4 + a] * dc[1] + M[2 * 4 + a] * dc[2];
  }
}

void prepare_scene(const OCam& c, const OSet* st, Scene& s) {
  s.R.resize(s.N);
  s.zc.resize(s.N);
  s.edge.assign(s.N, EDGE_NONE);
  const double band = st ? st->edge_tol : 0.0;
  for (int i = 0; i < s.N; ++i) {
    quat_to_rot(s.quat + 4 * i, s.R[i].data());
    const double* m = s.mu + 3 * i;
    double mc[3];
    for (int a = 0; a < 3; ++a)
      mc[a] = c.Rt[4 * a] * m[0] + c.Rt[4 * a + 1] * m[1] + c.Rt[4 * a + 2] * m[2] + c.Rt[4 * a + 3];
    s.zc[i] = mc[2];
    if (mc[2] > c.near_) {
      // edge-on test: camera-space normal n_c = R_cam n against mu_c / z_mu
      const double* R = s.R[i].data();
      double nc[3];
      for (int a = 0; a < 3; ++a)
        nc[a] = c.Rt[4 * a] * R[2] + c.Rt[4 * a + 1] * R[5] + c.Rt[4 * a + 2] * R[8];
      const double dn0 = (mc[0] * nc[0] + mc[1] * nc[1] + mc[2] * nc[2]) / mc[2];
      if (std::fabs(dn0) < kEdgeOn) s.edge[i] |= EDGE_CULLED;
      if (std::fabs(std::fabs(dn0) - kEdgeOn) <= band) s.edge[i] |= EDGE_BAND;
    }
  }
  s.order.clear();
  for (int i = 0; i < s.N; ++i)
    if (s.zc[i] > c.near_) s.order.push_back(i);
  std::stable_sort(s.order.begin(), s.order.end(),
                   [&](int a, int b) { return s.zc[a] < s.zc[b]; });
}

struct Contrib {
  int id, pos;
  double alpha, alpha_raw, T, w, t, u, v;
  bool clamped;
  double x[3];
};

struct PixelResult {
  double o[3], d[3];
  std::vector<Contrib> list;
  std::vector<int> sel;  // indices into list, slot order
  double T_final;
  int tie;
  int slot_tie[8];  // kink bits (TIE_CELL, TIE_RELU) of each slot's sample
  double notex[3], image[3];
  double tex[8][3];
  std::vector<std::vector<std::vector<double>>> acts;  // per slot MLP activations
  std::vector<std::vector<LevelEval>> lev;             // per slot level evals
};

enum {
  TIE_TOPK = 1, TIE_ALPHA = 2, TIE_TMIN = 4, TIE_NEAR = 8, TIE_ORDER = 16, TIE_CELL = 32,
  TIE_RELU = 64, TIE_EDGE = 128
};

inline bool near_rel(double a, double b, double tol) {
  return std::fabs(a - b) <= tol * std::max(std::fabs(a), std::fabs(b));
}

void render_pixel(const OCam& c, const OSet& st, const OField* fd, const Scene& s, int pix,
                  bool keep, PixelResult& r) {
  int px = pix % c.W, py = pix / c.W;
  ray_of(c, px, py, r.o, r.d);
  const double* o = r.o;
  const double* d = r.d;
  double dn = std::sqrt(dot3(d, d));
  double T = 1.0;
  r.list.clear();
  r.tie = 0;
  double tol = st.tie_tol;
  for (size_t pos = 0; pos < s.order.size(); ++pos) {
    int i = s.order[pos];
    const double* R = s.R[i].data();
    double v1[3] = {R[0], R[3], R[6]}, v2[3] = {R[1], R[4], R[7]}, n[3] = {R[2], R[5], R[8]};
    const double* mu = s.mu + 3 * i;
    double den = dot3(d, n);
    if (std::fabs(den) < 1e-9 * dn) continue;  // grazing
    double mo[3] = {mu[0] - o[0], mu[1] - o[1], mu[2] - o[2]};
    double t = dot3(mo, n) / den;
    if (t <= c.near_) {
      if (near_rel(t, c.near_, tol)) r.tie |= TIE_NEAR;
      continue;
    }
    double x[3] = {o[0] + t * d[0], o[1] + t * d[1], o[2] + t * d[2]};
    double rr[3] = {x[0] - mu[0], x[1] - mu[1], x[2] - mu[2]};
    double u = dot3(rr, v1) / s.scale[2 * i];
    double v = dot3(rr, v2) / s.scale[2 * i + 1];
    double a = s.opac[i] * std::exp(-0.5 * powabs(u, s.gamma[2 * i])) *
               std::exp(-0.5 * powabs(v, s.gamma[2 * i + 1]));
    if (near_rel(t, c.near_, tol)) r.tie |= TIE_NEAR;
    if (near_rel(a, st.alpha_min, tol)) r.tie |= TIE_ALPHA;
    if (a < st.alpha_min || a == 0.0) continue;
    // a surfel near the edge-on threshold would be composited here: a
    // lower-precision test of the threshold may keep or cull it
    if (s.edge[i] & EDGE_BAND) r.tie |= TIE_EDGE;
    if (s.edge[i] & EDGE_CULLED) continue;
    if (near_rel(a, st.alpha_max, tol)) r.tie |= TIE_ALPHA;
    double ac = std::min(a, st.alpha_max);
    double test = T * (1.0 - ac);
    if (near_rel(test, st.T_min, tol)) r.tie |= TIE_TMIN;
    if (test < st.T_min) break;  // stop before this surfel
    Contrib e;
    e.id = i; e.pos = (int)pos; e.alpha = ac; e.alpha_raw = a; e.clamped = a > st.alpha_max;
    e.T = T; e.w = ac * T; e.t = t; e.u = u; e.v = v;
    for (int k = 0; k < 3; ++k) e.x[k] = x[k];
    // equal depths are ordered by index on every side; only nearly equal,
    // unequal ones can be ordered differently by a lower-precision key
    if (!r.list.empty() && s.zc[r.list.back().id] != s.zc[i] &&
        near_rel(s.zc[r.list.back().id], s.zc[i], st.order_tol))
      r.tie |= TIE_ORDER;
    r.list.push_back(e);
    T = test;
  }
  r.T_final = T;
  // Top-K by weight (Sec. 4.2): the K largest positive weights, equal weights
  // resolved in favour of the front-most; slots in descending weight order.
  std::vector<int> idx(r.list.size());
  for (size_t k = 0; k < idx.size(); ++k) idx[k] = (int)k;
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int a, int b) { return r.list[a].w > r.list[b].w; });
  r.sel.clear();
  for (size_t k = 0; k < idx.size() && (int)k < st.K; ++k)
    if (r.list[idx[k]].w > 0.0) r.sel.push_back(idx[k]);
  size_t chk = std::min(idx.size(), (size_t)st.K + 1);
  for (size_t k = 0; k + 1 < chk; ++k)
    if (near_rel(r.list[idx[k]].w, r.list[idx[k + 1]].w, tol)) r.tie |= TIE_TOPK;
  // Eq. 5: non-textured render excludes the selected primitives.
  std::vector<char> is_sel(r.list.size(), 0);
  for (int k : r.sel) is_sel[k] = 1;
  for (int ch = 0; ch < 3; ++ch) r.notex[ch] = 0.0;
  for (size_t k = 0; k < r.list.size(); ++k) {
    if (is_sel[k]) continue;
    const double* col = s.color + 3 * r.list[k].id;
    for (int ch = 0; ch < 3; ++ch) r.notex[ch] += r.list[k].w * col[ch];
  }
  // Texturing pass: x = o + D d, Eq. 4, then Eq. 6.
  for (int ch = 0; ch < 3; ++ch) r.image[ch] = r.notex[ch] + r.T_final * st.bg[ch];
  r.acts.assign(r.sel.size(), {});
  r.lev.assign(r.sel.size(), {});
  for (int j = 0; j < 8; ++j) r.slot_tie[j] = 0;
  for (size_t j = 0; j < r.sel.size(); ++j) {
    const Contrib& e = r.list[r.sel[j]];
    for (int ch = 0; ch < 3; ++ch) r.tex[j][ch] = 0.0;
    if (!fd) continue;
    double x[3] = {o[0] + e.t * d[0], o[1] + e.t * d[1], o[2] + e.t * d[2]};
    // the integer cell of each level is decided by floor(s_l x): a point
    // within cell_tol (world units) of a cell face is a kink of the
    // trilinear interpolation, where a lower-precision x may fall on the
    // other side
    if (st.cell_tol > 0.0)
      for (int l = 0; l < fd->L; ++l)
        for (int a = 0; a < 3; ++a) {
          double g = fd->scale[l] * x[a];
          if (std::fabs(g - std::nearbyint(g)) < st.cell_tol * fd->scale[l]) r.slot_tie[j] |= TIE_CELL;
        }
    std::vector<double> feat(fd->L * fd->F);
    field_features(*fd, c.fx, x, e.t, feat.data(), keep ? &r.lev[j] : nullptr);
    std::vector<std::vector<double>> acts;
    mlp_forward(*fd, feat.data(), acts);
    texture_from_output(*fd, acts[fd->n_layers], d, r.tex[j]);
    for (int ch = 0; ch < 3; ++ch) r.image[ch] += e.w * r.tex[j][ch];
    // a hidden pre-activation within relu_tol of zero (relative to the sum
    // of the magnitudes of its terms) is a ReLU decision that a
    // lower-precision evaluation may take the other way
    if (st.relu_tol > 0.0) {
      const double* W = fd->weights;
      for (int l = 0; l + 1 < fd->n_layers; ++l) {
        int ni = fd->widths[l], no = fd->widths[l + 1];
        for (int o2 = 0; o2 < no; ++o2) {
          double a = 0.0, mag = 0.0;
          for (int i = 0; i < ni; ++i) {
            double term = W[(size_t)o2 * ni + i] * acts[l][i];
            a += term;
            mag += std::fabs(term);
          }
          if (std::fabs(a) <= st.relu_tol * mag && mag > 0.0) r.slot_tie[j] |= TIE_RELU;
        }
        W += (size_t)no * ni;
      }
    }
    r.tie |= r.slot_tie[j];
    if (keep) r.acts[j] = std::move(acts);
  }
}

Scene make_scene(const OCam& c, const OSet* st, int N, const double* mu, const double* quat,
                 const double* scale, const double* opac, const double* gamma,
                 const double* color) {
  Scene s;
  s.N = N; s.mu = mu; s.quat = quat; s.scale = scale; s.opac = opac; s.gamma = gamma; s.color = color;
  prepare_scene(c, st, s);
  return s;
}

constexpr int kSG = 15;  // per-surfel grad record: mu3 q4 sigma2 o1 gamma2 color3

struct PixGrad {
  std::vector<std::pair<int, std::array<double, kSG>>> surf;
  std::vector<std::pair<size_t, double>> tab;
};

}  // namespace

extern "C" {

uint64_t oracle_map_positive(int64_t k) { return map_positive(k); }

uint32_t oracle_hash(int64_t kx, int64_t ky, int64_t kz, uint32_t T) {
  return spatial_hash(kx, ky, kz, T);
}

// Down-weighted hash-grid features for n points; feat is [n][L*F].
void oracle_field_features(const OField* fd, double focal, int n, const double* x,
                           const double* t, double* feat) {
  for (int k = 0; k < n; ++k) field_features(*fd, focal, x + 3 * k, t[k], feat + (size_t)k * fd->L * fd->F, nullptr);
}

// MLP G on n input vectors; out is [n][widths[n_layers]].
void oracle_mlp(const OField* fd, int n, const double* in, double* out) {
  int no = fd->widths[fd->n_layers];
  for (int k = 0; k < n; ++k) {
    std::vector<std::vector<double>> acts;
    mlp_forward(*fd, in + (size_t)k * fd->widths[0], acts);
    for (int c = 0; c < no; ++c) out[(size_t)k * no + c] = acts[fd->n_layers][c];
  }
}

// Texture radiance of Eq. 4 at points x with depths t.
void oracle_texture(const OField* fd, double focal, int n, const double* x, const double* t,
                    double* out) {
  int no = fd->widths[fd->n_layers];
  for (int k = 0; k < n; ++k) {
    std::vector<double> feat(fd->L * fd->F);
    field_features(*fd, focal, x + 3 * k, t[k], feat.data(), nullptr);
    std::vector<std::vector<double>> acts;
    mlp_forward(*fd, feat.data(), acts);
    for (int c = 0; c < no; ++c) out[(size_t)k * no + c] = acts[fd->n_layers][c];
  }
}

// Centre-depth order (ascending, index ties ascending), culled surfels left out.
int oracle_depth_order(const OCam* c, int N, const double* mu, int* order) {
  Scene s;
  s.N = N; s.mu = mu;
  s.zc.resize(N);
  for (int i = 0; i < N; ++i) {
    const double* m = mu + 3 * i;
    s.zc[i] = c->Rt[8] * m[0] + c->Rt[9] * m[1] + c->Rt[10] * m[2] + c->Rt[11];
  }
  int n = 0;
  for (int i = 0; i < N; ++i)
    if (s.zc[i] > c->near_) order[n++] = i;
  std::stable_sort(order, order + n, [&](int a, int b) { return s.zc[a] < s.zc[b]; });
  return n;
}

// Forward render of the listed pixels (flat index y*W + x).  Any output
// pointer may be null.  field may be null (textures then zero).
int oracle_render(const OCam* c, const OSet* st, const OField* fd, int N, const double* mu,
                  const double* quat, const double* scale, const double* opac,
                  const double* gamma, const double* color, int n_pix, const int* pix,
                  double* image, double* notex, double* weights, int* ids, double* depths,
                  double* textures, double* T_final, int* n_contrib, int* tie, int* slot_tie) {
  if (st->K < 0 || st->K > 8) return -1;
  Scene s = make_scene(*c, st, N, mu, quat, scale, opac, gamma, color);
  int K = st->K;
#pragma omp parallel for schedule(dynamic, 16)
  for (int p = 0; p < n_pix; ++p) {
    PixelResult r;
    render_pixel(*c, *st, fd, s, pix[p], false, r);
    for (int ch = 0; ch < 3; ++ch) {
      if (image) image[3 * p + ch] = r.image[ch];
      if (notex) notex[3 * p + ch] = r.notex[ch];
    }
    for (int j = 0; j < K; ++j) {
      bool has = j < (int)r.sel.size();
      const Contrib* e = has ? &r.list[r.sel[j]] : nullptr;
      if (weights) weights[(size_t)p * K + j] = has ? e->w : 0.0;
      if (ids) ids[(size_t)p * K + j] = has ? e->id : -1;
      if (depths) depths[(size_t)p * K + j] = has ? e->t : 0.0;
      if (slot_tie) slot_tie[(size_t)p * K + j] = has ? r.slot_tie[j] : 0;
      for (int ch = 0; ch < 3; ++ch)
        if (textures) textures[((size_t)p * K + j) * 3 + ch] = has ? r.tex[j][ch] : 0.0;
    }
    if (T_final) T_final[p] = r.T_final;
    if (n_contrib) n_contrib[p] = (int)r.list.size();
    if (tie) tie[p] = r.tie;
  }
  return 0;
}

// Reference images for the learned-part test: the same compositing (Eq. 1)
// over all intersected surfels, but every surfel shows a known procedural
// world-space texture tau(x*) at its intersection instead of a colour:
//   tau_c(x) = 0.5 + 0.4 sin(f x_0 + 2c) sin(f x_1 + c) + 0.1 sin(f x_2 - c).
// image is [n_pix][3].
int oracle_render_procedural(const OCam* c, const OSet* st, int N, const double* mu,
                             const double* quat, const double* scale, const double* opac,
                             const double* gamma, double freq, int n_pix, const int* pix,
                             double* image) {
  std::vector<double> dummy(3 * (size_t)std::max(N, 1), 0.0);
  Scene s = make_scene(*c, st, N, mu, quat, scale, opac, gamma, dummy.data());
  OSet st0 = *st;
  st0.K = 0;
#pragma omp parallel for schedule(dynamic, 16)
  for (int p = 0; p < n_pix; ++p) {
    PixelResult r;
    render_pixel(*c, st0, nullptr, s, pix[p], false, r);
    for (int ch = 0; ch < 3; ++ch) {
      double v = r.T_final * st->bg[ch];
      for (const Contrib& e : r.list) {
        double tau = 0.5 + 0.4 * std::sin(freq * e.x[0] + 2.0 * ch) * std::sin(freq * e.x[1] + ch) +
                     0.1 * std::sin(freq * e.x[2] - ch);
        v += e.w * tau;
      }
      image[3 * p + ch] = v;
    }
  }
  return 0;
}

// Blended L1 error of every surfel (supp. Sec. 7.2, "Densification": the
// per-primitive error of Rota Bulo et al.): err[i] += sum over the listed
// pixels of w_ip e_p, with w_ip = alpha T the compositing weight of surfel i
// at pixel p (every composited surfel, textured or not) and e_p the pixel's
// error, given.
int oracle_blend_error(const OCam* c, const OSet* st, int N, const double* mu, const double* quat,
                       const double* scale, const double* opac, const double* gamma,
                       const double* color, int n_pix, const int* pix, const double* e_pix,
                       double* err) {
  Scene s = make_scene(*c, st, N, mu, quat, scale, opac, gamma, color);
  std::vector<std::vector<std::pair<int, double>>> acc(n_pix);
#pragma omp parallel for schedule(dynamic, 16)
  for (int p = 0; p < n_pix; ++p) {
    PixelResult r;
    render_pixel(*c, *st, nullptr, s, pix[p], false, r);
    for (const Contrib& e : r.list) acc[p].push_back({e.id, e.w * e_pix[p]});
  }
  for (int p = 0; p < n_pix; ++p)
    for (auto& q : acc[p]) err[q.first] += q.second;
  return 0;
}

// Backward of the listed pixels' outputs.  Upstream gradients:
//   d_image [n_pix][3] (required), d_weights [n_pix][K] and
//   d_textures [n_pix][K][3] (each may be null).
// Gradient outputs are OVERWRITTEN (zeroed first); any may be null.
// d_table is [L][T][F], d_mlp is packed like the weights.  With absolute
// != 0 the texture path is evaluated on magnitudes -- every product through
// the MLP backward, the trilinear weights and the positional gradient taken
// as the product of magnitudes, every sum as a sum of magnitudes -- and every
// contribution is added as its magnitude: each table and MLP entry then
// holds the sum of the magnitudes of all the terms that reach it (and each
// surfel entry the sum over pixels of |its per-pixel contribution|), the
// scale against which the rounding error of an evaluation that rounds the
// MLP's operands is bounded.
int oracle_render_bwd(const OCam* c, const OSet* st, const OField* fd, int N, const double* mu,
                      const double* quat, const double* scale, const double* opac,
                      const double* gamma, const double* color, int n_pix, const int* pix,
                      const double* d_image, const double* d_weights, const double* d_textures,
                      double* d_mu, double* d_quat, double* d_scale, double* d_opac,
                      double* d_gamma, double* d_color, double* d_table, double* d_mlp,
                      int absolute) {
  if (st->K < 0 || st->K > 8) return -1;
  const bool ab = absolute != 0;
  auto acc = [ab](double v) { return ab ? std::fabs(v) : v; };
  Scene s = make_scene(*c, st, N, mu, quat, scale, opac, gamma, color);
  int K = st->K;
  size_t n_mlp = 0;
  if (fd)
    for (int l = 0; l < fd->n_layers; ++l) n_mlp += (size_t)fd->widths[l] * fd->widths[l + 1];
  std::vector<PixGrad> pg(n_pix);
  int n_threads = 1;
#ifdef _OPENMP
  n_threads = omp_get_max_threads();
#endif
  std::vector<std::vector<double>> mlp_acc(n_threads, std::vector<double>(n_mlp, 0.0));
  // Gradient of the down-weighted trilinear features w.r.t. the point x and
  // depth t is taken through Delta (Eq. 3) and the interpolation weights
  // (supplementary Sec. 7.1, "positional gradient").
#pragma omp parallel for schedule(dynamic, 16)
  for (int p = 0; p < n_pix; ++p) {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    PixelResult r;
    render_pixel(*c, *st, fd, s, pix[p], true, r);
    const double* dC = d_image + 3 * p;
    size_t M = r.list.size();
    std::vector<double> e(M, 0.0), dt(M, 0.0), dt_mag(M, 0.0);
    std::vector<int> slot(M, -1);
    for (size_t j = 0; j < r.sel.size(); ++j) slot[r.sel[j]] = (int)j;
    PixGrad& G = pg[p];
    // texture slots: upstream to the texture, then through the field
    for (size_t j = 0; j < r.sel.size(); ++j) {
      int k = r.sel[j];
      const Contrib& ce = r.list[k];
      double gT[3];
      for (int ch = 0; ch < 3; ++ch) {
        gT[ch] = ce.w * dC[ch];
        if (d_textures) gT[ch] += d_textures[((size_t)p * K + j) * 3 + ch];
      }
      e[k] = dot3(r.tex[j], dC) + (d_weights ? d_weights[(size_t)p * K + j] : 0.0);
      if (!fd) continue;
      // the field's backward for this sample: MLP (weight gradients),
      // table scatter and the positional gradient dt; evaluated signed, and
      // in absolute mode once more on magnitudes for the table, the MLP and
      // the scale of dt's rounding error
      auto chain = [&](bool mag, double* dt_out) {
        auto am = [mag](double v) { return mag ? std::fabs(v) : v; };
        std::vector<double> gfeat(fd->widths[0]);
        const std::vector<double> gout = output_grad(*fd, gT, r.d);
        mlp_backward(*fd, r.acts[j], gout.data(), gfeat.data(),
                     (n_mlp && mag == ab) ? mlp_acc[tid].data() : nullptr, mag);
        double gx[3] = {0, 0, 0};
        double gt = 0.0;
        for (int l = 0; l < fd->L; ++l) {
          const LevelEval& le = r.lev[j][l];
          double sl = fd->scale[l];
          // d feature / d Delta
          double gd = 0.0;
          for (int f = 0; f < fd->F; ++f) gd += am(gfeat[l * fd->F + f] * le.acc[f]);
          gt += am(gd * downweight_dt(c->fx, sl, ce.t));
          for (int corner = 0; corner < 8; ++corner) {
            int dx = corner & 1, dy = (corner >> 1) & 1, dz = (corner >> 2) & 1;
            int dl[3] = {dx, dy, dz};
            double wa[3], dwa[3];
            for (int a = 0; a < 3; ++a) {
              wa[a] = dl[a] ? le.frac[a] : 1.0 - le.frac[a];
              dwa[a] = dl[a] ? 1.0 : -1.0;
            }
            double w = wa[0] * wa[1] * wa[2];
            uint32_t idx = spatial_hash(le.c0[0] + dx, le.c0[1] + dy, le.c0[2] + dz, (uint32_t)fd->T);
            const double* ent = fd->table + ((size_t)l * fd->T + idx) * fd->F;
            double ge = 0.0;
            for (int f = 0; f < fd->F; ++f) {
              double g = gfeat[l * fd->F + f];
              if (d_table && mag == ab)
                G.tab.push_back({((size_t)l * fd->T + idx) * fd->F + f, am(le.delta * w * g)});
              ge += am(g * ent[f]);
            }
            // d/dx_a of w = dwa[a] * prod_{b != a} wa[b] * s_l
            gx[0] += am(le.delta * ge * dwa[0] * wa[1] * wa[2] * sl);
            gx[1] += am(le.delta * ge * wa[0] * dwa[1] * wa[2] * sl);
            gx[2] += am(le.delta * ge * wa[0] * wa[1] * dwa[2] * sl);
          }
        }
        // x = o + t d
        for (int a = 0; a < 3; ++a) gt += am(gx[a] * r.d[a]);
        *dt_out += gt;
      };
      chain(false, &dt[k]);
      if (ab) chain(true, &dt_mag[k]);
    }
    for (size_t k = 0; k < M; ++k)
      if (slot[k] < 0) e[k] = dot3(s.color + 3 * r.list[k].id, dC);
    // Eq. 1 backward without division: with R_i the weighted sum of what lies
    // behind surfel i as seen from just behind it, dC/dalpha_i = T_i (e_i - R_i).
    // The background acts as a last layer of opacity 1.
    double Rb = dot3(st->bg, dC);
    std::vector<double> Rv(M, 0.0);
    for (size_t kk = M; kk-- > 0;) {
      Rv[kk] = Rb;
      Rb = r.list[kk].alpha * e[kk] + (1.0 - r.list[kk].alpha) * Rb;
    }
    for (size_t k = 0; k < M; ++k) {
      const Contrib& ce = r.list[k];
      int i = ce.id;
      std::array<double, kSG> g{};
      double da = ce.T * (e[k] - Rv[k]);
      if (slot[k] < 0)
        for (int ch = 0; ch < 3; ++ch) g[12 + ch] = ce.w * dC[ch];
      double du = 0.0, dv = 0.0;
      if (!ce.clamped) {
        double a = ce.alpha;
        double g1 = s.gamma[2 * i], g2 = s.gamma[2 * i + 1];
        g[9] = da * a / s.opac[i];
        double au = std::fabs(ce.u), av = std::fabs(ce.v);
        if (au > 0) {
          du = da * (-a * g1 * std::pow(au, 2 * g1 - 2) * ce.u);
          g[10] = da * (-a * std::pow(au, 2 * g1) * std::log(au));
        }
        if (av > 0) {
          dv = da * (-a * g2 * std::pow(av, 2 * g2 - 2) * ce.v);
          g[11] = da * (-a * std::pow(av, 2 * g2) * std::log(av));
        }
      }
      const double* R = s.R[i].data();
      double v1[3] = {R[0], R[3], R[6]}, v2[3] = {R[1], R[4], R[7]}, n[3] = {R[2], R[5], R[8]};
      const double* m = s.mu + 3 * i;
      double s1 = s.scale[2 * i], s2 = s.scale[2 * i + 1];
      double rr[3] = {ce.x[0] - m[0], ce.x[1] - m[1], ce.x[2] - m[2]};
      double gv1[3], gv2[3], gn[3], gmu[3];
      for (int a = 0; a < 3; ++a) {
        gv1[a] = du * rr[a] / s1;
        gv2[a] = dv * rr[a] / s2;
      }
      g[7] = -du * ce.u / s1;
      g[8] = -dv * ce.v / s2;
      double gr[3];
      for (int a = 0; a < 3; ++a) gr[a] = du * v1[a] / s1 + dv * v2[a] / s2;
      double gtt = dt[k] + dot3(gr, r.d);
      double den = dot3(r.d, n);
      for (int a = 0; a < 3; ++a) {
        gmu[a] = -gr[a] + gtt * n[a] / den;
        gn[a] = gtt * (m[a] - ce.x[a]) / den;
      }
      double GR[9] = {gv1[0], gv2[0], gn[0], gv1[1], gv2[1], gn[1], gv1[2], gv2[2], gn[2]};
      double dq[4];
      rot_backward(s.quat + 4 * i, GR, dq);
      for (int a = 0; a < 3; ++a) g[a] = gmu[a];
      for (int a = 0; a < 4; ++a) g[3 + a] = dq[a];
      if (ab && dt_mag[k] != 0.0) {
        // the record is linear in dt: add the magnitude of what the texture
        // path's dt (taken on magnitudes) moves mu and q by
        double gnx[3];
        for (int a = 0; a < 3; ++a) {
          g[a] = std::fabs(g[a]) + std::fabs(dt_mag[k] * n[a] / den);
          gnx[a] = dt_mag[k] * (m[a] - ce.x[a]) / den;
        }
        double GX[9] = {0, 0, gnx[0], 0, 0, gnx[1], 0, 0, gnx[2]};
        double dqx[4];
        rot_backward(s.quat + 4 * i, GX, dqx);
        for (int a = 0; a < 4; ++a) g[3 + a] = std::fabs(g[3 + a]) + std::fabs(dqx[a]);
      }
      G.surf.push_back({i, g});
    }
  }
  auto zero = [](double* p, size_t n) { if (p) std::memset(p, 0, n * sizeof(double)); };
  zero(d_mu, 3 * (size_t)N); zero(d_quat, 4 * (size_t)N); zero(d_scale, 2 * (size_t)N);
  zero(d_opac, N); zero(d_gamma, 2 * (size_t)N); zero(d_color, 3 * (size_t)N);
  if (fd) { zero(d_table, (size_t)fd->L * fd->T * fd->F); zero(d_mlp, n_mlp); }
  for (int p = 0; p < n_pix; ++p) {
    for (auto& sg : pg[p].surf) {
      int i = sg.first;
      const auto& g = sg.second;
      if (d_mu) for (int a = 0; a < 3; ++a) d_mu[3 * i + a] += acc(g[a]);
      if (d_quat) for (int a = 0; a < 4; ++a) d_quat[4 * i + a] += acc(g[3 + a]);
      if (d_scale) for (int a = 0; a < 2; ++a) d_scale[2 * i + a] += acc(g[7 + a]);
      if (d_opac) d_opac[i] += acc(g[9]);
      if (d_gamma) for (int a = 0; a < 2; ++a) d_gamma[2 * i + a] += acc(g[10 + a]);
      if (d_color) for (int a = 0; a < 3; ++a) d_color[3 * i + a] += acc(g[12 + a]);
    }
    if (d_table)
      for (auto& tg : pg[p].tab) d_table[tg.first] += acc(tg.second);
  }
  if (d_mlp)
    for (int t = 0; t < n_threads; ++t)
      for (size_t k = 0; k < n_mlp; ++k) d_mlp[k] += mlp_acc[t][k];
  return 0;
}

}  // extern "C"
