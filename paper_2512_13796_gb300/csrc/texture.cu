// Dispatch of the texturing pass over the supported MLP shapes and storage
// types.  The FP32 kernels are in texture_f32.cuh, the BF16 / FP16
// tensor-core (tcgen05) ones in texture_tc.cu.
#include "texture_f32.cuh"

namespace nexel {

// FP32 instantiations (input, hidden 1, hidden 2, outputs): 3 outputs are
// RGB, 48 the degree-3 SH coefficients of the texture (the chunked kernels;
// the tensor-core forms take 48 outputs too, in texture_tc.cu)
#define NEXEL_ARCH_LIST(X) \
  X(8, 16, 0, 3)           \
  X(16, 64, 0, 3)          \
  X(32, 64, 64, 3)         \
  X(16, 64, 0, 48)         \
  X(32, 64, 64, 48)

// Explicit instantiations live in one translation unit per architecture
// (texture_f32_<in>_<h1>_<h2>.cu) so that they compile in parallel.
#define X(a, b, cc, o)                                                                           \
  extern template cudaError_t tex_fwd_f32<a, b, cc, float, o>(                                   \
      const DevCam&, const nexel_settings&, const FieldDev&, const float*, const float*,         \
      const int*, const float*, const float*, float*, float*, cudaStream_t);                     \
  extern template cudaError_t tex_bwd_f32<a, b, cc, float, o>(                                   \
      const DevCam&, const nexel_settings&, const FieldDev&, char*, const BwdLayout&,            \
      const float*, const int*, const float*, const float*, const float*, const float*, float*,  \
      float*, cudaStream_t);                                                                     \

NEXEL_ARCH_LIST(X)
#undef X

static bool arch_match(const nexel_field& f, int in, int h1, int h2, int out) {
  if (h2 == 0)
    return f.n_layers == 2 && f.widths[0] == in && f.widths[1] == h1 && f.widths[2] == out;
  return f.n_layers == 3 && f.widths[0] == in && f.widths[1] == h1 && f.widths[2] == h2 &&
         f.widths[3] == out;
}

bool texture_arch_supported(const nexel_settings& s, const nexel_field& f) {
  if (f.F != 2 || f.L * f.F != f.widths[0]) return false;
  if (s.mlp_dtype == NEXEL_BF16 || s.mlp_dtype == NEXEL_F16) {
    const int h2 = f.n_layers == 3 ? f.widths[2] : 0;
    return tc_arch_supported(f.widths[0], f.widths[1], h2, f.widths[f.n_layers],
                             s.grid_dtype == NEXEL_F16);
  }
  if (s.grid_dtype != NEXEL_F32) return false;  // the FP32 form reads an FP32 table
#define X(a, b, c, o) if (arch_match(f, a, b, c, o)) return true;
  NEXEL_ARCH_LIST(X)
#undef X
  return false;
}

cudaError_t launch_texture_fwd(const DevCam& c, const nexel_settings& s, const nexel_field& f,
                               const float* notex, const float* weights, const int* ids,
                               const float* depths, const float* T_final, float* image,
                               float* textures, void* feat_cache, int* status, cudaStream_t st) {
  FieldDev fd = make_fielddev(c, f);
  fd.feat = feat_cache;
  fd.feat_mode = feat_cache ? 1 : 0;
  if (s.mlp_dtype == NEXEL_BF16 || s.mlp_dtype == NEXEL_F16)
    return launch_texture_fwd_tc(c, s, f, fd, notex, weights, ids, depths, T_final, image,
                                 textures, status, st);
#define X(a, b, cc, o)                                                                            \
  if (arch_match(f, a, b, cc, o))                                                                  \
    return tex_fwd_f32<a, b, cc, float, o>(c, s, fd, notex, weights, ids, depths, T_final, image, \
                                           textures, st);
  NEXEL_ARCH_LIST(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_texture_bwd(const DevCam& c, const nexel_settings& s, const nexel_field& f,
                               char* bws, const BwdLayout& B, const float* weights, const int* ids,
                               const float* depths, const float* d_image, const float* d_weights,
                               const float* d_textures, float* d_table, float* d_mlp,
                               bool feat_cached, int grad_mode, cudaStream_t st) {
  FieldDev fd = make_fielddev(c, f);
  fd.grad_mode = grad_mode;
  fd.feat = bws + B.feat;
  fd.feat_mode = feat_cached ? 2 : 0;
  if (s.mlp_dtype == NEXEL_BF16 || s.mlp_dtype == NEXEL_F16) {
    // tcgen05 backward from the features (cached by the forward of a
    // training step, else gathered again here), then the hash-grid backward
    int KP = 1;
    while (KP < s.K) KP <<= 1;
    const long long n_rows = ((long long)c.W * c.H * KP + 15) / 16 * 16;
    cudaError_t e = cudaSuccess;
    if (!feat_cached)
      e = launch_texture_gather_tc(c, s, f, fd, ids, depths, (uint32_t*)(bws + B.feat), st);
    const int h2 = f.n_layers == 3 ? f.widths[2] : 0;
    if (e == cudaSuccess)
      e = launch_texture_bwd_tc(c, s.K, KP, n_rows, f.widths[0], f.widths[1], h2,
                                f.widths[f.n_layers], s.mlp_dtype == NEXEL_F16, f.weights, (const uint32_t*)(bws + B.feat),
                                weights, ids, d_image, d_weights, d_textures,
                                (float*)(bws + B.dweff), (float2*)(bws + B.gin), d_mlp,
                                (int*)(bws + B.status), st);
    if (e != cudaSuccess) return e;
    return launch_hash_bwd(c, fd, s.K, KP, n_rows, s.grid_dtype == NEXEL_F16, ids, depths,
                           (const float2*)(bws + B.gin), (float*)(bws + B.ddepth), d_table, st);
  }
#define X(a, b, cc, o)                                                                       \
  if (arch_match(f, a, b, cc, o))                                                            \
    return tex_bwd_f32<a, b, cc, float, o>(c, s, fd, bws, B, weights, ids, depths, d_image,   \
                                           d_weights, d_textures, d_table, d_mlp, st);
  NEXEL_ARCH_LIST(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace nexel
