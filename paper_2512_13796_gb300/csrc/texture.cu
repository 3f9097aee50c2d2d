// Dispatch of the texturing pass over the supported MLP shapes and storage
// types.  The FP32 kernels are in texture_f32.cuh, the BF16 tensor-core ones
// in texture_bf16.cu.
#include "texture_f32.cuh"

namespace nexel {

#define NEXEL_ARCH_LIST(X) \
  X(8, 16, 0)              \
  X(16, 64, 0)             \
  X(32, 64, 64)

// Explicit instantiations live in one translation unit per architecture
// (texture_f32_<in>_<h1>_<h2>.cu) so that they compile in parallel.
#define X(a, b, cc)                                                                              \
  extern template cudaError_t tex_fwd_f32<a, b, cc, float>(                                      \
      const DevCam&, const nexel_settings&, const FieldDev&, const float*, const float*,         \
      const int*, const float*, const float*, float*, float*, cudaStream_t);                     \
  extern template cudaError_t tex_bwd_f32<a, b, cc, float>(                                      \
      const DevCam&, const nexel_settings&, const FieldDev&, char*, const BwdLayout&,            \
      const float*, const int*, const float*, const float*, const float*, const float*, float*,  \
      float*, cudaStream_t);                                                                     \

NEXEL_ARCH_LIST(X)
#undef X

static bool arch_match(const nexel_field& f, int in, int h1, int h2) {
  if (h2 == 0) return f.n_layers == 2 && f.widths[0] == in && f.widths[1] == h1 && f.widths[2] == 3;
  return f.n_layers == 3 && f.widths[0] == in && f.widths[1] == h1 && f.widths[2] == h2 &&
         f.widths[3] == 3;
}

bool texture_arch_supported(const nexel_settings& s, const nexel_field& f) {
  if (f.F != 2 || f.L * f.F != f.widths[0]) return false;
  if (s.mlp_dtype == NEXEL_BF16) return bf16_arch_supported(f);
  if (s.grid_dtype != NEXEL_F32) return false;  // the FP32 form reads an FP32 table
#define X(a, b, c) if (arch_match(f, a, b, c)) return true;
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
  if (s.mlp_dtype == NEXEL_BF16)
    return launch_texture_fwd_tc(c, s, f, fd, notex, weights, ids, depths, T_final, image,
                                 textures, status, st);
#define X(a, b, cc)                                                                                \
  if (arch_match(f, a, b, cc))                                                                     \
    return tex_fwd_f32<a, b, cc, float>(c, s, fd, notex, weights, ids, depths, T_final, image, \
                                        textures, st);
  NEXEL_ARCH_LIST(X)
#undef X
  return cudaErrorInvalidValue;
}

cudaError_t launch_texture_bwd(const DevCam& c, const nexel_settings& s, const nexel_field& f,
                               char* bws, const BwdLayout& B, const float* weights, const int* ids,
                               const float* depths, const float* d_image, const float* d_weights,
                               const float* d_textures, float* d_table, float* d_mlp,
                               bool feat_cached, cudaStream_t st) {
  FieldDev fd = make_fielddev(c, f);
  fd.feat = bws + B.feat;
  fd.feat_mode = feat_cached ? 2 : 0;
  if (s.mlp_dtype == NEXEL_BF16)
    return launch_texture_bwd_bf16(c, s, f, fd, bws, B, weights, ids, depths, d_image, d_weights,
                                   d_textures, d_table, d_mlp, st);
#define X(a, b, cc)                                                                          \
  if (arch_match(f, a, b, cc))                                                               \
    return tex_bwd_f32<a, b, cc, float>(c, s, fd, bws, B, weights, ids, depths, d_image,      \
                                        d_weights, d_textures, d_table, d_mlp, st);
  NEXEL_ARCH_LIST(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace nexel
