// FP32 texturing kernels for the 32 -> 64 -> 64 -> 48 MLP (degree-3 SH texture
// coefficients), in a translation unit of its own so that it compiles in
// parallel with the 3-output form.
#include "texture_f32.cuh"

namespace nexel {
template cudaError_t tex_fwd_f32<32, 64, 64, float, 48>(
    const DevCam&, const nexel_settings&, const FieldDev&, const float*, const float*, const int*,
    const float*, const float*, float*, float*, cudaStream_t);
template cudaError_t tex_bwd_f32<32, 64, 64, float, 48>(
    const DevCam&, const nexel_settings&, const FieldDev&, char*, const BwdLayout&, const float*,
    const int*, const float*, const float*, const float*, const float*, float*, float*,
    cudaStream_t);
}  // namespace nexel
