// Forward render for callers that cannot allocate device memory.
//
// Some callers of this library run where they may not call cudaMalloc: a
// renderer plugin inside a host application that owns every device
// allocation, a frame callback with a fixed memory budget where an
// allocation (which can synchronise the device) would stall the frame, or a
// caller that simply has no allocator of its own.  For them,
// nexel_render_fwd_static runs the same preprocess, binning and forward
// render as nexel_preprocess + nexel_render_fwd, but its workspace is the
// file-scope device array below instead of caller memory.  It calls no
// cudaMalloc / cudaFree and no allocating library routine.
//
// Costs and limits: every process that loads the library holds the array
// (kStaticBytes) on each device it uses, until the process exits.  Calls
// share the one array, so two calls whose work overlaps on the GPU (two
// streams, or two host threads) race and corrupt each other's results;
// serialise them.  The array keeps the last call's contents; the pipeline
// clears what must start at zero (instance counter, tile ranges) itself.
// Each call synchronises the stream once, as nexel_preprocess does, to read
// the instance count back.  The device address of the array is resolved once
// per device and kept: do not use the library across a cudaDeviceReset of
// that device.
#include "common.cuh"

#include <mutex>

namespace nexel {
namespace {

constexpr size_t kStaticBytes = size_t(12) << 20;  // 12 MiB per device
constexpr int kStaticMaxN = 16384;                 // surfels
constexpr long long kStaticMaxPixels = 65536;      // e.g. 256 x 256
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_ws[kStaticBytes];

std::mutex g_static_mu;
void* g_static_ptr[kMaxDevices] = {};

// Host code may not use g_static_ws directly: on the host that name is a
// stand-in, not a device address.  Resolve the device address once per
// device, with that device current.
int static_ws_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return NEXEL_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return NEXEL_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_ws) != cudaSuccess || !p) return NEXEL_ERR_CUDA;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return NEXEL_OK;
}

}  // namespace
}  // namespace nexel

using namespace nexel;

extern "C" int nexel_render_fwd_static(const nexel_camera* cam, const nexel_settings* settings,
                                       const nexel_field* field, int N, const float* mu,
                                       const float* quat, const float* scale,
                                       const float* opacity, const float* gamma,
                                       const float* color, float* image, float* notex,
                                       float* weights, int* ids, float* depths, float* textures,
                                       float* T_final, long long* n_instances_out,
                                       nexel_stream_t stream) {
  if (!cam || !settings || !n_instances_out) return NEXEL_ERR_INVALID_ARG;
  if (N < 0 || N > kStaticMaxN) return NEXEL_ERR_INVALID_ARG;
  // a render without a backward: there is no backward scratch to cache
  // features in
  if (settings->cache_features != 0 && settings->K > 0) return NEXEL_ERR_INVALID_ARG;
  if (cam->width <= 0 || cam->height <= 0 ||
      (long long)cam->width * cam->height > kStaticMaxPixels)
    return NEXEL_ERR_INVALID_ARG;
  void* ws = nullptr;
  int rc = static_ws_address(&ws);
  if (rc != NEXEL_OK) return rc;
  rc = nexel_preprocess(cam, settings, N, mu, quat, scale, opacity, gamma, color, ws,
                        kStaticBytes, n_instances_out, stream);
  if (rc != NEXEL_OK) return rc;
  return nexel_render_fwd(cam, settings, field, N, ws, kStaticBytes, nullptr, 0, image, notex,
                          weights, ids, depths, textures, T_final, stream);
}
