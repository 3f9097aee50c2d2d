/*
 * nexel.h — C ABI of the Nexels image-formation library (libnexel.so).
 *
 * The library renders neurally-textured surfels ("nexels") on one CUDA
 * device and differentiates the result:
 *   nexel_preprocess  per-surfel projection, tile binning and the
 *                     (tile, centre-depth) ordering of Sec. 3 ("Preliminaries":
 *                     surfels are sorted by the depth of their centres and
 *                     alpha-composited by a tile-based rasterizer);
 *   nexel_render_fwd  the collection pass (Sec. 4.2: alpha, transmittance,
 *                     the non-textured render N of Eq. 5 and the per-pixel
 *                     top-K buffers I, W, D) followed by the texturing pass
 *                     (Sec. 4.2 and Eqs. 3-4: x = o + D d, down-weighted
 *                     hash-grid features, MLP G) and the composite of Eq. 6;
 *   nexel_render_bwd  the gradient of those outputs with respect to every
 *                     surfel parameter, the hash table and the MLP weights.
 *
 * Conventions shared by every entry point
 *   - All array pointers are DEVICE pointers to caller-owned memory unless a
 *     comment says "host".  The library never allocates or frees device
 *     memory; scratch lives in the caller's workspace (nexel_workspace_size).
 *   - Arrays are dense, C order, float32 unless stated: mu [N][3],
 *     quat [N][4] as (w, x, y, z) (need not be unit: it is normalised
 *     inside, with the gradient taken through the normalisation),
 *     scale [N][2] (sigma_1, sigma_2 > 0), opacity [N], gamma [N][2] (>= 1),
 *     color [N][3].  Per-pixel outputs are [H][W][...] with pixel
 *     (x, y) at index y * W + x.  Parameters are passed activated.
 *   - Camera: pinhole, pixel centres at (x + 0.5, y + 0.5), world_to_cam is
 *     a row-major 3x4 [R | t] with x_cam = R x_world + t, +z forward and +y
 *     down.  The ray of pixel (x, y) is o + t d with o the camera centre and
 *     d = R^T ((x + .5 - cx) / fx, (y + .5 - cy) / fy, 1), NOT normalised, so
 *     t equals view depth.
 *   - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the
 *     legacy default stream) except nexel_preprocess, which synchronises the
 *     stream once to read the instance count back to the host, and
 *     nexel_read_status.
 *   - Return value: NEXEL_OK (0) or a negative NEXEL_ERR_* code; nothing is
 *     launched when an argument check fails.  nexel_status_string names it.
 */
#ifndef NEXEL_H_
#define NEXEL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NEXEL_OK 0
#define NEXEL_ERR_INVALID_ARG (-1)
#define NEXEL_ERR_CUDA (-2)
#define NEXEL_ERR_CAPACITY (-3)
#define NEXEL_ERR_UNSUPPORTED (-4)
#define NEXEL_ERR_TIMEOUT (-5)
#define NEXEL_ERR_NUMERIC (-6)

#define NEXEL_F32 0
#define NEXEL_F16 1
#define NEXEL_BF16 2

#define NEXEL_MAX_K 8
#define NEXEL_MAX_LEVELS 32
#define NEXEL_MAX_LAYERS 4
#define NEXEL_TILE 16

typedef void* nexel_stream_t; /* a cudaStream_t */

typedef struct {
  int width, height;
  float fx, fy, cx, cy;
  float world_to_cam[12];
  float near_plane; /* surfel centres and ray hits at depth <= near are dropped */
} nexel_camera;

/* Render settings.  alpha_min / alpha_max / T_min are the compositing
 * thresholds the paper inherits from 3DGS without stating them (defaults
 * 1/255, 0.99, 1e-4): a surfel with alpha < alpha_min is skipped, alpha is
 * clamped to alpha_max, and compositing stops before the surfel that would
 * take the transmittance below T_min.  K in 0..NEXEL_MAX_K is the number of
 * textured primitives per pixel (Sec. 4.2).  grid_dtype is the storage type
 * of the hash table (NEXEL_F32 or NEXEL_F16); mlp_dtype the arithmetic of
 * the MLP (NEXEL_F32: FP32 SIMT; NEXEL_BF16: BF16 operands on the tensor
 * cores with FP32 accumulation; NEXEL_F16: FP16 operands with FP32
 * accumulation, the backward scaling the gradient that enters the MLP by
 * 128 and unscaling the results, as the paper trains).  The tensor-core
 * forms support the MLPs 16 -> 64 -> OUT and 32 -> 64 -> 64 -> OUT with
 * OUT = 3, and with OUT = 48 (SH textures) on the FP16 table. */
typedef struct {
  int K;
  float alpha_min, alpha_max, T_min;
  float bg[3];
  int grid_dtype, mlp_dtype;
  /* 0: nexel_render_bwd reads the forward's saved I, W, D and T_final;
   * 1: it recomputes them (the collection pass runs again inside the
   * backward), so the caller need not keep them between the two calls and
   * passes NULL for them. */
  int recompute_buffers;
  /* 0: nexel_render_bwd gathers the hash-grid features of every textured
   * sample again; 1 (a training step): nexel_render_fwd leaves them in the
   * bwd_ws it is given, and the nexel_render_bwd that follows reads them
   * there instead.  Both calls must then get the same bwd_ws, with no other
   * call on it in between. */
  int cache_features;
  /* Per-primitive colour (Sec. 3: channel-wise spherical-harmonics
   * coefficients; Sec. 5: degree 3).  0: `color` is RGB [N][3], used as
   * is.  3: `color` is [N][16][3] coefficients of the real SH of degree
   * <= 3 (orthonormal, ordered by l then m = -l..l, Condon-Shortley phase),
   * evaluated in the direction from the camera centre to the surfel centre:
   * colour = 1/2 + sum_k Y_k(dir) c_k; d_color of nexel_render_bwd is then
   * [N][16][3] (16-byte aligned, else NEXEL_ERR_INVALID_ARG) and d_mu
   * includes the path through the direction. */
  int sh_degree;
} nexel_settings;

/* Neural field of Sec. 3 ("Instant-NGP") and Eq. 4: L hash tables of T
 * entries (T a power of two) with F features (F = 2), level scales s_l, and
 * an MLP without bias: widths[0] = L * F -> hidden ... -> widths[n_layers]
 * = 3 (RGB texture) or 48 (the texture's degree-3 SH coefficients o[3k + ch],
 * Sec. 3 and Sec. 5, evaluated in the pixel's normalised ray direction:
 * T_ch = sum_k Y_k(d / |d|) o[3k + ch]; the FP32 form with 64-wide hidden
 * layers, the tensor-core forms with the FP16 table), ReLU on hidden
 * layers, linear output.  weights are float32 packed
 * layer after layer, layer l row-major [widths[l+1]][widths[l]].  Hidden
 * widths must be multiples of 16 and at most 64; L * F a multiple of 8 and at
 * most 64. */
typedef struct {
  int L, T, F;
  float level_scale[NEXEL_MAX_LEVELS]; /* host values, s_l per world unit */
  const void* table;                   /* device [L][T][F], grid_dtype */
  int n_layers;
  int widths[NEXEL_MAX_LAYERS + 1];
  const float* weights; /* device, float32 */
} nexel_field;

/* Bytes of device workspace needed for N surfels and up to max_instances
 * (tile, surfel) pairs on this camera.  Writes *bytes (host).  The same
 * workspace must be passed, with the same ws_bytes, to nexel_preprocess and
 * to the nexel_render_fwd / nexel_render_bwd calls that follow it; its
 * instance capacity is derived from ws_bytes. */
int nexel_workspace_size(const nexel_camera* cam, int N, long long max_instances, size_t* bytes);

/* Bytes of the separate backward scratch (per-sample texture gradients and
 * field features) for this camera, K and field.  Writes *bytes (host). */
/* With settings->recompute_buffers the scratch also holds the recomputed
 * per-pixel buffers. */
int nexel_bwd_workspace_size(const nexel_camera* cam, const nexel_settings* settings,
                             const nexel_field* field, size_t* bytes);

/* Geometry preprocess and binning (Sec. 3, "Preliminaries", and Sec. 4.1,
 * the generalised-Gaussian kernel alpha = o exp(-|u|^(2 g1)/2) exp(-|v|^(2 g2)/2)):
 * per surfel the camera-space frame, the exact screen footprint of the
 * region where alpha >= alpha_min, the tiles it touches; then a stable radix
 * sort of surfels by centre depth (culled: centre depth <= near,
 * opacity < alpha_min, a surfel seen edge-on -- |d_mu . n| < 1e-7 for the
 * centre ray d_mu at unit depth, whose plane then passes through the camera
 * centre -- and a surfel with a NaN or infinite parameter, which is counted
 * for nexel_render_stats and nexel_read_status) and the per-tile lists of (tile, depth-rank)
 * instances in rank order, bit-exact (each instance placed directly at its
 * slot, or, for 64-bit keys or more than 8192 tiles, a stable radix sort of
 * the instances by tile).  Results stay in `ws`.  Writes the number of
 * instances to *n_instances_out (host); returns NEXEL_ERR_CAPACITY, without
 * binning, if it exceeds the capacity `ws` was sized for. */
int nexel_preprocess(const nexel_camera* cam, const nexel_settings* settings, int N,
                     const float* mu, const float* quat, const float* scale,
                     const float* opacity, const float* gamma, const float* color, void* ws,
                     size_t ws_bytes, long long* n_instances_out, nexel_stream_t stream);

/* Forward render, after nexel_preprocess on the same ws.  Outputs (device,
 * caller-owned, fully overwritten):
 *   image    [H][W][3]  C = N + sum_j W_j T_j + T_final bg     (Eq. 6)
 *   notex    [H][W][3]  N, non-textured render without the K  (Eq. 5)
 *   weights  [H][W][K]  W, blending weights w = alpha T, descending
 *   ids      [H][W][K]  I, surfel index, -1 for an empty slot (int32)
 *   depths   [H][W][K]  D, ray parameter t* of the intersection, 0 if empty
 *   textures [H][W][K][3] T_j = G(Delta * H(o + D_j d)), 0 if empty (Eq. 4)
 *   T_final  [H][W]     transmittance after the last composited surfel
 * Ties in weight keep the front-most surfel.  bwd_ws / bwd_ws_bytes: the
 * backward scratch (nexel_bwd_workspace_size) when settings->cache_features
 * is set and K > 0 (else NEXEL_ERR_INVALID_ARG); otherwise unused and may be
 * NULL / 0. */
int nexel_render_fwd(const nexel_camera* cam, const nexel_settings* settings,
                     const nexel_field* field, int N, void* ws, size_t ws_bytes, void* bwd_ws,
                     size_t bwd_ws_bytes, float* image, float* notex, float* weights, int* ids,
                     float* depths, float* textures, float* T_final, nexel_stream_t stream);

/* Backward of nexel_render_fwd (same ws, same saved outputs).  Upstream
 * gradients: d_image [H][W][3] (required); d_weights [H][W][K] and
 * d_textures [H][W][K][3] may be NULL.  The discrete choices (order,
 * skips, early stop, top-K) are held fixed.  Gradient outputs (device,
 * float32, shaped like their parameters; d_table is [L][T][F] float32 and
 * d_mlp is packed like field->weights) are overwritten, or added to when
 * accumulate != 0.  Any gradient pointer may be NULL to skip it.  bwd_ws is
 * scratch of nexel_bwd_workspace_size bytes.  Requires alpha_max < 1 (the
 * replay divides by 1 - alpha).  The colour gradient flows only to surfels
 * composited untextured (Eq. 5).  The gradient outputs belong to the call
 * until it completes on `stream`: no other work may read or write them
 * meanwhile (d_table is held in a reordered form while the hash-grid
 * backward runs -- entries 1 and 2 of each 4-entry group swapped -- and
 * restored before the call's last kernel ends). */
int nexel_render_bwd(const nexel_camera* cam, const nexel_settings* settings,
                     const nexel_field* field, int N, const float* mu, const float* quat,
                     const float* scale, const float* opacity, const float* gamma, void* ws,
                     size_t ws_bytes, void* bwd_ws, size_t bwd_ws_bytes, const float* weights,
                     const int* ids, const float* depths, const float* T_final,
                     const float* d_image, const float* d_weights, const float* d_textures,
                     int accumulate, float* d_mu, float* d_quat, float* d_scale, float* d_opacity,
                     float* d_gamma, float* d_color, float* d_table, float* d_mlp,
                     nexel_stream_t stream);

/* Device-count preprocess: the same work as nexel_preprocess, but the
 * instance count stays on the device, so nothing synchronises the stream and
 * the call can be captured in a CUDA graph.  Launches are sized for the
 * instance capacity ws_bytes gives (nexel_workspace_size); instances beyond
 * it are dropped, which leaves a partial render and sets the capacity flag
 * that nexel_read_status reports.  Returns only argument / launch errors. */
int nexel_preprocess_async(const nexel_camera* cam, const nexel_settings* settings, int N,
                           const float* mu, const float* quat, const float* scale,
                           const float* opacity, const float* gamma, const float* color,
                           void* ws, size_t ws_bytes, nexel_stream_t stream);

/* Batched multi-view training step (a deployment form: the paper renders
 * one view per call; each view follows the same passages as
 * nexel_preprocess / nexel_render_fwd / nexel_render_bwd).  n_views cameras
 * (cams: host array of n_views structs, resolutions may differ) of one
 * scene.  Every per-view argument is a host array of n_views entries: view
 * v has its own workspace ws[v] of ws_bytes[v] bytes, its own backward
 * scratch bwd_ws[v] (bwd_ws_bytes[v]; either array may be NULL when no
 * view needs scratch) and its own outputs, laid out as in
 * nexel_render_fwd.  nexel_render_batch_fwd runs the device-count
 * preprocess and the forward render of every view; nothing synchronises
 * the stream, so the pair can be captured in one CUDA graph.  The views run
 * as parallel branches: forked from `stream` onto streams the library owns
 * (created on the device's first batched call; make that call before a
 * capture) and joined back into it before the call returns, so later work
 * on `stream` sees every view's results.  nexel_render_batch_bwd sums the
 * gradients of all views into d_mu ... d_mlp (overwritten, or added to when
 * accumulate != 0), with atomics, so their summation order varies between
 * runs by rounding only.  d_weights and d_textures may be NULL arrays or
 * hold NULL entries.  All views' arguments are checked before any launch.
 * Capacity overflows and device timeouts are read per view with
 * nexel_read_status. */
int nexel_render_batch_fwd(int n_views, const nexel_camera* cams, const nexel_settings* settings,
                           const nexel_field* field, int N, const float* mu, const float* quat,
                           const float* scale, const float* opacity, const float* gamma,
                           const float* color, void* const* ws, const size_t* ws_bytes,
                           void* const* bwd_ws, const size_t* bwd_ws_bytes, float* const* image,
                           float* const* notex, float* const* weights, int* const* ids,
                           float* const* depths, float* const* textures, float* const* T_final,
                           nexel_stream_t stream);
int nexel_render_batch_bwd(int n_views, const nexel_camera* cams, const nexel_settings* settings,
                           const nexel_field* field, int N, const float* mu, const float* quat,
                           const float* scale, const float* opacity, const float* gamma,
                           void* const* ws, const size_t* ws_bytes, void* const* bwd_ws,
                           const size_t* bwd_ws_bytes, const float* const* weights,
                           const int* const* ids, const float* const* depths,
                           const float* const* T_final, const float* const* d_image,
                           const float* const* d_weights, const float* const* d_textures,
                           int accumulate, float* d_mu, float* d_quat, float* d_scale,
                           float* d_opacity, float* d_gamma, float* d_color, float* d_table,
                           float* d_mlp, nexel_stream_t stream);

/* Reads and clears the device status words of one view's workspaces
 * (bwd_ws may be NULL), synchronising the stream: NEXEL_ERR_TIMEOUT if a
 * bounded device wait of a tensor-core kernel ran out (that kernel's
 * results are invalid; the words cover the last preprocess and forward on
 * ws, which the preprocess resets, and the last backward on bwd_ws, which
 * that backward resets), else NEXEL_ERR_CAPACITY if a device-count
 * preprocess dropped instances, else NEXEL_ERR_NUMERIC if a preprocess
 * culled a surfel with a NaN or infinite parameter (or a zero quaternion:
 * such a surfel is skipped by the render and gets zero gradients;
 * nexel_render_stats counts them), else NEXEL_OK. */
int nexel_read_status(const nexel_camera* cam, const nexel_settings* settings,
                      const nexel_field* field, int N, void* ws, size_t ws_bytes, void* bwd_ws,
                      size_t bwd_ws_bytes, nexel_stream_t stream);

/* Training objective of Sec. 5 ("Losses"):
 *   L = (1 - l_dssim) L_1 + l_dssim L_D-SSIM + l_alpha L_alpha
 *       + l_texture L_texture + l_opacity L_opacity + l_grid L_grid
 * with the paper's weights l_dssim 0.2, l_alpha 0.005, l_texture 0.5,
 * l_opacity 0.01, l_grid 0.01.  L_D-SSIM = 1 - SSIM (3DGS's form: 11 x 11
 * Gaussian window, sigma 1.5, zero padding, C1 = 0.01^2, C2 = 0.03^2, mean
 * over pixels and channels); L_texture averages |I_GT - sum_j W_j T_j /
 * sum_j W_j| (pixels with sum_j W_j = 0 add nothing); L_alpha averages
 * 1 - sum_j W_j; L_opacity averages the opacities; L_grid =
 * sum_l s_l^-3 sum_{i,j} H_{l,i,j}^2 (the printed formula indexes s by the
 * entry and leaves H unsquared; this is the reading).  |.| has derivative
 * sign(.), sign(0) = 0. */
typedef struct {
  float dssim, alpha, texture, opacity, grid;
} nexel_loss_weights;

/* Bytes of device scratch for the objective on a width x height image. */
int nexel_loss_workspace_size(int width, int height, size_t* bytes);

/* Image-space terms.  image, target [H][W][3]; weights [H][W][K] and
 * textures [H][W][K][3] are the forward's W and T (may be NULL when K = 0:
 * the texture and alpha terms are then 0).  Writes (device, overwritten)
 * d_image = dL/dimage, d_weights = dL/dW, d_textures = dL/dT -- the upstream
 * gradients nexel_render_bwd takes -- and values[0..4] = L_1, L_D-SSIM,
 * L_texture, L_alpha and the weighted sum of these four (device floats,
 * summed in a fixed order, so repeated calls give identical values). */
int nexel_loss_image(int width, int height, int K, const nexel_loss_weights* lw,
                     const float* image, const float* target, const float* weights,
                     const float* textures, void* ws, size_t ws_bytes, float* values,
                     float* d_image, float* d_weights, float* d_textures, nexel_stream_t stream);

/* Parameter-space terms, after nexel_loss_image and nexel_render_bwd on the
 * same values array and ws (with the same width and height): ADDS
 * l_opacity / N to every d_opacity[i] and l_grid 2 s_l^-3 H to every
 * d_table entry (either pointer may be NULL), and writes values[5] =
 * L_opacity, values[6] = L_grid, values[7] = the total L.  table is the
 * FP32 master table [L][T][F] (field->table is not read); field may be NULL
 * (no grid term). */
int nexel_loss_params(int N, const float* opacity, const nexel_field* field, const float* table,
                      const nexel_loss_weights* lw, void* ws, size_t ws_bytes, int width,
                      int height, float* values, float* d_opacity, float* d_table,
                      nexel_stream_t stream);

/* One Adam step (Kingma and Ba; the optimiser of the 3DGS scheme the paper
 * follows) over n_tensors FP32 tensors in one launch per 16 tensors:
 * m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
 * p -= lr m / (1 - b1^step) / (sqrt(v / (1 - b2^step)) + eps).  Host arrays
 * of device pointers params, grads, m, v (moments start at zero), host
 * arrays sizes (elements) and lrs (per-tensor learning rate); step >= 1. */
int nexel_adam_step(int n_tensors, float* const* params, const float* const* grads,
                    float* const* m, float* const* v, const long long* sizes, const float* lrs,
                    float beta1, float beta2, float eps, int step, nexel_stream_t stream);

/* Adaptive density control (supp. Sec. 7.2; Sec. 5, "Adaptive Density
 * Control").
 *
 * nexel_fps: farthest point sampling of n points [n][3] (device): idx[0] =
 * 0, then idx[i] = the unselected point farthest from the selected ones
 * (ties: lowest index); d2sel[i] = its squared distance to them at
 * selection (d2sel[0] = +inf).  scale (nullable) receives the paper's
 * initial scale of each sampled point: the distance at which it was
 * selected, sqrt(d2sel[i]) (its nearest neighbour among the points sampled
 * before it), with scale[0] = scale[1] (the first point has no
 * predecessor; 0 when m = 1).  Squared distances are formed in FP32 with
 * every operation rounded, ((dx dx + dy dy) + dz dz).  scratch: n floats.
 * One CTA, m iterations: an initialisation step, not a per-iteration one.
 *
 * nexel_blend_error: ADDS to err[i] (original order) the blended L1 error of
 * Rota Bulo et al. that the paper accumulates across iterations:
 * sum over pixels of w e_p, w = alpha T the compositing weight of surfel i
 * at the pixel and e_p the mean over channels of |image - target|.  Runs on
 * the workspace of the last nexel_preprocess of this view.
 *
 * nexel_densify_count: the number of surfels a density step splits: 5 %
 * of the N current ones, rounded up, capped so that the total stays within
 * the budget P (the paper's primitive budget): max(0, min(ceil(N / 20),
 * budget - N)).  Host only; writes *n_select (host).
 *
 * nexel_densify_select: draws the surfels to split, nexel_densify_count(N,
 * budget) of them, without replacement with probabilities proportional to
 * err (Efraimidis-Spirakis): the caller passes exponential random numbers
 * expo[i] (mean 1), the call returns in sel the indices of the n_select
 * smallest expo[i] / err[i] (FP32; err[i] = 0 never drawn while a positive
 * error remains; ties by index) in increasing key order, and n_select in
 * *n_select_out (host).  sel (device) must hold ceil(N / 20) entries.
 *
 * nexel_densify_split: surfel sel[r] becomes two with scales halved along
 * the longer axis (v1 if sigma1 >= sigma2, else v2) and centres
 * mu -/+ (sigma_long / 2) v_long; the first stays at sel[r], the second
 * goes to index N + r; every other property is copied.  The arrays hold
 * N + n_select surfels; color has color_dim (3 or 48) floats per surfel.
 *
 * nexel_prune: copies the surfels with opacity >= threshold (the paper:
 * 0.005), in order, to the output arrays and writes their count to n_out
 * (device int).
 *
 * Scratch of the selection and the prune: nexel_density_workspace_size. */
int nexel_fps(int n, const float* points, int m, float* scratch, int* idx, float* d2sel,
              float* scale, nexel_stream_t stream);
int nexel_blend_error(const nexel_camera* cam, const nexel_settings* settings, int N, void* ws,
                      size_t ws_bytes, const float* image, const float* target, float* err,
                      nexel_stream_t stream);
int nexel_density_workspace_size(int N, size_t* bytes);
int nexel_densify_count(int N, long long budget, int* n_select);
int nexel_densify_select(int N, const float* err, const float* expo, long long budget, void* ws,
                         size_t ws_bytes, int* sel, int* n_select_out, nexel_stream_t stream);
int nexel_densify_split(int N, int n_select, const int* sel, int color_dim, float* mu, float* quat,
                        float* scale, float* opacity, float* gamma, float* color,
                        nexel_stream_t stream);
int nexel_prune(int N, float threshold, int color_dim, const float* mu, const float* quat,
                const float* scale, const float* opacity, const float* gamma, const float* color,
                void* ws, size_t ws_bytes, float* mu_out, float* quat_out, float* scale_out,
                float* opacity_out, float* gamma_out, float* color_out, int* n_out,
                nexel_stream_t stream);

/* Launch-shape tuning (process-wide; no counterpart in the paper): CTAs
 * per SM that the persistent texturing kernels keep in flight -- the tile
 * pipeline depth of the tcgen05 forward (1..2, default 2), of the tcgen05
 * backward (1..3, default 3: tiles in flight per SM; 3 is one CTA of three
 * tile groups with a dedicated MMA warp, for RGB textures with two hidden
 * layers of 64 units and up to 32 inputs, and means 2 for other shapes; 1
 * where the shared memory of the other shapes allows one) and of
 * the FP32 chunked kernels (1..2, default 2) -- the CTA size of the hash
 * backward (128 or 256, default 256), the number of surfel records the
 * collection kernels stage in shared memory per batch (128, 256 or 512,
 * default 256; Sec. 3's tile-based rasterizer walks each 16 x 16 tile's
 * list in such batches) and the depth of the tcgen05 forward's ring of
 * operand tiles (2..4, default 4: how many tiles its gather warps may run
 * ahead of its MMAs).  Every choice computes the same values; the weight-gradient and table-gradient sums may differ by
 * rounding (their atomic order).  nexel_autotune runs the caller's own
 * training step (preprocess once, then forward + backward per candidate,
 * `reps` timed steps after an untimed one, CUDA events on `stream`; with a
 * device buffer `flush` of flush_bytes > 0, larger than the L2, it is
 * written before every timed step so that each starts from a cold L2),
 * tunes one knob after another keeping the fastest value (a value replaces
 * the current one only when at least 1 % faster), leaves the best
 * tuning set and returns it (and its median step time in ms); it
 * synchronises the stream.  Arguments as for nexel_render_fwd /
 * nexel_render_bwd (gradients are overwritten). */
typedef struct {
  int tex_fwd_ctas_per_sm, tex_bwd_ctas_per_sm, f32_ctas_per_sm, hash_block;
  int collect_batch, tex_fwd_stages;
} nexel_tuning;
int nexel_get_tuning(nexel_tuning* out);

/* Test hook of the failure path (no counterpart in the paper).  With
 * polls in 1..65536 the tensor-core texturing kernels (forward and
 * backward) launched afterwards issue no MMA and give up each wait for MMA
 * completion after `polls` polls of its mbarrier, which nothing then
 * arrives at: each CTA ends its tile loop, frees its TMEM, returns, and
 * sets the timeout bit that nexel_read_status reports as
 * NEXEL_ERR_TIMEOUT (the outputs of those launches are invalid).  No GPU
 * fault and no unbounded wait is involved.  polls = 0 (the default)
 * restores normal operation.  Process-wide. */
int nexel_test_tc_wait_timeout(int polls);
int nexel_set_tuning(const nexel_tuning* t);
int nexel_autotune(const nexel_camera* cam, const nexel_settings* settings,
                   const nexel_field* field, int N, const float* mu, const float* quat,
                   const float* scale, const float* opacity, const float* gamma,
                   const float* color, void* ws, size_t ws_bytes, void* bwd_ws,
                   size_t bwd_ws_bytes, float* image, float* notex, float* weights, int* ids,
                   float* depths, float* textures, float* T_final, const float* d_image,
                   float* d_mu, float* d_quat, float* d_scale, float* d_opacity, float* d_gamma,
                   float* d_color, float* d_table, float* d_mlp, int reps, void* flush,
                   size_t flush_bytes, nexel_tuning* best, float* best_ms,
                   nexel_stream_t stream);

/* Inspection of the binning done by the last nexel_preprocess on ws: the
 * n_instances (tile, surfel) pairs in the order the collection pass walks
 * them, i.e. by tile, then by centre view depth (Sec. 3, "Preliminaries"),
 * then by surfel index.  Writes tile index (ty * tiles_x + tx), surfel index
 * and the float32 centre depth used as the sort key; any output may be NULL.
 * Device outputs of n_instances elements each. */
int nexel_instance_list(const nexel_camera* cam, int N, const void* ws, size_t ws_bytes,
                        long long n_instances, int* tile_out, int* id_out, float* depth_out,
                        nexel_stream_t stream);

/* Work statistics of the last nexel_render_fwd on ws (a device reduction;
 * synchronises `stream`).  Writes out[8] (host):
 *   out[0] (tile, surfel) instances of the binning (Sec. 3, "Preliminaries"),
 *   out[1] surfels with at least one instance (not culled, on screen),
 *   out[2] sum over pixels of the last list position the pixel composited
 *          (Sec. 4.2): the (pixel, surfel) pairs the collection backward
 *          evaluates, a lower bound of those the forward evaluates,
 *   out[3] sum over tiles of list length x pixels of the tile: the pairs a
 *          pass without early termination would evaluate,
 *   out[4] the longest tile list, out[5] the number of 16 x 16 tiles,
 *   out[6] sum over tiles of (largest last list position of its pixels) x
 *          pixels of the tile: the pair evaluations the collection backward
 *          runs (every thread of a tile walks back from the tile's largest),
 *   out[7] surfels the last preprocess culled for a NaN or infinite
 *          parameter (or a zero quaternion).
 * The counters block of ws holds the reduction; nothing else is changed. */
int nexel_render_stats(const nexel_camera* cam, const nexel_settings* settings, int N,
                       void* ws, size_t ws_bytes, long long* out, nexel_stream_t stream);

/* Instrumentation (no counterpart in the paper).  nexel_launch_count: the
 * number of kernels this library has launched in the process.
 * nexel_profile_enable(1) starts recording a CUDA event pair on the launch
 * stream around every kernel launch (0 stops and discards);
 * nexel_profile_read synchronises those events and reports, per kernel
 * name, the summed device time in ms and the launch count: up to
 * max_entries rows into names (32 chars each, host), total_ms and launches
 * (host arrays), and the number of distinct kernels into *n_out. */
long long nexel_launch_count(void);
int nexel_profile_enable(int on);
int nexel_profile_read(int max_entries, char* names, float* total_ms, int* launches, int* n_out);

/* Device measurement (no counterpart in the paper): the rate of random
 * float2 reductions (red.global.add of two float32) into an L2-resident
 * table, the resource that bounds the hash-grid backward's scatter (the
 * adjoint of the trilinear lookup, Eq. 4).  buf (device, 8-byte aligned,
 * buf_bytes >= 8) holds the table: its largest power-of-two count of float2
 * entries that fits is zeroed, then each of `reps` launches adds (1, 1) at
 * n_ops hashed indices; the table then holds 2 * n_ops * reps in total.
 * Writes the median rate over the reps in 1e9 reductions per second to
 * *gops_out (host).  Synchronises `stream`. */
int nexel_peak_l2_reductions(void* buf, size_t buf_bytes, long long n_ops, int reps,
                             float* gops_out, nexel_stream_t stream);

/* Allocation-free forward render (the paper has no counterpart: this is a
 * deployment variant).  For callers that cannot allocate device memory --
 * e.g. a plugin inside a host application that owns all device
 * allocations, or a frame callback on a fixed memory budget where an
 * allocation could synchronise the device -- this runs nexel_preprocess and
 * nexel_render_fwd with a workspace that is a file-scope device array of the
 * library (12 MiB on each device that uses it, held until the process
 * exits) instead of caller memory; it allocates nothing.  Inputs and outputs
 * are as for nexel_preprocess / nexel_render_fwd; settings->cache_features
 * must be 0 when K > 0 (no backward follows, so there is no scratch to
 * cache features in; else NEXEL_ERR_INVALID_ARG, nothing launched).
 * Limits: N <= 16384 surfels and width * height <= 65536 pixels (else
 * NEXEL_ERR_INVALID_ARG, nothing launched); more (tile, surfel) instances
 * than the array holds returns NEXEL_ERR_CAPACITY with the count in
 * *n_instances_out.  Like nexel_preprocess, every call synchronises the
 * stream once to read the instance count back, so no call can be captured
 * into a CUDA graph.  The first call on a device resolves the array's device
 * address (once per device, with that device current, kept for the life of
 * the process: do not use the library across a cudaDeviceReset of that
 * device).  All calls share the array: calls that overlap on the
 * GPU race, so serialise them; it keeps the previous call's contents, and
 * the pipeline clears what must start at zero itself. */
int nexel_render_fwd_static(const nexel_camera* cam, const nexel_settings* settings,
                            const nexel_field* field, int N, const float* mu, const float* quat,
                            const float* scale, const float* opacity, const float* gamma,
                            const float* color, float* image, float* notex, float* weights,
                            int* ids, float* depths, float* textures, float* T_final,
                            long long* n_instances_out, nexel_stream_t stream);

/* Human-readable name of a status code (static string). */
const char* nexel_status_string(int status);

/* Library version (major * 10000 + minor * 100 + patch). */
int nexel_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NEXEL_H_ */
