/*
 * fgs.h - C ABI of the GB300 (sm_103a) fisheye Gaussian-splatting hot path.
 *
 * The method is Fisheye-GS (arXiv 2409.04751): 3D Gaussian splatting in which the pinhole
 * projection is replaced by the equidistant fisheye model r_d = f * theta (Sec. 3.2). The
 * path is the renderer's four stages (Sec. 4.1: preprocess, tile binning, sort, rasterize)
 * and their backward (Sec. 4.2, 4.3). Every stage runs in hand-written CUDA kernels.
 *
 * Conventions shared by every call:
 *  - All array pointers are DEVICE pointers unless stated otherwise; the caller allocates and
 *    owns every buffer (this library never allocates or frees device memory). Camera arrays
 *    and the background colour are HOST pointers, read during the call.
 *  - Every call is asynchronous and ordered on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream). No call synchronises the host, so a sequence of calls can be captured
 *    in a CUDA graph.
 *  - A call returns FGS_ERR_INVALID_ARG before launching anything if an argument is wrong
 *    (null pointer with a non-zero size, negative size, sh_degree outside 0..3, no views or
 *    more than FGS_MAX_VIEWS, a non-positive image size, a workspace that is too small, a
 *    record buffer not 16-byte aligned). FGS_ERR_CUDA reports a failed launch.
 *  - Errors found on the device (more intersections than `capacity`; a bounded wait that ran
 *    out) are written to a status word in the workspace; fgs_bin_sort resets it and
 *    fgs_read_status reads it. Outputs are then undefined but every access stays in bounds:
 *    after a wait of the binning ran out its later kernels do nothing, and while the word is
 *    set fgs_rasterize draws the background only and fgs_backward's screen-space pass adds
 *    nothing.
 *  - Gradients are overwritten, not accumulated. The workspace and every output buffer may hold
 *    anything before a call: each call clears or overwrites what it reads from them (the
 *    backward zeroes its accumulators itself; fgs_bin_sort writes every tile range).
 *  - The library keeps no settings of its own: the work shape, the measurement counters and
 *    the wait bound are chosen per call (fgs_options). Calls on distinct workspaces are
 *    independent; calls sharing a workspace must not overlap in time (they share its
 *    counters).
 *  - Checked build. The same sources compiled with -DFGS_CHECK=1 give libfgs_check.so, a
 *    debugging build with the same ABI and the same results on valid inputs. In it, every
 *    index a kernel reads from memory is compared with the size of the buffer it selects
 *    before it is used: record indices from `vals` and from the binning's compacted record
 *    list, tile ids from the binning's tile lists, sorted keys and the backward's tile order,
 *    and [start, end) of every tile in `tile_ranges`. An index outside sets FGS_ERR_BOUNDS in
 *    the status word and the access is skipped (the index taken as 0, the range as empty), so
 *    a corrupted input or a kernel bug shows up as a status and not as an access out of
 *    bounds. The rasterizers bound record indices and list ends by the record count and key
 *    capacity that the last fgs_bin_sort / fgs_bin_sort_ex on the same workspace recorded
 *    there (with no such binning, e.g. after fgs_bin_sort_noalloc, only start <= end is
 *    checked). The product build (libfgs.so) has none of these comparisons.
 */
#ifndef FGS_H
#define FGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *fgs_stream; /* == cudaStream_t */

typedef enum {
  FGS_OK = 0,
  FGS_ERR_INVALID_ARG = 1,
  FGS_ERR_CAPACITY = 2, /* more (Gaussian, tile) intersections than the key buffers hold */
  FGS_ERR_TIMEOUT = 3,  /* a bounded device-side wait gave up */
  FGS_ERR_CUDA = 4,
  FGS_ERR_BOUNDS = 5    /* checked build only: an index read from memory was out of range */
} fgs_status;

#define FGS_TILE 16        /* tiles are 16 x 16 pixels (Sec. 3.1 "Rendering") */
#define FGS_MAX_VIEWS 128  /* views per call */

/* Camera models. The method is the equidistant fisheye (Sec. 3.2, r_d = f theta). Sec. 3.2
 * names the other radial fisheye models, r_d = f r(theta) with r = 2 sin(theta/2)
 * (equisolid), 2 tan(theta/2) (stereographic), sin(theta) (orthographic), and Sec. 6
 * ("Extension to Other Camera Models") gives the equirectangular panorama:
 *   x_p = cx + fx atan2(x_c, z_c), y_p = cy + fy atan2(y_c, sqrt(x_c^2 + z_c^2)),
 * which with fx = w / 2 pi, cx = w / 2, fy = h / pi, cy = h / 2 is the paper's pair. */
typedef enum {
  FGS_CAM_EQUIDISTANT = 0,
  FGS_CAM_EQUISOLID = 1,
  FGS_CAM_STEREOGRAPHIC = 2,
  FGS_CAM_ORTHOGRAPHIC = 3,
  FGS_CAM_EQUIRECTANGULAR = 4,
  FGS_CAM_PINHOLE = 5 /* r = tan(theta): x_p = cx + fx x_c / z_c, the comparison camera */
} fgs_camera_model;

/* A camera (Sec. 3.1 "Transformation", Sec. 3.2):
 *   mu_c = W mu + b (W row-major, world -> camera; camera x right, y down, z forward),
 *   radial models: theta = atan2(|(x_c, y_c)|, z_c), x_p = cx + fx r(theta) x_c / l_z,
 *   y_p = cy + fy r(theta) y_c / l_z (r(theta) = theta for the equidistant model);
 *   panorama: as above. Field of view: theta < pi - 0.05 (orthographic, pinhole: pi/2 - 0.05), or
 *   |latitude| < pi/2 - 0.05 for the panorama, which does not wrap at longitude +-pi. The
 *   pinhole also culls a Gaussian whose projected mean lies outside the guard band
 *   |x_p - cx| <= 1.3 width / 2, |y_p - cy| <= 1.3 height / 2 (the 1.3 tan(FOV/2) limit of the
 *   pinhole renderer the method is compared with, applied as a cull).
 * Pixel (i, j) is sampled at (i + 0.5, j + 0.5).
 * A view holds at most 2^20 tiles and at most 65535 tile columns and rows (the record's tile
 * rect is 16-bit); a call with a larger view, or a model outside fgs_camera_model, returns
 * FGS_ERR_INVALID_ARG. */
typedef struct {
  float W[9];
  float b[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  int32_t model; /* fgs_camera_model */
} fgs_camera;

/* The Gaussian set (Sec. 3.1 "Definition"): device pointers, FP32, contiguous.
 *   means [n,3]; scales [n,3] (activated, > 0; S = diag(scales)); quats [n,4] (w, x, y, z,
 *   any non-zero norm: normalised inside); opacities [n] (activated, in (0, 1));
 *   sh [n, (sh_degree+1)^2, 3] real spherical-harmonic coefficients (Condon-Shortley phase,
 *   order l = 0..3, m = -l..l), colour = max(0, sum_k sh_k Y_k(dir) + 0.5). */
typedef struct {
  const float *means;
  const float *scales;
  const float *quats;
  const float *opacities;
  const float *sh;
  int64_t n;
  int32_t sh_degree;
} fgs_gaussians;

/* Per-(view, Gaussian) record written by fgs_preprocess, 48 bytes, 16-byte aligned.
 * Record r = v * n + i belongs to Gaussian i in view v.
 *   xy      projected mean mu_p (pixels)
 *   conic   (A, B, C) = inverse of Sigma_p + 0.3 I; alpha(p) = min(0.99, opacity *
 *           exp(-0.5 (A dx^2 + 2 B dx dy + C dy^2))), d = p - xy
 *   depth   |mu_c| (distance along the ray; the sort key's low 32 bits are its FP32 bits)
 *   rect    x0, y0, x1, y1: inclusive tile rectangle in the view's tile grid; it contains
 *           every pixel centre where alpha >= 1/255. Empty (tiles_touched = 0) if the
 *           Gaussian is culled: |mu_c| <= 0.2, theta >= pi - 0.05, opacity < 1/255, or the
 *           footprint misses the image. Other fields are unspecified then. */
typedef struct {
  float xy[2];
  float conic[3];
  float opacity;
  float rgb[3];
  float depth;
  uint16_t rect[4];
} fgs_record;

/* Per-call options of fgs_bin_sort_ex, fgs_rasterize_ex, fgs_backward_ex and
 * fgs_backward_raster_ex (HOST pointer, read during the call; NULL = every field 0 = the
 * defaults). None of them changes a result beyond the order of floating-point sums.
 *   fwd_pixels_per_thread  work shape of the forward rasterizer: 1, 2 or 4 pixels per thread
 *                          (a 16x16 tile runs on 256 / that many threads); 0 = 4.
 *   bwd_pixels_per_thread  the same for the backward rasterizer: 1, 2, 4 or 8 (8 = one warp
 *                          per tile); 0 = 8.
 *                          Images, final transmittances and processed counts do not depend on
 *                          either, bit for bit; gradients only through the order of their
 *                          floating-point sums. A tuner may pick whichever is fastest.
 *   flags                  FGS_OPT_INSTRUMENT: fgs_rasterize_ex and fgs_backward_ex /
 *                          fgs_backward_raster_ex launch variants of their kernels that also
 *                          count work into the workspace (fgs_read_counters); slower, they
 *                          exist to size the algorithmic work of a timed, uninstrumented run.
 *                          FGS_OPT_NO_WAIT: the decoupled look-back waits of fgs_bin_sort_ex
 *                          (record scan, tile scan, onesweep passes) give up before their first
 *                          poll, so every partition that has a predecessor reports
 *                          FGS_ERR_TIMEOUT; this exercises the timeout path of a real call.
 *   wait_limit             polls after which one look-back wait gives up with FGS_ERR_TIMEOUT;
 *                          0 = 2^20 (about a second of polling). The waits of the rasterizers'
 *                          bulk copies keep their own bound of 2^20 polls.
 *   main_kernel_events     a measurement hook: two cudaEvent_t (created by the caller) that
 *                          fgs_rasterize_ex and fgs_backward_ex / fgs_backward_raster_ex record
 *                          on `stream` immediately before and after the launch of the call's
 *                          main kernel (the rasterizer, the backward rasterizer), so that its
 *                          duration can be read apart from the call's small set-up kernels and
 *                          memsets; NULL = none. Other calls ignore them.
 * Unknown flag bits or a shape outside the lists: FGS_ERR_INVALID_ARG before any launch. */
#define FGS_OPT_INSTRUMENT 1u
#define FGS_OPT_NO_WAIT 2u
typedef struct {
  int32_t fwd_pixels_per_thread;
  int32_t bwd_pixels_per_thread;
  uint32_t flags;
  uint32_t wait_limit;
  void *main_kernel_events[2];
} fgs_options;

/* Bytes of workspace needed by fgs_bin_sort, fgs_rasterize and fgs_backward for this set of
 * views, n Gaussians and a key capacity (0 < capacity < 2^32). */
fgs_status fgs_workspace_size(int64_t n, const fgs_camera *cams, int n_views, int64_t capacity,
                              size_t *bytes);

/* Workspace for fgs_bin_sort_ex with the given flags (fgs_workspace_size = flags 0; only
 * FGS_BIN_ONESWEEP needs more). */
fgs_status fgs_workspace_size_ex(int64_t n, const fgs_camera *cams, int n_views, int64_t capacity,
                                 uint32_t flags, size_t *bytes);

/* Number of 16x16 tiles over all views (global tile ids are view-major, row-major inside a
 * view) and number of pixels over all views. Host-only helpers. */
int64_t fgs_total_tiles(const fgs_camera *cams, int n_views);
int64_t fgs_total_pixels(const fgs_camera *cams, int n_views);

/* Stage 1, per-Gaussian preprocess (Sec. 4.1 preprocessCUDA, modified by Sec. 4.2 / 4.3):
 * view transform, equidistant projection of the mean, fisheye Jacobian J, covariance
 * Sigma = R S S^T R^T, Sigma_p = (J W) Sigma (J W)^T + 0.3 I, conic, colour from SH along
 * (mu - camera centre), depth and tile rectangle.
 * Outputs: records [n_views * n] (fgs_record), tiles_touched [n_views * n] (rect area, 0 if
 * culled). */
fgs_status fgs_preprocess(const fgs_gaussians *g, const fgs_camera *cams, int n_views,
                          fgs_record *records, uint32_t *tiles_touched, fgs_stream stream);

/* Stages 2-4, tile binning + sort (Sec. 3.1 "Rendering", Sec. 4.1 duplicateWithKeys and
 * radixSort): for every record r with a non-empty rect and every tile t of the rect,
 * one pair (key = t << 32 | bits(depth_r), value = r), t the global tile id; the pairs are
 * sorted by key, equal keys in increasing r (a stable sort of the emission in record order).
 * Inputs: records, tiles_touched [n_views * n] (as written by fgs_preprocess, or any records
 * whose rect and depth fields are set and tiles_touched = rect area). With a smaller
 * tiles_touched a record's pairs are the first tiles_touched tiles of its rect in row-major
 * order; a larger one keeps the rect's tiles only (the surplus pairs are dropped, by both sorts,
 * and not counted in *n_intersections), and so does a rect outside its view's tile grid (no
 * pairs). Every write stays inside its buffer.
 * Outputs: keys [capacity] u64, vals [capacity] u32 (first *n_intersections entries valid),
 * tile_ranges [fgs_total_tiles * 2] u32 = [start, end) of each global tile,
 * n_intersections (device int64, the true count even when it exceeds capacity).
 * Resets the workspace status word; sets FGS_ERR_CAPACITY there if the count exceeds
 * capacity. */
fgs_status fgs_bin_sort(const fgs_record *records, const uint32_t *tiles_touched, int64_t n,
                        const fgs_camera *cams, int n_views, uint64_t *keys, uint32_t *vals,
                        int64_t capacity, uint32_t *tile_ranges, int64_t *n_intersections,
                        void *workspace, size_t workspace_bytes, fgs_stream stream);

/* fgs_bin_sort with options. flags = 0 is fgs_bin_sort. flags = FGS_BIN_ELLIPSE emits only the
 * pairs whose tile the Gaussian's alpha >= 1/255 ellipse d^T conic d <= 2 ln(255 opacity)
 * reaches: the minimum of the quadratic over the rectangle of the tile's pixel centres is
 * compared with the level (times 1 + 1e-3, plus 1e-2, a conservative margin). This is the
 * precise Gaussian-tile intersection of the renderers the method adapts to (Sec. 6 and
 * Table 3, FlashGS). A dropped pair has alpha < 1/255 at every pixel of its tile, so the images,
 * transmittances and gradients equal those of the rect binning; only the lists are shorter.
 * *n_intersections is then the number of pairs kept (the rect count if it exceeds capacity,
 * with FGS_ERR_CAPACITY); capacity must still hold the rect count. Unknown flag bits:
 * FGS_ERR_INVALID_ARG. */
#define FGS_BIN_ELLIPSE 1u
/* flags = FGS_BIN_ONESWEEP sorts the rect pairs with a device-wide onesweep LSD radix sort over
 * the key bits (the renderer's own sort design) instead of the default per-tile sort; same
 * output bit for bit. It needs the larger workspace of fgs_workspace_size_ex(..., flags, ...)
 * and cannot be combined with FGS_BIN_ELLIPSE. */
#define FGS_BIN_ONESWEEP 2u
fgs_status fgs_bin_sort_ex(const fgs_record *records, const uint32_t *tiles_touched, int64_t n,
                           const fgs_camera *cams, int n_views, uint64_t *keys, uint32_t *vals,
                           int64_t capacity, uint32_t *tile_ranges, int64_t *n_intersections,
                           void *workspace, size_t workspace_bytes, uint32_t flags,
                           const fgs_options *opt, fgs_stream stream);

/* Stage 5, rasterize (Sec. 3.1 "Rendering", Sec. 4.1 renderCUDA): per pixel, front to back
 * over its tile's sorted list: skip alpha < 1/255, stop before a Gaussian whose blend would
 * take T below 1e-4, C += rgb alpha T, T *= 1 - alpha; finally C += T bg.
 * bg: HOST float[3] (NULL = black).
 * Outputs: images (planar [3][H][W] per view, views packed in order), final_T [pixels],
 * n_processed [pixels] u32 = 1 + position in the tile list of the last blended Gaussian
 * (0 if none); the backward reads final_T and n_processed. */
fgs_status fgs_rasterize(const fgs_record *records, const uint32_t *vals,
                         const uint32_t *tile_ranges, const fgs_camera *cams, int n_views,
                         const float *bg, float *images, float *final_T,
                         uint32_t *n_processed, void *workspace, size_t workspace_bytes,
                         fgs_stream stream);
fgs_status fgs_rasterize_ex(const fgs_record *records, const uint32_t *vals,
                            const uint32_t *tile_ranges, const fgs_camera *cams, int n_views,
                            const float *bg, float *images, float *final_T,
                            uint32_t *n_processed, void *workspace, size_t workspace_bytes,
                            const fgs_options *opt, fgs_stream stream);

/* Stages 5-1 backward (Sec. 4.2 / 4.3 backward and the blend derivative): gradients of
 * L = <dL_dimages, images> with respect to the fgs_gaussians inputs, summed over views.
 * The blend state per pixel is recomputed from the records, final_T and n_processed;
 * J and dJ/dmu_c are recomputed from the inputs; the gradient of mu is the sum of its
 * mean-projection and covariance paths.
 * Outputs (overwritten): d_means [n,3], d_scales [n,3], d_quats [n,4], d_opacities [n],
 * d_sh [n,(d+1)^2,3]. bg: HOST float[3] or NULL (as given to fgs_rasterize). */
fgs_status fgs_backward(const fgs_gaussians *g, const fgs_camera *cams, int n_views,
                        const fgs_record *records, const uint32_t *tiles_touched,
                        const uint32_t *vals, const uint32_t *tile_ranges, const float *bg,
                        const float *final_T, const uint32_t *n_processed,
                        const float *dL_dimages, float *d_means, float *d_scales,
                        float *d_quats, float *d_opacities, float *d_sh, void *workspace,
                        size_t workspace_bytes, fgs_stream stream);
fgs_status fgs_backward_ex(const fgs_gaussians *g, const fgs_camera *cams, int n_views,
                           const fgs_record *records, const uint32_t *tiles_touched,
                           const uint32_t *vals, const uint32_t *tile_ranges, const float *bg,
                           const float *final_T, const uint32_t *n_processed,
                           const float *dL_dimages, float *d_means, float *d_scales,
                           float *d_quats, float *d_opacities, float *d_sh, void *workspace,
                           size_t workspace_bytes, const fgs_options *opt, fgs_stream stream);

/* Training (Sec. 5.1 "Optimization": the loss, optimiser and hyperparameters of the renderer
 * the method plugs into - Adam on the per-Gaussian parameters).
 *
 * fgs_loss_l1: L = scale * sum_i |images_i - targets_i| into *loss (DEVICE float, reset by the
 * call) and dL_dimages_i = scale * sign(images_i - targets_i) (0 where equal); n floats.
 *
 * fgs_adam_step: one Adam step (Kingma & Ba, Algorithm 1; bias-corrected moments) over up to
 * FGS_ADAM_MAX_GROUPS parameter tensors in one launch. Per group: raw parameters (updated in
 * place), the gradient of the ACTIVATED parameters (as fgs_backward writes it), the two moment
 * buffers (zero before step 1), and the activation act = raw (FGS_ACT_NONE), exp(raw)
 * (FGS_ACT_EXP, for scales) or 1 / (1 + exp(-raw)) (FGS_ACT_SIGMOID, for opacities); the
 * gradient is chained through it at the current raw value, and act(new raw) is written to `act`
 * (NULL or == raw: not written). step: DEVICE int64 holding the number of steps taken (0
 * before the first); the call advances it on the device and uses the new value t in the bias
 * correction, so the call can be captured in a CUDA graph and replayed. All other pointers of
 * a group are DEVICE, FP32, `count` elements each; the group array itself is HOST memory. */
#define FGS_ADAM_MAX_GROUPS 8
typedef enum { FGS_ACT_NONE = 0, FGS_ACT_EXP = 1, FGS_ACT_SIGMOID = 2 } fgs_activation;
typedef struct {
  float *raw;
  float *act;
  const float *grad;
  float *m, *v;
  int64_t count;
  int32_t activation; /* fgs_activation */
  float lr;
} fgs_adam_group;
fgs_status fgs_loss_l1(const float *images, const float *targets, float *dL_dimages, int64_t n,
                       float scale, float *loss, fgs_stream stream);
fgs_status fgs_adam_step(const fgs_adam_group *groups, int n_groups, double beta1,
                         double beta2, float eps, int64_t *step, fgs_stream stream);

/* fgs_bin_sort for callers that cannot allocate device memory (the paper has no counterpart:
 * this is a deployment variant). Plugins running inside a host application that owns the GPU
 * memory budget, and real-time loops that must never call cudaMalloc / cudaFree (which can
 * synchronise the device), have no workspace to pass; this entry point keeps the sort's scratch
 * in a fixed array inside the library instead, and the caller passes only inputs and outputs.
 * Results are the same as fgs_bin_sort's for the same inputs.
 *  - Limits: n_views * n <= 2^19 records, capacity <= 2^19 key slots and at most 2^17 tiles
 *    over all views; larger sizes return FGS_ERR_INVALID_ARG before anything is launched.
 *    Every GPU that loads the library holds the array (about 22 MB) until the process exits.
 *  - status: DEVICE pointer to one uint32 the call fills, in stream order, with the device
 *    status word (FGS_OK, FGS_ERR_CAPACITY or FGS_ERR_TIMEOUT) once the sort has run.
 *  - The first call on a device looks up the array's device address (cudaGetSymbolAddress);
 *    make that first call before any stream capture on that device. The address is kept with
 *    the id of the context it belongs to; a call that finds another context current (a
 *    non-primary one, or the new primary context after cudaDeviceReset) looks it up again.
 *  - All calls share the one array and leave their contents in it (each call clears what must
 *    start at zero): calls whose work overlaps on the GPU race; calls ordered on one stream
 *    are safe. */
fgs_status fgs_bin_sort_noalloc(const fgs_record *records, const uint32_t *tiles_touched,
                                int64_t n, const fgs_camera *cams, int n_views, uint64_t *keys,
                                uint32_t *vals, int64_t capacity, uint32_t *tile_ranges,
                                int64_t *n_intersections, uint32_t *status, fgs_stream stream);

/* The two halves of fgs_backward, for callers that time or reuse them separately:
 * fgs_backward_raster replays the blend and accumulates per-record screen-space gradient sums
 * (the moments of dL/d exponent over the pixel offsets, dL/d opacity and dL/d rgb terms) into
 * the workspace; fgs_backward_preprocess
 * pulls them back to the Gaussian inputs (overwriting the d_* outputs). Called in this order
 * on one workspace they equal fgs_backward. n = Gaussians per view. The _ex variants take
 * fgs_options; the others use the defaults. */
fgs_status fgs_backward_raster(const fgs_record *records, const uint32_t *vals,
                               const uint32_t *tile_ranges, int64_t n, const fgs_camera *cams,
                               int n_views, const float *bg, const float *final_T,
                               const uint32_t *n_processed, const float *dL_dimages,
                               void *workspace, size_t workspace_bytes, fgs_stream stream);
fgs_status fgs_backward_raster_ex(const fgs_record *records, const uint32_t *vals,
                                  const uint32_t *tile_ranges, int64_t n, const fgs_camera *cams,
                                  int n_views, const float *bg, const float *final_T,
                                  const uint32_t *n_processed, const float *dL_dimages,
                                  void *workspace, size_t workspace_bytes,
                                  const fgs_options *opt, fgs_stream stream);
fgs_status fgs_backward_preprocess(const fgs_gaussians *g, const fgs_camera *cams, int n_views,
                                   const fgs_record *records, const uint32_t *tiles_touched,
                                   float *d_means, float *d_scales, float *d_quats,
                                   float *d_opacities, float *d_sh, void *workspace,
                                   size_t workspace_bytes, fgs_stream stream);

/* Synchronises `stream` and returns the device status word of `workspace` in *status
 * (an fgs_status value). */
fgs_status fgs_read_status(const void *workspace, fgs_stream stream, int *status);

/* Measurement hook (not part of the rendering path): after calls made with FGS_OPT_INSTRUMENT,
 * the workspace holds counters[0] = forward (pixel, Gaussian) evaluations, [1] = forward
 * blends, [2] = backward evaluations, [3] = backward contributions, [4] = records the forward
 * rasterizer copied into shared memory (48 bytes each), [5] = the backward's. The counters are
 * reset by fgs_bin_sort. fgs_read_counters synchronises `stream` and copies the six counters to
 * host memory (counters: HOST uint64[6]). */
fgs_status fgs_read_counters(const void *workspace, fgs_stream stream, uint64_t *counters);

/* Static description of a status code. */
const char *fgs_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* FGS_H */
