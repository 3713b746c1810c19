/*
 * rc.h -- C ABI of the GB300 direct-volume-rendering raycaster.
 *
 * The calls follow the paper's statement of the problem (Adeshina et al.,
 * "Hardware-Accelerated Raycasting: Towards an Effective Brain MRI
 * Visualization"): a scalar volume on a Cartesian voxel grid (Sec. 2.1) whose
 * slices have a thickness and gaps (Sec. 1, anisotropic spacing), colour and
 * opacity transfer functions (Sec. 2.6, Sec. 6), camera settings (Sec. 6) and a
 * raycast function that computes the compositing integral for every pixel
 * (Sec. 4.1-4.2, Eq. 1-5; Sec. 6).
 *
 * Conventions shared by every call:
 *  - Status codes only; no exception or longjmp crosses this boundary.
 *    rc_last_error() gives the text of the last failure of a context.
 *  - Arguments are validated before anything is launched or changed; a call
 *    that fails leaves the earlier state of its objects as it was.
 *  - Library objects (context, volume) are opaque, owned by the library and
 *    released by their *_destroy call. Inputs are copied. Output buffers are
 *    caller-owned DEVICE memory unless stated otherwise.
 *  - Every device operation is asynchronous on the context's CUDA stream
 *    (set at creation or by rc_context_set_stream). A call that returns
 *    statistics to host memory synchronises that stream.
 *  - One context per host thread; contexts are independent.
 *  - Index space: voxel (i, j, k) has its centre at integer coordinates,
 *    world position (i*sx, j*sy, k*sz) mm; the volume box is [0, N-1] per axis.
 *    Voxel arrays are x fastest, then y, then z.
 *  - Images are row-major H x W x 4 floats, y = 0 at the top, premultiplied
 *    RGBA on a black background.
 */
#ifndef RC_H
#define RC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RC_OK = 0,
    RC_ERR_INVALID_ARG = 1,   /* null pointer, bad size, out-of-range value */
    RC_ERR_OOM = 2,           /* device or host allocation failed */
    RC_ERR_CUDA = 3,          /* a CUDA runtime call or a kernel failed */
    RC_ERR_STATE = 4,         /* call out of order (e.g. render before upload) */
    RC_ERR_TIMEOUT = 5,       /* a bounded device wait ran out */
    RC_ERR_UNSUPPORTED = 6,   /* valid but not supported combination */
    RC_ERR_FORMAT = 7         /* malformed serialized blob */
} rc_status;

/* How the volume is held on the device (Sec. 2.1 scalar data):
 * F32: FP32 codes (exact copies of the uint16 codes);
 * F16: FP16 of (code - o) / o, normalised to [-1, 1] by the offset o, the
 *      smallest power of two (>= 1) with 2o >= vmax (2048 for 12-bit data):
 *      |code - o| <= 2048 is an integer FP16 holds exactly, so every code of
 *      a volume with vmax <= 4096 is stored exactly in 2 bytes;
 * U16: the raw uint16 codes. */
typedef enum { RC_STORE_F32 = 0, RC_STORE_F16 = 1, RC_STORE_U16 = 2 } rc_storage;

/* Ray functions listed in Sec. 4.1 (and Sec. 2.4 ii). The default and the
 * subject of the paper is compositing (Sec. 4.2). Output channels of the
 * others: MIP / AVERAGE: (m, m, m, 1), m = max / mean sample value over full
 * scale; XRAY: (x, x, x, 1), x = sum of sample values times the step in mm over
 * full scale; ISO: (t*, headlight-shaded intensity at the first sample at or
 * above iso, index of that sample, 1), t* = the crossing distance in mm,
 * linearly interpolated between the two samples around it; THRESHOLD:
 * (transfer-function colour of the first sample at or above iso, 1). A ray
 * that misses the box, or finds no crossing, gives 0 in all four channels. */
typedef enum {
    RC_FUNC_COMPOSITE = 0, RC_FUNC_MIP = 1, RC_FUNC_AVERAGE = 2,
    RC_FUNC_XRAY = 3, RC_FUNC_ISO = 4, RC_FUNC_THRESHOLD = 5
} rc_ray_function;

/* Reconstruction filter of the resampling step (Sec. 4.1 step 2; Sec. 3.2
 * names trilinear filtering and, for higher quality, cubic filters).
 * TRILINEAR: 8 voxels per sample, gradient by central differences of the
 * trilinear field (one index unit per axis).
 * BSPLINE: uniform cubic B-spline on the voxel values (no interpolating
 * prefilter, so it smooths): f(p) = sum over the 4 x 4 x 4 voxels around p of
 * V * b(dx) b(dy) b(dz), b(x) = (4 - 6x^2 + 3|x|^3)/6 for |x| < 1,
 * (2 - |x|)^3/6 for 1 <= |x| < 2; indices outside the volume take the
 * nearest border voxel. Gradient: the analytic derivative of that sum. Every
 * ray function supports it; the table gradient and the learned proposal do
 * not (RC_ERR_UNSUPPORTED). */
typedef enum { RC_FILTER_TRILINEAR = 0, RC_FILTER_BSPLINE = 1 } rc_filter;

typedef struct rc_context rc_context;
typedef struct rc_volume rc_volume;

/* Perspective pinhole camera (Sec. 6, camera settings). The camera basis is
 * f = normalize(target - eye), r = normalize(f x up), u = r x f, computed in
 * FP64 and rounded to FP32. Pixel (x, y) looks along
 * normalize(f + ndc_x r + ndc_y u) with ndc_x = ((x + 0.5)/W * 2 - 1) tan(fovy/2) W/H
 * and ndc_y = (1 - (y + 0.5)/H * 2) tan(fovy/2), each operation an FP32
 * operation rounded once. */
typedef struct {
    float eye[3], target[3], up[3];   /* world, mm */
    float fovy_deg;                   /* vertical field of view, (0, 180) */
    int32_t width, height;            /* pixels, >= 1 */
} rc_camera;

typedef struct {
    float step_vox;     /* sample spacing ds in units of the finest spacing (>= 1e-3).
                           Opacity is per reference step ds_ref = min(spacing) and
                           is corrected to 1 - (1 - a)^(ds/ds_ref) (Eq. 3). */
    float term;         /* early ray termination once 1 - T >= term; (0, 1] */
    int32_t shade;      /* 1: central-difference gradients, headlight Blinn-Phong */
    float ka, kd, ks;   /* shading weights; specular exponent 16 */
    int32_t func;       /* rc_ray_function */
    float iso;          /* iso-value / threshold, in the volume's code units */
    int32_t skip;       /* 1: skip bricks the occupancy mask marks empty (exact) */
    int32_t filter;     /* rc_filter (0: trilinear) */
} rc_render_params;

typedef struct {
    uint64_t dense_samples;      /* samples up to termination, skipped ones included
                                    (0 for the importance-sampled renders) */
    uint64_t evaluated_samples;  /* samples resampled and classified */
    uint64_t rays_hit;           /* rays that intersect the volume box */
    uint64_t rays_total;
    uint64_t fallback_rays;      /* importance-sampled renders: rays re-marched */
    float device_ms;             /* device time of the call's work: CUDA events on the
                                    context's stream before its first launch and after
                                    its last one (copies of rc_render_views_host included) */
} rc_stats;

/* Text of a status code (static storage). */
const char *rc_status_string(rc_status s);

/* Text of the last failure on ctx (valid until the next call on ctx); for a
 * NULL ctx, the last failure of a call that had no context (thread-local). */
const char *rc_last_error(const rc_context *ctx);

/* Creates a context on CUDA device `device`, launching on `cuda_stream` (a
 * cudaStream_t; NULL = the legacy default stream). */
rc_status rc_context_create(int device, void *cuda_stream, rc_context **out);
rc_status rc_context_set_stream(rc_context *ctx, void *cuda_stream);
/* Synchronises the context's stream and reports device-side failures of the
 * calls queued since the last check: RC_ERR_TIMEOUT when a kernel's bounded
 * wait (the tensor-core network's MMA or weight-copy completion) gave up,
 * in which case that launch's outputs are invalid. Calls that return
 * statistics make the same check. */
rc_status rc_context_sync(rc_context *ctx);

/* Synchronises the context's stream and frees everything the context owns.
 * Volumes must be destroyed first (RC_ERR_STATE otherwise). */
rc_status rc_context_destroy(rc_context *ctx);

/* Volume of nx x ny x nz voxels (each >= 2) with spacing sx, sy, sz mm (> 0) and
 * valid codes 0..vmax (>= 1; larger codes clamp to vmax) (Sec. 2.1, Sec. 1).
 * The device holds it in cell-bricks (the trilinear cells whose base index
 * lies in 16b..16b+15 per axis), each stored with an apron as the 19^3 voxels
 * 16b-1..16b+17 (clamped to the volume) in the chosen storage, with a min/max
 * grid over the cell-bricks (footprint voxels 16b..min(16b+16, N-1)). FP32
 * storage, uint16 storage with vmax < 32768 and FP16 storage with
 * vmax <= 4096 also hold value+gradient bricks (each voxel's stored value and
 * the central differences of its codes: 16 bytes per voxel for FP32, 8 for
 * the others) that shaded and 2-D-table samples read. */
rc_status rc_volume_create(rc_context *ctx, int nx, int ny, int nz,
                           float sx, float sy, float sz, uint16_t vmax,
                           rc_storage storage, rc_volume **out);
/* Copies n_voxels (== nx*ny*nz) uint16 codes, x fastest, from host memory
 * (src_is_device = 0; pinned memory makes the copy asynchronous) or device
 * memory (1), re-lays them out in bricks and rebuilds the min/max grid. */
rc_status rc_volume_upload(rc_volume *vol, const uint16_t *src, size_t n_voxels,
                           int src_is_device);
rc_status rc_volume_destroy(rc_volume *vol);

/* Number of cell-bricks per axis, ceil((N-1)/16). */
rc_status rc_volume_brick_dims(const rc_volume *vol, int dims[3]);

/* Transfer function (Sec. 2.6, Sec. 6): n_entries (2..4096) straight RGBA
 * entries in [0, 1], host memory, entry i at code i*vmax/(n_entries-1); a value
 * between entries is the linear interpolation of its two neighbours (table
 * coordinate u = fl(v * fl((n_entries-1) / vmax)), see rc_skip_mask_get). fp16 = 1
 * stores the table as FP16 (the precision form). The table is copied into a
 * page-locked buffer of the context during the call (rgba may be reused at
 * once) and reaches the device in stream order, without waiting for the work
 * queued before it; the copy before it must have run (in a frame loop it ran
 * before the previous frame's render). */
rc_status rc_tf_set(rc_context *ctx, const float *rgba, int n_entries, int fp16);
/* Same from device memory (asynchronous device-to-device copy). Values are not
 * range-checked on this path. */
rc_status rc_tf_set_device(rc_context *ctx, const float *rgba_dev, int n_entries, int fp16);

/* Two-dimensional transfer function over (value, gradient magnitude), the
 * classification by scalar value and gradient magnitude that Sec. 3.1 cites
 * for boundary emphasis. rgba: host memory, n_grad rows of n_values straight
 * RGBA entries in [0, 1] (value index fastest: entry (i, j) at
 * rgba[4 * (j * n_values + i)]); value entry i sits at code i*vmax/(n_values-1)
 * as in rc_tf_set, row j at gradient magnitude j*gmax/(n_grad-1) codes per mm.
 * A sample's gradient (central differences, or the B-spline derivative) gives
 * the row coordinate w = fl(|g| * fl((n_grad-1) * vmax / (vscale * gmax))),
 * clamped to [0, n_grad-1] (vscale: the full scale in stored units, vmax,
 * or vmax / o for F16 storage, whose gradient is in units of o codes); the
 * four entries around (u, w) blend
 * bilinearly. n_values 2..4096, n_grad 2..4096, n_values * n_grad <= 2^20,
 * gmax finite and > 0. fp16 = 1 rounds the entries to FP16. Replaces the
 * current table (1-D or 2-D). Copied as rc_tf_set copies (rgba may be reused
 * at once; no wait for the queued work). Compositing, the table gradient and the ray
 * functions that do not classify use it; thresholding and the learned
 * proposal need a 1-D table (RC_ERR_UNSUPPORTED). Shading off still computes
 * the gradient. Empty-space skipping stays exact: a brick is empty only when
 * every row of its value entries has zero opacity. */
rc_status rc_tf2d_set(rc_context *ctx, const float *rgba, int n_values, int n_grad, float gmax, int fp16);
/* Same from device memory (asynchronous device-to-device copy; the opacity
 * maxima and the FP16 rounding are computed on the context's stream). Values
 * are not range-checked on this path. */
rc_status rc_tf2d_set_device(rc_context *ctx, const float *rgba_dev, int n_values, int n_grad, float gmax,
                             int fp16);

rc_status rc_camera_set(rc_context *ctx, const rc_camera *cam);

/* Renders the current camera view of vol with the current transfer function
 * (Sec. 4.1-4.2): per pixel one ray, evenly spaced samples reconstructed by
 * params->filter,
 * classification, optional shading, front-to-back compositing with early
 * termination. out_rgba: device, width*height*4 floats, caller-owned,
 * overwritten. stats: optional host pointer; when given the call synchronises
 * the stream and fills it. */
rc_status rc_render(rc_context *ctx, const rc_volume *vol, const rc_render_params *params,
                    float *out_rgba, rc_stats *stats);

/* Renders nviews cameras (1..65535, all with the same image size) of vol in one
 * launch: the same images as nviews rc_render calls, written view-major into
 * out_rgba (device, nviews*H*W*4 floats, caller-owned). A whole orbit becomes
 * one grid, so the GPU does not drain between frames (Sec. 1's interactive
 * speed). stats (optional, synchronises) sums over the views. The context's
 * own camera is not changed. */
rc_status rc_render_views(rc_context *ctx, const rc_volume *vol, const rc_render_params *params,
                          const rc_camera *cams, int nviews, float *out_rgba, rc_stats *stats);

/* rc_render_views with the images delivered to host memory: host_rgba
 * (nviews*H*W*4 floats, view-major, caller-owned). The views are rendered in
 * groups of `group` views (0: groups of at least 2 M pixels), alternately on
 * the context's stream and a second stream of the library, each into its own
 * device buffer, and each group's images are copied to host_rgba on a third
 * stream while the next groups render. With
 * page-locked host_rgba (cudaHostAlloc / cudaHostRegister) the copies overlap
 * the rendering; pageable memory gives the same images without the overlap.
 * Each image equals rc_render_views'. host_rgba in device or managed memory
 * is refused (RC_ERR_INVALID_ARG). Synchronises: the images are in host_rgba
 * when the call returns RC_OK (on an error its contents are undefined). stats (optional) sums over the views. The context's own camera
 * is not changed. */
rc_status rc_render_views_host(rc_context *ctx, const rc_volume *vol, const rc_render_params *params,
                               const rc_camera *cams, int nviews, int group, float *host_rgba, rc_stats *stats);

/* Renders nviews cameras of each of nvols volumes in one launch (the
 * compositing function): the volumes must share shape, spacing, vmax and
 * storage (RC_ERR_INVALID_ARG otherwise), and the context's table and the
 * cameras apply to all; nvols * nviews <= 65535. out_rgba: device
 * nvols*nviews*H*W*4 floats, volume-major then view-major; each image equals
 * rc_render_views of its volume. stats (optional, synchronises) sums over
 * everything. */
rc_status rc_render_batch(rc_context *ctx, const rc_volume *const *vols, int nvols, const rc_render_params *params,
                          const rc_camera *cams, int nviews, float *out_rgba, rc_stats *stats);

/* Gradient of a loss with respect to the transfer function entries, given the
 * gradient of the loss with respect to the composited image (Eq. 4-5 are
 * differentiable in the table). dL_dimage: device, width*height*4 floats;
 * dL_dtf: device, 4 floats per table entry (K*4 for a 1-D table, M*K*4 for
 * a 2-D table, row-major like the table), overwritten. Compositing function
 * only; trilinear or cubic B-spline reconstruction. A 2-D table's gradient
 * flows into the four entries of each sample's bilinear cell (value and
 * gradient-magnitude weights); the gradient-magnitude coordinate itself is
 * not differentiated (it does not depend on the table). The gradient pass
 * does not skip empty space (an
 * empty brick still has a gradient). The forward march is recomputed per ray;
 * nothing is stored per sample. The result does not depend on thread
 * scheduling: each warp sums in its own program order, and the sums across
 * warps and blocks are 64-bit fixed point (scale 2^32 / max|dL/dI|). */
rc_status rc_render_backward(rc_context *ctx, const rc_volume *vol,
                             const rc_render_params *params, const float *dL_dimage,
                             float *dL_dtf);

/* The gradient summed over nviews cameras (1..65535, one image size) in one
 * launch, for a loss over several views of the same volume and table (the
 * fitting of a table to an orbit): dL_dimages device nviews*H*W*4 floats,
 * view-major; dL_dtf as above, overwritten with the sum. Same per-view
 * arithmetic as rc_render_backward; the fixed-point scale is set by the
 * largest |dL/dI| over all views. The context's own camera is not changed. */
rc_status rc_render_backward_views(rc_context *ctx, const rc_volume *vol, const rc_render_params *params,
                                   const rc_camera *cams, int nviews, const float *dL_dimages, float *dL_dtf);

/* rc_render_backward_views for a caller that still holds the forward images:
 * images (device, nviews*H*W*4 floats, view-major) are the images
 * rc_render_views wrote for the same volume, table, parameters and cameras.
 * Each ray's final colour C and transmittance T = 1 - alpha are read from them
 * instead of being recomputed by a first forward march, and the gradient
 * march stops at the forward's termination sample by itself (it rebuilds the
 * transmittance sample by sample): one march per ray instead of two. The
 * result equals rc_render_backward_views' up to the rounding of T = 1 - alpha
 * (and the few ulps by which compiled instances may differ); images of other
 * inputs give a wrong gradient, not an error. */
rc_status rc_render_backward_views_with_forward(rc_context *ctx, const rc_volume *vol,
                                                const rc_render_params *params, const rc_camera *cams,
                                                int nviews, const float *images, const float *dL_dimages,
                                                float *dL_dtf);

/* The gradient of rc_render_backward for callers that cannot allocate device
 * memory once they are running: for example a host application whose device
 * memory is all handed out up front by its own allocator, or a frame loop in
 * which a cudaMalloc (which can synchronise the whole device) is not allowed.
 * The paper has no counterpart; this is a service of the library.
 * Same arguments and result as rc_render_backward. It allocates nothing: the
 * fixed-point accumulators live in one file-scope device array sized for
 * tables of at most 1024 entries, K or M*K (32 KB + 256 B, held on every GPU that loads
 * the library until the process exits); a larger table returns
 * RC_ERR_UNSUPPORTED. The first call on a device looks up that array's device
 * address (and may load the library's device code), so make the first call
 * before any stream capture. Every call shares the one array and clears it on
 * the stream before use; calls whose work overlaps on the GPU (other streams or
 * contexts on the same device) race on it and must be serialised by the caller.
 * It reads the same stored values as rc_render_backward: a volume whose pair
 * bricks an earlier render allocated has them refreshed in place, and a volume
 * that never had them is read from its apron bricks (the same voxels in the
 * same arithmetic, so the same gradient). */
rc_status rc_render_backward_noalloc(rc_context *ctx, const rc_volume *vol,
                                     const rc_render_params *params, const float *dL_dimage,
                                     float *dL_dtf);

/* Copies the cell-brick min/max grid (uint16, brick_dims order x fastest) into
 * caller device buffers mn, mx. */
rc_status rc_brick_grid_get(rc_context *ctx, const rc_volume *vol, uint16_t *mn, uint16_t *mx);

/* The grid of a reconstruction filter: over the voxels its samples read,
 * 16b .. min(16b+16, N-1) per axis for RC_FILTER_TRILINEAR (the grid of
 * rc_brick_grid_get), max(16b-1, 0) .. min(16b+17, N-1) for RC_FILTER_BSPLINE. */
rc_status rc_brick_grid_get_filter(rc_context *ctx, const rc_volume *vol, int filter, uint16_t *mn,
                                   uint16_t *mx);

/* Writes the occupancy mask of vol under the current transfer function into
 * caller device memory (one byte per cell-brick, 1 = may hold non-zero
 * opacity). A brick is empty when every table entry a sample inside it can
 * touch, floor(u(min)) .. min(floor(u(max)) + 1, K - 1), has opacity 0, with
 * the table coordinate u(v) = fl(v * fl((K-1) / vmax)) of a raw code v, or
 * u(v) = fl((h + 1) * fl((K-1) / fl(vmax / o))) with h = fp16(fl((v - o) / o))
 * for F16 storage (FP32 operations rounded once). */
rc_status rc_skip_mask_get(rc_context *ctx, const rc_volume *vol, uint8_t *occ);

/* The mask of a reconstruction filter, from that filter's grid
 * (rc_brick_grid_get_filter). With a 2-D table an entry counts as transparent
 * only when it is transparent in every gradient row. The B-spline value is a
 * convex combination of its footprint, so skipping stays exact up to the FP32
 * rounding of the 64-term sum (a sample could leave its brick's value range
 * by a few units in the last place; with 256-entry tables over 12-bit codes
 * no coordinate lies that close below an entry boundary). */
rc_status rc_skip_mask_get_filter(rc_context *ctx, const rc_volume *vol, int filter, uint8_t *occ);

/* ---- learned sampling proposal -------------------------------------------
 * The paper marches evenly spaced samples (Sec. 4.1). This extension lets a
 * small network predict, per ray, a 32-bin opacity PDF over the ray's chord
 * [t_near, t_far] and the ray's final transmittance T^. The PDF marks where
 * the ray's contribution ends: b_end is one bin past the first bin >= b_start
 * where the running sum of the PDF reaches 1 - 1/64 (a margin for early
 * predictions; at most 31, and 31 if never); b_start is the first
 * bin whose start, centre or end lies in an occupied cell-brick (the whole
 * chord when none does). nimp samples at the centres of nimp equal segments of
 * [t_a, t_b] (start of bin b_start to end of bin b_end) replace the evenly
 * spaced march of Sec. 4.1 and are composited as in Sec. 4.2, each opacity
 * corrected to its segment (Eq. 3). Rays whose composited transmittance differs
 * from T^ by more than eps are re-marched by the plain march. The paper has no
 * learned part.
 *
 * Features of a ray (112 floats): e = fma(t_near, d, o) / (N - 1) per axis (the
 * entry point in [0, 1]^3) and the world direction, x = (e, dir); for each x_c
 * and j = 0..5: sin(2^j pi x_c), cos(2^j pi x_c) (72 values, c outer, j inner);
 * for b = 0..31 the occupancy (0/1) of the cell-brick holding the point at
 * t = fma(b + 0.5, (t_far - t_near)/32, t_near); then 2 zeros. A ray that misses
 * the box has all-zero features.
 *
 * Network: h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), h3 = relu(h2 W3 + b3),
 * z = h3 W4 + b4 with W1 112x64, W2 and W3 64x64, W4 64x40; weights and layer
 * inputs rounded to BF16, FP32 accumulation, FP32 biases; PDF = softmax(z[0:32]),
 * T^ = sigmoid(z[32]); z[33:40] is padding. Parameters (FP32, RC_PROPOSAL_PARAMS
 * floats) in the order W1 (input-major: W1[k*64 + n]), b1, W2, b2, W3, b3, W4
 * (W4[k*40 + n]), b4. */
#define RC_PROPOSAL_BINS 32
#define RC_PROPOSAL_FEATURES 112
#define RC_PROPOSAL_OUTPUTS 33
#define RC_PROPOSAL_PARAMS 18152

/* Loads the network from a little-endian blob: "RCPROP01", uint32 version (1),
 * n_features (112), n_hidden (64), n_hidden_layers (3), n_out (40),
 * n_out_used (33), n_params (18152), has_adam (0/1), uint64 adam_step, then
 * n_params FP32 parameters and, with has_adam, the Adam first and second
 * moments (n_params FP32 each). Malformed blobs return RC_ERR_FORMAT and leave
 * the previous network in place. */
rc_status rc_proposal_load(rc_context *ctx, const void *blob, size_t bytes);
/* Writes the blob (with Adam state) into host memory. With blob == NULL only
 * *bytes_out is set. Synchronises the stream. */
rc_status rc_proposal_save(rc_context *ctx, void *blob, size_t capacity, size_t *bytes_out);

/* Training targets for the current camera: per pixel 33 floats (device,
 * H*W*33): the weights T_k a'_k of 512 samples at the centres of 512 equal
 * segments of the chord (no early termination) summed 16 per bin, then the
 * final transmittance (1 and zero weights for rays that miss). */
rc_status rc_profiles_generate(rc_context *ctx, const rc_volume *vol,
                               const rc_render_params *params, float *out);
/* Features of every pixel's ray for the current camera (device, H*W*112). */
rc_status rc_proposal_features(rc_context *ctx, const rc_volume *vol,
                               const rc_render_params *params, float *out);
/* Network on n feature rows (device n*112) -> n rows of (PDF[32], T^) (device).
 * Runs on the tcgen05 tensor cores: BF16 features and weights, FP32
 * accumulators in tensor memory, one 128-ray tile per MMA, bias + ReLU +
 * BF16 rounding of every hidden layer, softmax / sigmoid in FP32. */
rc_status rc_proposal_forward(rc_context *ctx, const float *features, int64_t n, float *out);
/* Gradient of the mean loss over n rays with respect to the FP32 parameters
 * (device RC_PROPOSAL_PARAMS floats) and the loss (device float, may be NULL).
 * targets: n rows of 33 (profile bins, final transmittance). Loss per ray:
 * w KL(q || p) + (T^ - T)^2 with q = bins / sum(bins), w = sum(bins); BF16
 * rounding treated as identity in the backward. Runs on the tcgen05 tensor
 * cores: the forward as in rc_proposal_forward, then per 128-ray tile the
 * weight gradients (H^T dZ, accumulated in tensor memory over the tiles of a
 * CTA) and the data gradients (dZ W^T) as BF16 MMAs with FP32 accumulation;
 * dZ is rounded to BF16 as an MMA operand. Per-CTA partial sums are reduced
 * in a fixed order: deterministic for a given n. */
rc_status rc_proposal_grad(rc_context *ctx, const float *features, const float *targets, int64_t n,
                           float *grad, float *loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) on that
 * gradient; loss as above (device, may be NULL). */
rc_status rc_proposal_train_step(rc_context *ctx, const float *features, const float *targets, int64_t n,
                                 float lr, float *loss);
/* Placement of the importance samples along a ray's chord (the learned
 * proposal's two readings of "few samples where the opacity is"):
 * RANGE: nimp samples at the centres of nimp equal segments of the range the
 * PDF marks (described above); the default of rc_render_proposal and
 * rc_render_importance.
 * INVCDF: stratified inverse-CDF sampling of the mixture
 * q_b = (1 - lambda) pdf_b + lambda / 32 (piecewise constant over the 32 bins
 * of the chord): sample j where the mixture's CDF reaches (j + 0.5) / nimp of
 * its total; each sample stands for the stretch between the midpoints to its
 * neighbours (t_near and t_far at the ends), so the segments tile the chord,
 * with its opacity corrected to that length (Eq. 3). lambda = 1 is the
 * uniform march of nimp samples over the whole chord. FP32 specification:
 * q_b = fma(1 - lambda, pdf_b, lambda / 32); Q_0 = 0, Q_{b+1} = Q_b + q_b;
 * y_j = ((j + 0.5) / nimp) * Q_32; b = the first bin with Q_{b+1} > y_j (31 if
 * none); f = q_b > 0 ? clamp((y_j - Q_b) / q_b, 0, 1) : 0;
 * t_j = fma(b + f, (t_far - t_near) / 32, t_near); midpoints
 * (t_{j-1} + t_j) * 0.5. */
typedef enum { RC_SAMPLING_RANGE = 0, RC_SAMPLING_INVCDF = 1 } rc_sampling;

/* Importance-sampled render from given per-pixel PDFs (device H*W*32) and
 * transmittances T^ (device H*W): nimp (1..4096) samples per ray over the range
 * described above; rays with |T - T^| > eps fall back to the plain march
 * (eps > 1: never). fallback: per-pixel flags (device) or NULL. stats counts
 * fallback rays in fallback_rays. */
rc_status rc_render_importance(rc_context *ctx, const rc_volume *vol, const rc_render_params *params,
                               const float *pdf, const float *that, int nimp, float eps,
                               float *out_rgba, uint8_t *fallback, rc_stats *stats);
/* The importance-sampled render of nviews cameras (1..65535, one image size)
 * in one launch with a choice of placement (rc_sampling; lambda in [0, 1] for
 * INVCDF, ignored for RANGE). pdf: device nviews*H*W*32 floats, view-major (may
 * be NULL for INVCDF with lambda = 1); that: device nviews*H*W floats, or NULL
 * for no fallback (eps is then ignored; RANGE needs it). out_rgba device
 * nviews*H*W*4, fallback (optional) nviews*H*W bytes. With RANGE each image
 * equals rc_render_importance's for that view. The context's own camera is
 * not changed. */
rc_status rc_render_importance_views(rc_context *ctx, const rc_volume *vol, const rc_render_params *params,
                                     const rc_camera *cams, int nviews, int sampling, float lambda,
                                     const float *pdf, const float *that, int nimp, float eps,
                                     float *out_rgba, uint8_t *fallback, rc_stats *stats);
/* The same with the loaded network choosing the samples: a tensor-core kernel
 * encodes each ray's features, runs the network (as rc_proposal_forward) and
 * keeps per ray only its sample range (from the PDF and the occupancy, as in
 * rc_render_importance) and T^; the importance march then renders from those
 * 8-byte records, with the same fallback. The result equals
 * rc_render_importance fed with rc_proposal_forward's outputs for the rays'
 * rc_proposal_features. */
rc_status rc_render_proposal(rc_context *ctx, const rc_volume *vol, const rc_render_params *params,
                             int nimp, float eps, float *out_rgba, uint8_t *fallback, rc_stats *stats);
/* rc_render_proposal for nviews cameras (1..65535, one image size) in two
 * launches: the network kernel over every view's rays, then one importance
 * march over all views. out_rgba: device nviews*H*W*4 floats, view-major;
 * fallback (optional): device nviews*H*W bytes. stats sum over the views. The
 * context's own camera is not changed. */
rc_status rc_render_proposal_views(rc_context *ctx, const rc_volume *vol, const rc_render_params *params,
                                   const rc_camera *cams, int nviews, int nimp, float eps, float *out_rgba,
                                   uint8_t *fallback, rc_stats *stats);
/* rc_render_proposal_views with a choice of placement: RC_SAMPLING_RANGE is
 * rc_render_proposal_views; with RC_SAMPLING_INVCDF (lambda in [0, 1]) the
 * network kernel writes every ray's PDF and T^ (132 bytes per ray, in a
 * buffer the context owns and grows) and the inverse-CDF march renders every
 * view from them: the result equals rc_render_importance_views fed with the
 * network's outputs. */
rc_status rc_render_proposal_sampled(rc_context *ctx, const rc_volume *vol, const rc_render_params *params,
                                     const rc_camera *cams, int nviews, int sampling, float lambda, int nimp,
                                     float eps, float *out_rgba, uint8_t *fallback, rc_stats *stats);

#ifdef __cplusplus
}
#endif

#endif /* RC_H */
