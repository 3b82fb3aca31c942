/*
 * fs4d.h -- C ABI of the GB300 (sm_103a) render path of 4D Gaussian Splatting
 * (Wu et al., "4D Gaussian Splatting for Real-Time Dynamic Scene Rendering",
 * arXiv 2310.08528).
 *
 * The path renders, for a view matrix M = [R, T] and a timestamp t, the image
 * I = S(M, G') with G' = G + F(G, t)  (Sec. 4.1):
 *   F : HexPlane deformation field -- six planes xy xz yz xt yt zt per level,
 *       bilinear interpolation, Hadamard product over planes, concatenation over
 *       levels (Sec. 4.2, Eq. 5), tiny MLP phi_d and heads phi_x, phi_r, phi_s
 *       (Sec. 4.2), update X' = X + dX, r' = r + dr, s' = s + ds (Eq. 6).
 *   S : differentiable splatting -- EWA projection Sigma' = J W Sigma W^T J^T
 *       (Eq. 2, Eq. 3), tile binning with (tile, depth) keys, radix sort, per-tile
 *       front-to-back alpha compositing (Eq. 1, Eq. 4).
 *
 * Conventions shared by every call:
 *  - Every call returns an fs4d_status; no C++ exception crosses the ABI.  On an
 *    error, fs4d_last_error(ctx) returns a message (valid until the next call on
 *    that context from the same thread).
 *  - Pointers named d_* are DEVICE pointers on the context's device, owned by the
 *    caller, and must stay valid until the work is complete.  Pointers named h_*
 *    (and the desc/camera structs) are HOST pointers, read during the call only.
 *  - Work is queued asynchronously on the context's stream; outputs are valid
 *    once that stream has been synchronised, unless a call says otherwise.
 *  - Float arrays are float32, C-contiguous, in the layouts stated per field.
 *  - Readings of the paper that the paper leaves open (corner-aligned bilinear
 *    interpolation with border clamping; biases in every linear layer; sigmoid
 *    opacity; log-space scales; 0.3 low-pass dilation; alpha clamped to 0.99,
 *    terms below 1/255 skipped, stop before the term that takes transmittance
 *    below 1e-4; pixel centres at +0.5; SH colour + 0.5 clamped at 0) are the
 *    library's conventions; the CPU oracle in this repository states each one.
 */
#ifndef FS4D_H
#define FS4D_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FS4D_API __attribute__((visibility("default")))
#else
#define FS4D_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum fs4d_status {
  FS4D_OK = 0,
  FS4D_ERR_INVALID_ARG = 1,   /* a pointer, size or enum outside what the call accepts */
  FS4D_ERR_OOM = 2,           /* device memory could not be allocated */
  FS4D_ERR_CAPACITY = 3,      /* a fixed-capacity buffer (tile pairs) overflowed */
  FS4D_ERR_CUDA = 4,          /* a CUDA runtime call failed (message has the CUDA error) */
  FS4D_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up (status word set) */
  FS4D_ERR_NOT_FOUND = 6,     /* unknown scene id or frame */
  FS4D_ERR_UNIMPLEMENTED = 7, /* a shape this build does not support (message says which) */
  FS4D_ERR_CANCELLED = 8,     /* a queued serving request was cancelled or its server stopped */
  FS4D_ERR_CORRUPT = 9        /* a canary word after a device buffer was overwritten (debug build) */
} fs4d_status;

typedef enum fs4d_precision {
  FS4D_FP32 = 0, /* planes and MLP in float32, SIMT FMA */
  FS4D_BF16 = 1  /* planes and MLP operands in bfloat16 on tcgen05 tensor cores, float32 accumulate */
} fs4d_precision;

/* How a frame groups its (tile, Gaussian) pairs by tile in (depth, index) order
 * (Sec. 3.1: the per-tile depth order of the tile-based rasteriser).  Both give the
 * same pair lists, bit for bit. */
typedef enum fs4d_binning {
  FS4D_BINNING_AUTO = 0,   /* the tile bitmap when it fits (at most 256 MB: tiles x Gaussians / 8
                              bytes) and the frame keeps no state for a backward, else the sort */
  FS4D_BINNING_SORT = 1,   /* emit one (tile | depth) key per pair and radix-sort on the tile bits */
  FS4D_BINNING_BITMAP = 2  /* (only reported by fs4d_last_binning) one bit per (tile, depth rank),
                              each tile's row read in rank order */
} fs4d_binning;

typedef struct fs4d_ctx fs4d_ctx;     /* one device + one stream; not thread-safe */
typedef struct fs4d_frame fs4d_frame; /* saved forward state of one render, for the backward */
typedef int32_t fs4d_scene_id;

/* Canonical scene (Sec. 3.1: X, s, r, opacity, SH; Sec. 4.2: HexPlane and MLP).
 * All pointers are HOST pointers; fs4d_load_scene copies them to the device. */
typedef struct fs4d_scene_desc {
  int32_t n;                   /* number of Gaussians, >= 1 */
  int32_t sh_degree;           /* 0..3; K = (sh_degree+1)^2 coefficients per channel */
  const float* means;          /* [n][3] canonical centres X */
  const float* log_scales;     /* [n][3] s; scale = exp(s) */
  const float* quats;          /* [n][4] r as (w, x, y, z); normalised only inside projection */
  const float* opacity_logits; /* [n]; opacity = sigmoid(logit) */
  const float* sh;             /* [n][K][3] real-SH coefficients (degree-major, m = -l..l) */
  float aabb_min[3];           /* box mapped onto the HexPlane grid [-1,1]^3 */
  float aabb_max[3];
  int32_t n_levels;            /* multi-resolution levels: the layout holds up to 4; the
                                  kernels of this build run 1..3 (4 returns
                                  FS4D_ERR_UNIMPLEMENTED from fs4d_load_scene) */
  int32_t res_spatial[4];      /* spatial grid resolution per level (>= 2) */
  int32_t res_time;            /* temporal grid resolution (>= 2), the same at every level */
  int32_t feat_dim;            /* h, features per plane: 16 or 32 */
  const float* planes;         /* per level, per plane (xy,xz,yz,xt,yt,zt): [R_b][R_a][h],
                                  R_a/R_b the resolutions of the plane's first/second axis */
  int32_t mlp_width;           /* hidden width W; this build supports 64 */
  const float* mlp;            /* layers d1 (W x h*L), d2 (W x W), x1, x2 (3 x W), r1, r2 (4 x W),
                                  s1, s2 (3 x W), and with color_heads c1 (W x W), c2 (3K x W),
                                  a1 (W x W), a2 (1 x W); each weight [out][in] then bias [out] */
  int32_t color_heads;         /* 0, or 1: the colour and opacity heads of App. B, applied in
                                  every frame: C' = C + phi_C(f_d) over the [K][3] SH
                                  coefficients, logit' = logit + phi_alpha(f_d) (f_d the output of
                                  phi_d); in FP32 frames by float32 SIMT arithmetic, in BF16 frames
                                  as two BF16 tensor-core GEMMs per 128 Gaussians (FP32
                                  accumulation).  Such scenes render (fs4d_render*, composition) but
                                  have no backward, trainer or serving (FS4D_ERR_UNIMPLEMENTED), and
                                  fs4d_deform returns only X', r', s'. */
} fs4d_scene_desc;

/* Pinhole camera.  world_to_cam maps world to camera coordinates (x right,
 * y down, z forward); pixel (i, j) is evaluated at (i + 0.5, j + 0.5). */
typedef struct fs4d_camera {
  int32_t width, height;       /* pixels, 1..8192 */
  float fx, fy, cx, cy;        /* focal lengths and principal point, pixels */
  float znear;                 /* Gaussians with camera z <= znear are culled */
  float world_to_cam[16];      /* row-major 4x4 */
} fs4d_camera;

/* Per-Gaussian output of the projection stage (device, caller-owned). */
typedef struct fs4d_projected {
  float* xy;            /* [n][2] projected mean, pixels */
  float* conic_opacity; /* [n][4] inverse dilated 2-D covariance (a, b, c) and opacity */
  float* rgb;           /* [n][3] view-dependent colour */
  float* depth;         /* [n] camera-space z (its float32 bits form the low key word) */
  int32_t* radius;      /* [n] 3-sigma radius in pixels; 0 = culled */
  int32_t* rect;        /* [n][4] touched tiles x0, y0, x1, y1 (x1, y1 exclusive) */
} fs4d_projected;

/* Gradients of a scalar loss with respect to the scene (device, caller-owned,
 * the layouts of fs4d_scene_desc).  Any pointer may be NULL to skip it. */
typedef struct fs4d_grads {
  float* means;          /* [n][3] */
  float* log_scales;     /* [n][3] */
  float* quats;          /* [n][4] */
  float* opacity_logits; /* [n] */
  float* sh;             /* [n][K][3] */
  float* planes;         /* flat, like desc.planes */
  float* mlp;            /* flat, like desc.mlp */
} fs4d_grads;

/* ---------------------------------------------------------------- context */

/* Create a context on `device` that queues work on `cuda_stream` (a cudaStream_t;
 * NULL = the legacy default stream).  *out receives the handle. */
FS4D_API fs4d_status fs4d_create(int32_t device, void* cuda_stream, fs4d_ctx** out);
/* Free every scene, frame and work buffer of the context, after synchronising its stream. */
FS4D_API fs4d_status fs4d_destroy(fs4d_ctx* ctx);
/* Message of the last error on this context (never NULL). */
FS4D_API const char* fs4d_last_error(const fs4d_ctx* ctx);
/* Replace the stream the context queues work on. */
FS4D_API fs4d_status fs4d_set_stream(fs4d_ctx* ctx, void* cuda_stream);
/* Read and clear the device status word (bounded waits that timed out, pair
 * capacity overflow in capacity mode).  Synchronises the context's stream.
 * Returns FS4D_OK, FS4D_ERR_TIMEOUT or FS4D_ERR_CAPACITY.  A frame in which a
 * wait timed out has an unreliable image; the context stays usable and the next
 * frame is computed afresh. */
FS4D_API fs4d_status fs4d_check_device_status(fs4d_ctx* ctx);
/* Debug build (compiled with FS4D_CHECK_BOUNDS: libfs4d_debug.so): every device
 * buffer the library allocates carries 256 canary bytes (0xA5) after its end.
 * fs4d_check_canaries synchronises the device and checks them all (every context
 * of the process): FS4D_OK, or FS4D_ERR_CORRUPT naming the first buffer whose
 * canary was overwritten -- a kernel wrote past the end of it.  The release build
 * returns FS4D_ERR_UNIMPLEMENTED.  fs4d_debug_corrupt_canary overwrites one canary
 * byte of the most recently allocated buffer (a test of the check itself; release
 * build: FS4D_ERR_UNIMPLEMENTED). */
FS4D_API fs4d_status fs4d_check_canaries(fs4d_ctx* ctx);
FS4D_API fs4d_status fs4d_debug_corrupt_canary(fs4d_ctx* ctx);
/* Polls a look-back wait (radix sort, key emission) of this context's later
 * launches makes before it gives up and sets the timeout bit of the status word;
 * 0 restores the default (2^22 polls of ~100 ns).  A diagnostic for exercising
 * the timeout path: a small limit makes waits give up while their predecessors
 * are still running, so results are wrong but every access stays in bounds. */
FS4D_API fs4d_status fs4d_set_wait_limit(fs4d_ctx* ctx, uint32_t polls);

/* ---------------------------------------------------------------- scenes */

/* Copy a canonical scene to the device and prepare both precisions (float32
 * planes/MLP and the bfloat16 tensor-core operand layouts).  Synchronous. */
FS4D_API fs4d_status fs4d_load_scene(fs4d_ctx* ctx, const fs4d_scene_desc* desc, fs4d_scene_id* out);
FS4D_API fs4d_status fs4d_unload_scene(fs4d_ctx* ctx, fs4d_scene_id id);
/* Overwrite the parameters of a loaded scene (same n, SH degree, plane and MLP
 * shapes; the box may not change).  Array pointers are DEVICE pointers when
 * on_device != 0, else HOST pointers; a NULL array keeps its current values.
 * Re-derives the BF16 and transposed MLP copies.  Synchronises the stream. */
FS4D_API fs4d_status fs4d_update_scene(fs4d_ctx* ctx, fs4d_scene_id id, const fs4d_scene_desc* desc,
                                       int32_t on_device);
/* Copy the scene's current parameters (after any training steps) into the
 * non-NULL arrays of *out, in the layouts of fs4d_scene_desc: HOST memory when
 * to_device == 0, else DEVICE memory.  Synchronises the context's stream. */
FS4D_API fs4d_status fs4d_read_scene(fs4d_ctx* ctx, fs4d_scene_id id, const fs4d_grads* out, int32_t to_device);
/* Write the scene (sizes, box and current parameters) to a binary file: an
 * 8-byte magic "FS4DSCN2", eleven int32 (n, sh_degree, n_levels, res_spatial[4],
 * res_time, feat_dim, mlp_width, color_heads), the box (6 float32), the arrays means,
 * log_scales, quats, opacity_logits, sh, planes, mlp as little-endian float32,
 * and a 64-bit FNV-1a checksum of everything after the magic.  The file is
 * written under path + ".tmp" and renamed, so a reader never sees half a file. */
FS4D_API fs4d_status fs4d_save_scene(fs4d_ctx* ctx, fs4d_scene_id id, const char* path);
/* Load a file written by fs4d_save_scene as a new scene (FS4D_ERR_NOT_FOUND if it
 * cannot be opened, FS4D_ERR_INVALID_ARG if it is not a complete scene file).  Files
 * with the magic "FS4DSCN1" (ten int32, no color_heads) load as scenes without them. */
FS4D_API fs4d_status fs4d_load_scene_file(fs4d_ctx* ctx, const char* path, fs4d_scene_id* out);
/* Bytes the scene holds resident on the device, and the per-frame work memory a
 * render at (width, height) needs with `pairs_per_gaussian` tile pairs per
 * Gaussian (used for admission by device-memory footprint). */
FS4D_API fs4d_status fs4d_scene_bytes(fs4d_ctx* ctx, fs4d_scene_id id, int32_t width, int32_t height,
                             float pairs_per_gaussian, size_t* resident, size_t* per_frame);

/* ---------------------------------------------------------------- the path */

/* Eq. 5 + Sec. 4.2 + Eq. 6: deform the scene at each of n_t timestamps in ONE
 * launch.  h_ts: host [n_t] in [0,1].  Outputs (device, caller-owned):
 * d_means [n_t][n][3], d_quats [n_t][n][4], d_log_scales [n_t][n][3]. */
FS4D_API fs4d_status fs4d_deform(fs4d_ctx* ctx, fs4d_scene_id id, fs4d_precision prec, const float* h_ts, int32_t n_t,
                        float* d_means, float* d_quats, float* d_log_scales);

/* Render one frame, I = S(M, G') with G' = G + F(G, t) (Sec. 4.1): deform at t
 * (Eq. 5, Eq. 6), project (Eq. 2, Eq. 3), bin, sort, composite (Eq. 1, Eq. 4).
 * A frame with more than 2^30 - 1 tile pairs (what one pair-sort pass counts) is
 * rendered in horizontal bands of whole tile rows, each binned, sorted and
 * composited on its own over the same deformed Gaussians (fs4d_last_pairs then
 * gives the pairs of all bands); a frame saved for the backward must fit one
 * pass (FS4D_ERR_CAPACITY otherwise).  d_image:
 * device [height][width][3]; d_t_final [height][width] and d_n_contrib
 * [height][width] may be NULL.  If `saved` is non-NULL, *saved receives the
 * forward state needed by fs4d_render_backward (free it with fs4d_frame_free).
 * The number of tile pairs is read back once per call (one stream sync). */
FS4D_API fs4d_status fs4d_render(fs4d_ctx* ctx, fs4d_scene_id id, fs4d_precision prec, const fs4d_camera* cam, float t,
                        float* d_image, float* d_t_final, int32_t* d_n_contrib, fs4d_frame** saved);

/* Composition (Sec. 5.4): one frame of several loaded scenes, I = S(M, G') with
 * G' = {G'_1, ..., G'_n} the union of every scene's Gaussians deformed at t (each
 * by its own HexPlane and MLP), binned, sorted and composited together, so that
 * their Gaussians interleave in depth.  h_shifts (host [n_scenes][3], or NULL)
 * translates each scene in the world (its SH colour sees the view direction from
 * the camera to the translated mean).  Outputs as fs4d_render; the frame must fit
 * one band of tile pairs (FS4D_ERR_CAPACITY otherwise). */
FS4D_API fs4d_status fs4d_render_composed(fs4d_ctx* ctx, const fs4d_scene_id* ids, const float* h_shifts,
                                          int32_t n_scenes, fs4d_precision prec, const fs4d_camera* cam, float t,
                                          float* d_image, float* d_t_final, int32_t* d_n_contrib);

/* The same frame end to end with HOST buffers: the camera and t go host->device,
 * the image comes back into h_image [height][width][3] (pinned memory is fastest).
 * One host synchronisation per frame: the pair count comes back with the image, and
 * a frame whose pairs overflowed the context's capacity is rendered again with the
 * capacity grown.  Returns after the image is on the host. */
FS4D_API fs4d_status fs4d_render_host(fs4d_ctx* ctx, fs4d_scene_id id, fs4d_precision prec, const fs4d_camera* cam,
                             float t, float* h_image);
/* n frames to HOST images: frame k is (cams[k], ts[k]) into h_images[k] ([height]
 * [width][3]; every camera of one size; host arrays of n entries).  Frames render
 * into two device image buffers in turn, and each image's copy to the host overlaps
 * the next frame's render (pinned destinations keep the copies asynchronous; the
 * same destination may be given for several frames: they are written in order).
 * Returns when every image is on the host; frames whose pairs overflowed the
 * context's capacity are rendered again with the capacity grown. */
FS4D_API fs4d_status fs4d_render_host_batch(fs4d_ctx* ctx, fs4d_scene_id id, fs4d_precision prec,
                                            const fs4d_camera* cams, const float* ts, int32_t n,
                                            float* const* h_images);

/* Capacity mode: render without any host synchronisation (so the call can be
 * captured into a CUDA graph).  The tile-pair buffers hold `pair_capacity` pairs;
 * a frame that needs more sets the device status word (fs4d_check_device_status
 * then returns FS4D_ERR_CAPACITY) and its image is incomplete.  The camera and t
 * are read from DEVICE memory (d_cam: one fs4d_camera, d_t: one float) so that a
 * captured graph can be replayed for new views. */
FS4D_API fs4d_status fs4d_reserve(fs4d_ctx* ctx, fs4d_scene_id id, int32_t width, int32_t height, int64_t pair_capacity);
FS4D_API fs4d_status fs4d_render_async(fs4d_ctx* ctx, fs4d_scene_id id, fs4d_precision prec, const fs4d_camera* h_cam_shape,
                              const fs4d_camera* d_cam, const float* d_t, float* d_image);

/* Backward of one saved frame (training, Sec. 4.3): gradients of
 * sum(d_dl_dimage * image) with respect to every scene parameter.
 * d_dl_dimage: device [height][width][3].  Gradients are ACCUMULATED (+=) into the
 * non-NULL pointers of *d_grads. */
FS4D_API fs4d_status fs4d_render_backward(fs4d_ctx* ctx, fs4d_frame* saved, const float* d_dl_dimage,
                                 const fs4d_grads* d_grads);
FS4D_API fs4d_status fs4d_frame_free(fs4d_ctx* ctx, fs4d_frame* frame);
/* Number of tile pairs K of a saved frame, and of the last render on the context:
 * the pairs of the Gaussians' tile rectangles (frames of the tile bitmap binning that
 * report no list positions list a Gaussian only in the tiles its ellipse
 * {alpha >= 1/255} reaches, which leaves the image unchanged and their lists shorter). */
FS4D_API fs4d_status fs4d_frame_pairs(const fs4d_frame* frame, int64_t* pairs);
FS4D_API fs4d_status fs4d_last_pairs(const fs4d_ctx* ctx, int64_t* pairs);
/* Number of kernels the last fs4d_render or fs4d_render_async call on the context
 * launched from the calling thread (memsets and copies not counted; a frame captured
 * into a graph launches the same kernels on every replay).  FS4D_ERR_INVALID_ARG on
 * NULL arguments. */
FS4D_API fs4d_status fs4d_last_launches(const fs4d_ctx* ctx, int64_t* launches);
/* Number of bands of tile rows the last fs4d_render / fs4d_render_host frame on the
 * context was rendered in (1 unless its pairs exceeded one pair-sort pass). */
FS4D_API fs4d_status fs4d_last_bands(const fs4d_ctx* ctx, int32_t* bands);
/* Most tile pairs one band of a frame may hold (0 = the default and maximum,
 * 2^30 - 1).  A smaller value bounds the pair buffers' device memory (24 bytes per
 * pair with the sort's second buffer) at the cost of more bands. */
FS4D_API fs4d_status fs4d_set_band_pairs(fs4d_ctx* ctx, int64_t max_pairs);

/* Binning policy of the context's frames (FS4D_BINNING_AUTO or FS4D_BINNING_SORT;
 * FS4D_ERR_INVALID_ARG otherwise), and the binning the last frame rendered on the
 * context (not the server's) used.  fs4d_bin_sort follows the same policy. */
FS4D_API fs4d_status fs4d_set_binning(fs4d_ctx* ctx, int32_t mode);
FS4D_API fs4d_status fs4d_last_binning(const fs4d_ctx* ctx, int32_t* mode);

/* Per-stage device timing of frames rendered by fs4d_render / fs4d_render_async
 * (also inside a captured CUDA graph): when enabled, CUDA events are recorded on
 * the context's stream around each stage.  fs4d_stage_times waits for the last
 * recorded frame and writes ms[6] = deform, project, depth sort, binning (key
 * emission or tile bitmap, with the tile scan that writes the ranges), pair sort,
 * composite (milliseconds, that frame only; for a frame rendered in bands of tile
 * rows, each stage summed over the bands). */
FS4D_API fs4d_status fs4d_set_stage_timing(fs4d_ctx* ctx, int32_t enable);
FS4D_API fs4d_status fs4d_stage_times(fs4d_ctx* ctx, float* h_ms);
/* With stage timing enabled, the last fs4d_render_backward's stages: h_ms[4] =
 * compositing backward, projection + SH backward, MLP + HexPlane backward,
 * weight-gradient reductions (milliseconds; waits for that backward). */
FS4D_API fs4d_status fs4d_backward_times(fs4d_ctx* ctx, float* h_ms);

/* ---------------------------------------------------------------- training
 * One training step (Sec. 4.3) on a loaded scene, on the device: render the view
 * keeping the backward's state, the loss L = |I^ - I| + L_tv, its gradient with
 * respect to every parameter group (the backward of fs4d_render_backward plus
 * the TV gradient on the planes), and one Adam update of each group at a learning
 * rate decayed over the run (App. A gives the HexPlane rate 1.6e-3 -> 1.6e-4 and
 * the MLP rate 1.6e-4 -> 1.6e-5).  The scene's parameters are updated in place and
 * its derived copies (BF16 planes and MLP operands) refreshed, so the next frame
 * of any call renders the updated scene.  Readings where the paper is silent:
 *  - |I^ - I| is the mean absolute difference over every pixel and channel;
 *  - L_tv = tv_weight x sum over levels and planes of the mean squared difference
 *    of neighbouring cells along each of the plane's two axes (every channel);
 *  - the decay is log-linear: lr(k) = lr0 (lr1 / lr0)^min(1, k / total_steps);
 *  - Adam is bias-corrected (step k + 1 for the k-th update, k from 0). */
typedef struct fs4d_train_config {
  int32_t total_steps;     /* steps over which every rate decays from [0] to [1] */
  float lr_means[2];       /* initial and final learning rate of each group */
  float lr_log_scales[2];
  float lr_quats[2];
  float lr_opacity[2];
  float lr_sh_dc[2];       /* the degree-0 SH coefficients */
  float lr_sh_rest[2];     /* the higher-degree SH coefficients */
  float lr_planes[2];
  float lr_mlp[2];
  float beta1, beta2, eps; /* Adam */
  float tv_weight;         /* weight of L_tv */
} fs4d_train_config;
typedef struct fs4d_trainer fs4d_trainer;

/* Optimiser state (Adam moments and gradients of every group, zeroed) for scene
 * `id` of the context.  The scene must stay loaded while the trainer exists. */
FS4D_API fs4d_status fs4d_train_create(fs4d_ctx* ctx, fs4d_scene_id id, const fs4d_train_config* cfg,
                                       fs4d_trainer** out);
/* One step on view (cam, t) against d_target (device [height][width][3]): the
 * frame renders with `prec` (the backward is float32 either way).  d_losses
 * (device float[2], or NULL for the trainer's own) receives the L1 and TV losses
 * of this step's frame, before the update.  One host synchronisation (the
 * frame's pair count).  A frame whose pairs exceed one band returns
 * FS4D_ERR_CAPACITY before any update. */
FS4D_API fs4d_status fs4d_train_step(fs4d_trainer* tr, fs4d_precision prec, const fs4d_camera* cam, float t,
                                     const float* d_target, float* d_losses);
/* The L1 and TV losses of the last step into h_losses[2] (when the step wrote
 * them to the trainer's own buffer); synchronises the context's stream. */
FS4D_API fs4d_status fs4d_train_losses(fs4d_trainer* tr, float* h_losses);
FS4D_API fs4d_status fs4d_train_steps_done(const fs4d_trainer* tr, int64_t* steps);
FS4D_API fs4d_status fs4d_train_destroy(fs4d_trainer* tr);
/* Adam moments of parameter group `group` (0 means, 1 log_scales, 2 quats,
 * 3 opacity_logits, 4 sh, 5 planes, 6 mlp; the layouts of fs4d_scene_desc) into
 * the non-NULL host arrays h_m, h_v (the group's size in floats each).
 * Synchronises the context's stream. */
FS4D_API fs4d_status fs4d_train_read_state(fs4d_trainer* tr, int32_t group, float* h_m, float* h_v);

/* ---------------------------------------------------------------- densification
 * Adaptive density control (App. A: the paper keeps the densification and
 * pruning of 3D Gaussian splatting, growing the set until late in training).
 * Statistics: per Gaussian, the summed norm of the gradient of the loss with
 * respect to its projected mean (pixel units) over the backward passes in which
 * it was visible (radius > 0), and the number of those passes.  Readings where
 * the paper is silent: the gradient is taken in pixel units (the threshold is the
 * caller's); a Gaussian is densified when sum / count >= grad_threshold (count 0
 * gives 0), copied when its largest log-scale is at or below split_log_scale,
 * else replaced by two children drawn from N(mu, R S S^T R^T) (Eq. 2) with the
 * scales divided by 1.6; a Gaussian whose opacity logit is below prune_logit is
 * removed, and so is what it would have produced.  The three decisions are taken
 * in float32.  The new set is the kept Gaussians, then the copies, then the first
 * and the second children, each in the old order; copies and children start with
 * zero Adam moments, kept Gaussians keep theirs. */
typedef struct fs4d_view_stats {
  float* grad_norm_sum;  /* device [n], accumulated (+=) */
  float* visible;        /* device [n], accumulated (+=) */
} fs4d_view_stats;
typedef struct fs4d_densify_config {
  float grad_threshold;
  float split_log_scale;
  float prune_logit;
} fs4d_densify_config;

/* fs4d_render_backward that also accumulates the statistics into *d_stats. */
FS4D_API fs4d_status fs4d_render_backward_stats(fs4d_ctx* ctx, fs4d_frame* saved, const float* d_dl_dimage,
                                                const fs4d_grads* d_grads, const fs4d_view_stats* d_stats);
/* Densify and prune scene `id` in place from the statistics *d_stats (device, the
 * scene's current n) and d_normals (device [n][2][3] standard normal draws; row i
 * is read only if Gaussian i is split).  If `trainer` (of this scene) is not
 * NULL its optimiser state follows the Gaussians and its statistics restart at
 * zero (another trainer of the scene can then no longer step: FS4D_ERR_INVALID_ARG).
 * *n_out receives the new
 * number of Gaussians.  FS4D_ERR_INVALID_ARG (and the scene unchanged) if every
 * Gaussian would be removed; FS4D_ERR_CANCELLED if serving requests on the scene
 * are in flight; the scene's capacity reservation (fs4d_reserve) is dropped.
 * Synchronises the context's stream (the new size decides the allocations). */
FS4D_API fs4d_status fs4d_densify(fs4d_ctx* ctx, fs4d_scene_id id, const fs4d_densify_config* cfg,
                                  const fs4d_view_stats* d_stats, const float* d_normals, fs4d_trainer* trainer,
                                  int64_t* n_out);
/* Copy the trainer's own statistics (accumulated by every fs4d_train_step since
 * its creation or last densify) into the caller's non-NULL fields of *d_out
 * (device arrays of the scene's current n floats each). */
FS4D_API fs4d_status fs4d_train_stats(fs4d_trainer* tr, const fs4d_view_stats* d_out);
/* fs4d_densify of the trainer's scene with the trainer's statistics, which then
 * restart at zero. */
FS4D_API fs4d_status fs4d_train_densify(fs4d_trainer* tr, const fs4d_densify_config* cfg, const float* d_normals,
                                        int64_t* n_out);

/* ---------------------------------------------------------------- serving
 * A continuous-batching request loop over the context's resident scenes, run by
 * a native scheduler thread.  Requests (scene, camera, t) are admitted in FIFO
 * order as work slots and device memory free up (a slot holds one in-flight
 * frame's work memory; slots together stay within hbm_budget_bytes).  Admitted
 * requests that share a scene and precision are deformed together in ONE
 * persistent launch (one timestamp per request), then each request's
 * project/bin/sort/composite sequence is replayed from a CUDA graph captured
 * per (slot, scene, resolution, precision) on the slot's own stream, so frames
 * of different requests overlap on the device.  A frame whose tile pairs
 * overflow its slot's capacity is re-run with a larger capacity.  Results do
 * not depend on what else is in flight.  While a server runs, unload a scene
 * only after its requests completed (fs4d_unload_scene waits for in-flight
 * ones; queued ones then complete with FS4D_ERR_NOT_FOUND). */
typedef struct fs4d_server fs4d_server;
typedef struct fs4d_server_config {
  int32_t max_inflight;      /* work slots, i.e. requests on the GPU at once (>= 1) */
  int32_t max_batch;         /* requests of one scene deformed by one launch (>= 1) */
  int64_t hbm_budget_bytes;  /* device memory all slots may hold together */
  float pairs_per_gaussian;  /* first tile-pair capacity guess per Gaussian (grown on overflow) */
} fs4d_server_config;
typedef struct fs4d_request {
  fs4d_scene_id scene;
  fs4d_precision prec;
  fs4d_camera cam;
  float t;
  float* out;                /* [height][width][3]: DEVICE pointer if out_on_device, else HOST
                                pointer (page-locked memory keeps the copy asynchronous) */
  int32_t out_on_device;
} fs4d_request;
typedef struct fs4d_completion {
  uint64_t ticket;
  int32_t status;            /* FS4D_OK, or why this request failed */
  int32_t slot;              /* work slot that ran it (-1 if none) */
  int64_t pairs;             /* tile pairs of the frame */
  double submit_ms, start_ms, done_ms; /* host clock, ms since the server started */
} fs4d_completion;
typedef struct fs4d_server_stats {
  int64_t submitted, completed, failed, retried, batches, deformed;
  int32_t slots, max_concurrent;
  int64_t slot_bytes, peak_slot_bytes;
} fs4d_server_stats;

/* Start a server on the context (at most one per context). */
FS4D_API fs4d_status fs4d_server_create(fs4d_ctx* ctx, const fs4d_server_config* cfg, fs4d_server** out);
/* Queue a request; *ticket identifies its completion.  Thread-safe. */
FS4D_API fs4d_status fs4d_server_submit(fs4d_server* srv, const fs4d_request* req, uint64_t* ticket);
/* Queue n requests at once (they enter the queue together, so requests of one
 * scene among them can share a deformation launch); tickets[n]. */
FS4D_API fs4d_status fs4d_server_submit_batch(fs4d_server* srv, const fs4d_request* reqs, int32_t n,
                                              uint64_t* tickets);
/* Remove a still-queued request (it completes with FS4D_ERR_CANCELLED);
 * FS4D_ERR_NOT_FOUND if it already started or finished. */
FS4D_API fs4d_status fs4d_server_cancel(fs4d_server* srv, uint64_t ticket);
/* Move up to max finished requests into out[]; *n_out = how many. */
FS4D_API fs4d_status fs4d_server_poll(fs4d_server* srv, fs4d_completion* out, int32_t max, int32_t* n_out);
/* Block until nothing is queued or in flight. */
FS4D_API fs4d_status fs4d_server_drain(fs4d_server* srv);
FS4D_API fs4d_status fs4d_server_stats_get(fs4d_server* srv, fs4d_server_stats* out);
/* Stop: queued requests complete with FS4D_ERR_CANCELLED, in-flight ones finish. */
FS4D_API fs4d_status fs4d_server_destroy(fs4d_server* srv);

/* ---------------------------------------------------------------- stages
 * Stateless stages of the path on caller-owned device buffers, so that each can
 * be checked on its own.  The context supplies the stream and work memory. */

/* Eq. 2 + Eq. 3 + SH colour for n Gaussians (d_sh: [n][K][3]); tile = 16. */
FS4D_API fs4d_status fs4d_project(fs4d_ctx* ctx, int32_t n, const float* d_means, const float* d_quats,
                         const float* d_log_scales, const float* d_opacity_logits, const float* d_sh,
                         int32_t sh_degree, const fs4d_camera* cam, const fs4d_projected* out);

/* Tile binning + radix sort + tile ranges.  Inputs: d_depth [n] (float32 whose
 * bits are the low key word) and d_rect [n][4].  Emits one key
 * (tile_id << 32 | depth bits) per (Gaussian, touched tile), tile_id = y*tiles_x + x,
 * sorts the pairs by key (ties keep Gaussian-index order) and writes
 * d_keys/d_values [capacity], d_ranges [tiles_y*tiles_x][2] ([start, end) per tile)
 * and *h_num_pairs = K (the call synchronises once to read it).  Returns
 * FS4D_ERR_CAPACITY (and writes nothing past capacity) if K > capacity. */
FS4D_API fs4d_status fs4d_bin_sort(fs4d_ctx* ctx, int32_t n, const float* d_depth, const int32_t* d_rect, int32_t tiles_x,
                          int32_t tiles_y, int64_t capacity, uint64_t* d_keys, uint32_t* d_values,
                          uint32_t* d_ranges, int64_t* h_num_pairs);

/* Stable LSD radix sort of (key, value) pairs on the low `key_bits` bits of the
 * keys (1..64), in place: d_keys/d_values [n] hold the sorted pairs on return.
 * Uses context-owned work memory. */
FS4D_API fs4d_status fs4d_sort_pairs(fs4d_ctx* ctx, int64_t n, int32_t key_bits, uint64_t* d_keys, uint32_t* d_values);

/* Allocation-free radix sort (no counterpart in the paper; an integration aid).
 * Some callers must not have this library allocate device memory: a host
 * application that owns the whole device-memory budget and hands out every
 * buffer itself, or a latency-critical loop in which cudaMalloc/cudaFree (which
 * can synchronise the whole device) are not allowed.  Such a caller can sort
 * with this call: it needs no context and allocates nothing.  It sorts like
 * fs4d_sort_pairs (stable, low key_bits bits, in place in d_keys/d_values [n])
 * on the given stream (a cudaStream_t of the CURRENT device; NULL = legacy
 * default stream), using a fixed work area of about 14.7 MB that the library
 * keeps in device memory of every GPU that loads it, until the process exits.
 *  - n may be at most FS4D_NOALLOC_MAX_PAIRS; a larger n returns
 *    FS4D_ERR_CAPACITY and launches nothing.  Other bad arguments return
 *    FS4D_ERR_INVALID_ARG, a failed CUDA call FS4D_ERR_CUDA.
 *  - The first call on each device performs a one-time set-up (it looks up the
 *    device address of the work area); make that first call before any stream
 *    capture begins.
 *  - All calls on a device share the one work area (it keeps the last call's
 *    contents; every call clears what must start at zero).  Calls whose work
 *    overlaps on the GPU race with each other: serialise them (one stream, or
 *    events between streams).
 *  - The device address of the work area is cached per device for the life of
 *    the process: do not call it again on a device after cudaDeviceReset.
 *  - The sort's look-back waits are bounded; a wait that gives up sets a status
 *    word instead of hanging, and the call still returns FS4D_OK (it does not
 *    synchronise).  fs4d_sort_pairs_noalloc_status reads that word. */
#define FS4D_NOALLOC_MAX_PAIRS (1 << 20)
FS4D_API fs4d_status fs4d_sort_pairs_noalloc(void* cuda_stream, int64_t n, int32_t key_bits, uint64_t* d_keys,
                                             uint32_t* d_values);
/* Queue on cuda_stream a copy of the status word of the last
 * fs4d_sort_pairs_noalloc queued on the current device into *out (4 bytes of
 * device or page-locked host memory; valid once the stream has been
 * synchronised): 0 when the sort completed, bit 0 set when one of its bounded
 * waits gave up (the sorted output is then unreliable).  Allocates nothing. */
FS4D_API fs4d_status fs4d_sort_pairs_noalloc_status(void* cuda_stream, uint32_t* out);

/* Eq. 4 per 16x16 tile over the sorted lists: d_ranges [tiles][2], d_values [K]
 * Gaussian indices, per-Gaussian d_xy [n][2], d_conic_opacity [n][4], d_rgb [n][3].
 * Writes d_image [height][width][3] and, when non-NULL, d_t_final and
 * d_n_contrib [height][width]. */
FS4D_API fs4d_status fs4d_composite(fs4d_ctx* ctx, int32_t width, int32_t height, const uint32_t* d_ranges,
                           const uint32_t* d_values, const float* d_xy, const float* d_conic_opacity,
                           const float* d_rgb, float* d_image, float* d_t_final, int32_t* d_n_contrib);

#ifdef __cplusplus
}
#endif
#endif /* FS4D_H */
