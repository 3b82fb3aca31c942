/*
 * FP64 CPU oracle for the 4D Gaussian Splatting render path (arXiv 2310.08528).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this code; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark load it.  It shares no header, helper or constant with the CUDA
 * path.
 *
 * Every function computes in double precision from the float32 scene as stored.
 * Where a floating-point value decides an integer (the depth key of a tile
 * pair), the oracle takes that decision in float32, the kernels' precision.
 *
 * Which passage each function follows:
 *   orc_plane_sample / orc_features  Sec. 4.2, Eq. 5 (bilinear interp, Hadamard
 *                                    product over six planes, concat over levels)
 *   orc_mlp / orc_deform             Sec. 4.2 (tiny MLP phi_d, heads phi_x phi_r
 *                                    phi_s) and Eq. 6 (X'=X+dX, r'=r+dr, s'=s+ds)
 *   orc_appearance                   App. B (heads phi_C, phi_alpha: C'=C+dC,
 *                                    opacity logit' = logit + dalpha)
 *   orc_project                      Sec. 3.1, Eq. 2 (Sigma = R S S^T R^T) and
 *                                    Eq. 3 (Sigma' = J W Sigma W^T J^T), SH colour
 *   orc_bin_sort                     tile binning and (tile, depth) ordering of the
 *                                    differentiable splatting the paper uses (Sec. 4.1)
 *   orc_composite                    Eq. 1 (Gaussian weight) and Eq. 4
 *                                    (front-to-back alpha blending)
 *   orc_composite_bruteforce         the same blend as a per-pixel loop over all
 *                                    Gaussians (no tiling), used as a pin
 *   orc_pixel_outcomes               Eq. 4 for one pixel with its near-threshold
 *                                    decisions taken either way (parity support)
 *   orc_*_backward                   chain rule of all of the above (training,
 *                                    Sec. 4.3)
 *   orc_l1_loss / orc_tv_loss        the training loss L = |I^ - I| + L_tv (Sec. 4.3)
 *   orc_lr / orc_adam_step           learning-rate decay and Adam update (App. A)
 *   orc_densify                      densification and pruning (App. A, following
 *                                    3D Gaussian splatting's adaptive density control)
 *
 * Parity pins: tests/test_oracle_pins.py and tests/test_oracle_backward.py;
 * tests/test_oracle_planted_mistakes.py builds copies of this oracle with one
 * plausible mistake each and checks that some pin fails for every one.
 * Agreement with the paper's trained results is parity unpinned (no trained
 * weights or datasets exist here).
 */
#ifndef FS4D_ORACLE_H
#define FS4D_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_scene {
  int32_t n;
  int32_t sh_degree;        /* 0..3 */
  const float* means;       /* [n][3] */
  const float* log_scales;  /* [n][3] */
  const float* quats;       /* [n][4] w x y z */
  const float* opacity_logits; /* [n] */
  const float* sh;          /* [n][(deg+1)^2][3] */
  double aabb_min[3];
  double aabb_max[3];
  int32_t n_levels;
  int32_t res_spatial[4];
  int32_t res_time;
  int32_t feat_dim;
  const float* planes;      /* per level, per plane xy xz yz xt yt zt: [R_b][R_a][h] */
  int32_t mlp_width;
  const float* mlp;         /* d1 d2 x1 x2 r1 r2 s1 s2 [c1 c2 a1 a2]: W[out][in] then b[out] */
  int32_t color_heads;      /* 1: the colour and opacity heads phi_C, phi_alpha (App. B) follow */
} orc_scene;

typedef struct orc_camera {
  int32_t width, height;
  double fx, fy, cx, cy, znear;
  double world_to_cam[16]; /* row-major, x right, y down, z forward */
} orc_camera;

/* Projected Gaussian set, all caller-owned arrays of length n (x k). */
typedef struct orc_projected {
  double* xy;       /* [n][2] pixel coordinates of the projected mean */
  double* conic;    /* [n][3] inverse of the dilated 2-D covariance (a, b, c) */
  double* cov2d;    /* [n][3] dilated 2-D covariance (a, b, c) */
  double* opacity;  /* [n] sigmoid(logit) */
  double* rgb;      /* [n][3] */
  double* depth;    /* [n] camera-space z */
  int32_t* radius;  /* [n] 0 = culled */
  int32_t* rect;    /* [n][4] tile x0, y0, x1, y1 (x1, y1 exclusive) */
  double* margin;   /* [n] pixels between a rect/radius decision and its boundary */
} orc_projected;

void orc_set_threads(int32_t n);

void orc_plane_sample(const orc_scene* s, int32_t level, int32_t plane, double ua, double ub, double* out);
void orc_features(const orc_scene* s, const double* xyz, int32_t n, double t, double* fh);
void orc_mlp(const orc_scene* s, const double* fh, int32_t n, double* delta);
void orc_deform(const orc_scene* s, double t, double* means, double* quats, double* log_scales);
void orc_sh_basis(int32_t degree, const double* dir, double* basis);
/* App. B: SH coefficients [n][K][3] and opacity logits [n] after the colour and
 * opacity heads at time t (the canonical values when the scene has none). */
void orc_appearance(const orc_scene* s, double t, double* sh, double* opacity_logits);
/* orc_project with the SH coefficients and opacity logits taken from sh / opacity_logits
 * (double, the shapes of the scene's) instead of the scene's. */
void orc_project_appearance(const orc_scene* s, const double* means, const double* quats,
                            const double* log_scales, const double* sh, const double* opacity_logits,
                            const orc_camera* cam, int32_t tile, orc_projected* out);
void orc_project(const orc_scene* s, const double* means, const double* quats, const double* log_scales,
                 const orc_camera* cam, int32_t tile, orc_projected* out);
int64_t orc_bin_sort(int32_t n, const uint32_t* depth_bits, const int32_t* rect, int32_t tiles_x,
                     int32_t tiles_y, int64_t capacity, uint64_t* keys, uint32_t* values, uint32_t* ranges);
void orc_composite(int32_t width, int32_t height, int32_t tile, const uint32_t* ranges, const uint32_t* values,
                   const double* xy, const double* conic, const double* opacity, const double* rgb,
                   const double* depth, double* image, double* t_final, int32_t* n_contrib, double* margin);
void orc_composite_bruteforce(int32_t n, int32_t width, int32_t height, int32_t tile, const int32_t* radius,
                              const int32_t* rect, const double* xy, const double* conic,
                              const double* opacity, const double* rgb, const double* depth,
                              double* image, double* t_final);
/* Test support (not part of the method): every colour one pixel's blend over
 * `list` can take when its discrete decisions within rounding of their thresholds
 * (alpha vs 1/255 and T vs 1e-4 within rel_tol relative, blended depths within
 * depth_tol relative) are taken either way.  Each outcome is 5 doubles: colour
 * (3), final transmittance, 1 + list position of the last blended term; out[0..4]
 * is the blend as computed.  Returns the number of outcomes (2^m for m such
 * decisions), or -1 when m > max_flip or 2^m > max_out. */
int32_t orc_pixel_outcomes(int32_t len, const uint32_t* list, double px, double py, const double* xy,
                           const double* conic, const double* opacity, const double* rgb, const double* depth,
                           double rel_tol, double depth_tol, int32_t max_flip, int32_t max_out, double* out);
int64_t orc_render(const orc_scene* s, const orc_camera* cam, double t, int32_t deform, int32_t tile,
                   double* image, double* t_final, int32_t* n_contrib, double* margin);

/* Backward (Sec. 4.3 training): gradients of sum(dl_dimage * image) with respect to
 * every scene parameter.  grads arrays have the shapes of the scene arrays. */
typedef struct orc_grads {
  double* means;          /* [n][3] */
  double* log_scales;     /* [n][3] */
  double* quats;          /* [n][4] */
  double* opacity_logits; /* [n] */
  double* sh;             /* [n][k][3] */
  double* planes;         /* flat, like the scene's planes */
  double* mlp;            /* flat, like the scene's mlp */
  double* planes_abs;     /* optional: per plane value, the sum over Gaussians of the
                             magnitudes of the terms its gradient sums (test support) */
  double* planes_sens;    /* optional: per plane value, the change of its gradient that a
                             unit error in every Gaussian's ten output gradients (dX', dr',
                             ds') can cause at most: sum over Gaussians of |J|^T 1 (test
                             support: propagation of upstream float32 error) */
  double* xy;             /* optional: [n][2] gradient of the projected mean (pixels),
                             the view-space gradient that densification accumulates */
} orc_grads;

int32_t orc_render_backward(const orc_scene* s, const orc_camera* cam, double t, int32_t deform,
                            int32_t tile, const double* dl_dimage, orc_grads* grads);

/* Training step (Sec. 4.3, App. A). */
double orc_l1_loss(int64_t count, const double* image, const double* target, double* grad);
double orc_tv_loss(const orc_scene* s, double weight, double* grad);
double orc_lr(double lr0, double lr1, int64_t k, int64_t total);
void orc_adam_step(int64_t count, double* param, const double* g, double* m, double* v, double lr, double beta1,
                   double beta2, double eps, int64_t step);

/* Densification and pruning (App. A).  grad_sum[n]: summed |dL/d(projected mean)|
 * over the views a Gaussian was visible in; visible[n]: that number of views;
 * normals[n][2][3]: standard normal draws for the two children of a split.
 * Writes at most cap outputs; returns their number, or -1 if cap is too small. */
int64_t orc_densify(const orc_scene* s, const float* grad_sum, const float* visible, const float* normals,
                    float grad_threshold, float split_log_scale, float prune_logit, int64_t cap, int64_t* src,
                    int32_t* kind, double* means, double* log_scales, double* quats, double* opacity_logits,
                    double* sh);

#ifdef __cplusplus
}
#endif
#endif
