// FP64 CPU oracle for the 4D-GS render path.  TEST INFRASTRUCTURE ONLY: see
// fs4d_oracle.h for what it is, which passage each function follows, and who may
// call it.  Plain loops, no blocking or fusion, so it can be checked by eye
// against the paper.
#include "fs4d_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

// The six planes of the HexPlane, as (first axis, second axis); axis 3 is time
// (Sec. 4.2: (x,y), (x,z), (y,z), (x,t), (y,t), (z,t)).
const int kPlaneAxes[6][2] = {{0, 1}, {0, 2}, {1, 2}, {0, 3}, {1, 3}, {2, 3}};
const int kHeadOut[3] = {3, 4, 3};

int plane_res(const orc_scene* s, int level, int axis) {
  return axis < 3 ? s->res_spatial[level] : s->res_time;
}

// Start (in floats) of plane (level, p) inside the packed plane buffer.
int64_t plane_offset(const orc_scene* s, int level, int p) {
  int64_t off = 0;
  for (int l = 0; l < s->n_levels; ++l)
    for (int q = 0; q < 6; ++q) {
      if (l == level && q == p) return off;
      off += (int64_t)plane_res(s, l, kPlaneAxes[q][0]) * plane_res(s, l, kPlaneAxes[q][1]) * s->feat_dim;
    }
  return off;
}


// Bilinear-interpolation setup along one axis of resolution R, for a coordinate
// u normalised to [-1, 1].  Vertex k sits at u = -1 + 2k/(R-1) (corner-aligned);
// coordinates outside the box are clamped to its border.
void axis_setup(double u, int R, int* i0, double* f, double* dgdu) {
  double uc = std::min(1.0, std::max(-1.0, u));
  double g = (uc + 1.0) * 0.5 * (R - 1);
  int i = (int)std::floor(g);
  if (i > R - 2) i = R - 2;
  if (i < 0) i = 0;
  *i0 = i;
  *f = g - i;
  // d g / d u, zero where the coordinate is clamped.
  *dgdu = (u > -1.0 && u < 1.0) ? 0.5 * (R - 1) : 0.0;
}

// Layer (out, in) shapes d1 d2 x1 x2 r1 r2 s1 s2 and the float offset of each.
struct MlpLayout {
  int out[8], in[8];
  int64_t w[8], b[8];
  int64_t total;
};

MlpLayout mlp_layout(const orc_scene* s) {
  MlpLayout L;
  int W = s->mlp_width, hin = s->feat_dim * s->n_levels;
  L.out[0] = W; L.in[0] = hin;
  L.out[1] = W; L.in[1] = W;
  for (int h = 0; h < 3; ++h) {
    L.out[2 + 2 * h] = W; L.in[2 + 2 * h] = W;
    L.out[3 + 2 * h] = kHeadOut[h]; L.in[3 + 2 * h] = W;
  }
  int64_t off = 0;
  for (int k = 0; k < 8; ++k) {
    L.w[k] = off; off += (int64_t)L.out[k] * L.in[k];
    L.b[k] = off; off += L.out[k];
  }
  L.total = off;
  return L;
}

// y = W x + b for layer k of the packed MLP.
void linear(const orc_scene* s, const MlpLayout& L, int k, const double* x, double* y) {
  for (int o = 0; o < L.out[k]; ++o) {
    double acc = s->mlp[L.b[k] + o];
    for (int i = 0; i < L.in[k]; ++i) acc += (double)s->mlp[L.w[k] + (int64_t)o * L.in[k] + i] * x[i];
    y[o] = acc;
  }
}

double relu(double v) { return v > 0.0 ? v : 0.0; }

// Normalised 4-D coordinate (x, y, z, t) in [-1, 1]: the scene box maps to the
// grid (Sec. 4.2, "bounding plane voxels"), t in [0, 1] maps to [-1, 1].
void normalise(const orc_scene* s, const double* xyz, double t, double c[4]) {
  for (int a = 0; a < 3; ++a) c[a] = 2.0 * (xyz[a] - s->aabb_min[a]) / (s->aabb_max[a] - s->aabb_min[a]) - 1.0;
  c[3] = 2.0 * t - 1.0;
}

// Real spherical harmonics up to degree 3 (textbook real basis, no Condon-Shortley
// phase), ordered by degree then m = -l..l.
void sh_basis(int degree, const double d[3], double* Y) {
  const double x = d[0], y = d[1], z = d[2];
  const double PI = 3.14159265358979323846;
  Y[0] = 0.5 * std::sqrt(1.0 / PI);
  if (degree < 1) return;
  const double c1 = std::sqrt(3.0 / (4.0 * PI));
  Y[1] = c1 * y; Y[2] = c1 * z; Y[3] = c1 * x;
  if (degree < 2) return;
  Y[4] = 0.5 * std::sqrt(15.0 / PI) * x * y;
  Y[5] = 0.5 * std::sqrt(15.0 / PI) * y * z;
  Y[6] = 0.25 * std::sqrt(5.0 / PI) * (3.0 * z * z - 1.0);
  Y[7] = 0.5 * std::sqrt(15.0 / PI) * x * z;
  Y[8] = 0.25 * std::sqrt(15.0 / PI) * (x * x - y * y);
  if (degree < 3) return;
  Y[9] = 0.25 * std::sqrt(35.0 / (2.0 * PI)) * y * (3.0 * x * x - y * y);
  Y[10] = 0.5 * std::sqrt(105.0 / PI) * x * y * z;
  Y[11] = 0.25 * std::sqrt(21.0 / (2.0 * PI)) * y * (5.0 * z * z - 1.0);
  Y[12] = 0.25 * std::sqrt(7.0 / PI) * z * (5.0 * z * z - 3.0);
  Y[13] = 0.25 * std::sqrt(21.0 / (2.0 * PI)) * x * (5.0 * z * z - 1.0);
  Y[14] = 0.25 * std::sqrt(105.0 / PI) * z * (x * x - y * y);
  Y[15] = 0.25 * std::sqrt(35.0 / (2.0 * PI)) * x * (x * x - 3.0 * y * y);
}

// Rotation matrix of a unit quaternion (w, x, y, z).
void quat_to_rot(const double q[4], double R[3][3]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - w * z);     R[0][2] = 2 * (x * z + w * y);
  R[1][0] = 2 * (x * y + w * z);     R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - w * x);
  R[2][0] = 2 * (x * z - w * y);     R[2][1] = 2 * (y * z + w * x);     R[2][2] = 1 - 2 * (x * x + y * y);
}

double frac_margin(double v) {  // distance (in v's units) to the nearest integer
  return std::fabs(v - std::floor(v + 0.5));
}

const double kAlphaMax = 0.99;
const double kAlphaMin = 1.0 / 255.0;
const double kTMin = 1e-4;
const double kDilation = 0.3;
const double kGuard = 1.3;

}  // namespace

extern "C" {

void orc_set_threads(int32_t n) {
#ifdef _OPENMP
  omp_set_num_threads(n > 0 ? n : 1);
#else
  (void)n;
#endif
}

// Eq. 5 "interp": bilinear interpolation of the 4 grid vertices around (ua, ub).
void orc_plane_sample(const orc_scene* s, int32_t level, int32_t p, double ua, double ub, double* out) {
  const int h = s->feat_dim;
  const int Ra = plane_res(s, level, kPlaneAxes[p][0]);
  const int Rb = plane_res(s, level, kPlaneAxes[p][1]);
  const float* P = s->planes + plane_offset(s, level, p);
  int i0, j0;
  double fa, fb, da, db;
  axis_setup(ua, Ra, &i0, &fa, &da);
  axis_setup(ub, Rb, &j0, &fb, &db);
  for (int c = 0; c < h; ++c) {
    double v00 = P[((int64_t)j0 * Ra + i0) * h + c];
    double v10 = P[((int64_t)j0 * Ra + i0 + 1) * h + c];
    double v01 = P[((int64_t)(j0 + 1) * Ra + i0) * h + c];
    double v11 = P[((int64_t)(j0 + 1) * Ra + i0 + 1) * h + c];
    out[c] = (1 - fa) * (1 - fb) * v00 + fa * (1 - fb) * v10 + (1 - fa) * fb * v01 + fa * fb * v11;
  }
}

// Eq. 5: f_h = concat over levels of the Hadamard product over the six planes.
void orc_features(const orc_scene* s, const double* xyz, int32_t n, double t, double* fh) {
  const int h = s->feat_dim, L = s->n_levels;
#pragma omp parallel for schedule(static)
  for (int g = 0; g < n; ++g) {
    double c[4];
    normalise(s, xyz + 3 * (int64_t)g, t, c);
    std::vector<double> v(h);
    for (int l = 0; l < L; ++l) {
      double* f = fh + (int64_t)g * h * L + (int64_t)l * h;
      for (int k = 0; k < h; ++k) f[k] = 1.0;
      for (int p = 0; p < 6; ++p) {
        orc_plane_sample(s, l, p, c[kPlaneAxes[p][0]], c[kPlaneAxes[p][1]], v.data());
        for (int k = 0; k < h; ++k) f[k] *= v[k];
      }
    }
  }
}

// Sec. 4.2: f_d = phi_d(f_h); dX = phi_x(f_d), dr = phi_r(f_d), ds = phi_s(f_d).
// delta is [n][10] = (dX 3, dr 4, ds 3).
void orc_mlp(const orc_scene* s, const double* fh, int32_t n, double* delta) {
  const MlpLayout Lo = mlp_layout(s);
  const int W = s->mlp_width, hin = s->feat_dim * s->n_levels;
#pragma omp parallel for schedule(static)
  for (int g = 0; g < n; ++g) {
    std::vector<double> a1(W), fd(W), hid(W), out(4);
    linear(s, Lo, 0, fh + (int64_t)g * hin, a1.data());
    for (auto& v : a1) v = relu(v);
    linear(s, Lo, 1, a1.data(), fd.data());
    for (auto& v : fd) v = relu(v);
    int col = 0;
    for (int head = 0; head < 3; ++head) {
      linear(s, Lo, 2 + 2 * head, fd.data(), hid.data());
      for (auto& v : hid) v = relu(v);
      linear(s, Lo, 3 + 2 * head, hid.data(), out.data());
      for (int o = 0; o < kHeadOut[head]; ++o) delta[(int64_t)g * 10 + col + o] = out[o];
      col += kHeadOut[head];
    }
  }
}

// Eq. 6: (X', r', s') = (X + dX, r + dr, s + ds); opacity and SH are unchanged.
void orc_deform(const orc_scene* s, double t, double* means, double* quats, double* log_scales) {
  const int n = s->n, hin = s->feat_dim * s->n_levels;
  std::vector<double> xyz(3 * (int64_t)n), fh((int64_t)n * hin), delta((int64_t)n * 10);
  for (int64_t i = 0; i < 3 * (int64_t)n; ++i) xyz[i] = s->means[i];
  orc_features(s, xyz.data(), n, t, fh.data());
  orc_mlp(s, fh.data(), n, delta.data());
  for (int64_t g = 0; g < n; ++g) {
    for (int a = 0; a < 3; ++a) means[3 * g + a] = (double)s->means[3 * g + a] + delta[10 * g + a];
    for (int a = 0; a < 4; ++a) quats[4 * g + a] = (double)s->quats[4 * g + a] + delta[10 * g + 3 + a];
    for (int a = 0; a < 3; ++a) log_scales[3 * g + a] = (double)s->log_scales[3 * g + a] + delta[10 * g + 7 + a];
  }
}

void orc_sh_basis(int32_t degree, const double* dir, double* basis) { sh_basis(degree, dir, basis); }

// Eq. 2 and Eq. 3 (EWA splatting), colour from SH, screen-space tile rectangle.
void orc_project(const orc_scene* s, const double* means, const double* quats, const double* log_scales,
                 const orc_camera* cam, int32_t tile, orc_projected* out) {
  const int n = s->n;
  const int K = (s->sh_degree + 1) * (s->sh_degree + 1);
  const int tiles_x = (cam->width + tile - 1) / tile, tiles_y = (cam->height + tile - 1) / tile;
  const double* M = cam->world_to_cam;
  double Rc[3][3], tc[3], campos[3];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) Rc[r][c] = M[4 * r + c];
    tc[r] = M[4 * r + 3];
  }
  for (int c = 0; c < 3; ++c) campos[c] = -(Rc[0][c] * tc[0] + Rc[1][c] * tc[1] + Rc[2][c] * tc[2]);
  const double limx = kGuard * cam->width / (2.0 * cam->fx), limy = kGuard * cam->height / (2.0 * cam->fy);

#pragma omp parallel for schedule(static)
  for (int g = 0; g < n; ++g) {
    const double* X = means + 3 * (int64_t)g;
    out->radius[g] = 0;
    for (int k = 0; k < 4; ++k) out->rect[4 * (int64_t)g + k] = 0;
    out->margin[g] = 1e30;
    double p[3];
    for (int r = 0; r < 3; ++r) p[r] = Rc[r][0] * X[0] + Rc[r][1] * X[1] + Rc[r][2] * X[2] + tc[r];
    out->depth[g] = p[2];
    out->opacity[g] = 1.0 / (1.0 + std::exp(-(double)s->opacity_logits[g]));
    out->margin[g] = std::min(out->margin[g], std::fabs(p[2] - cam->znear));
    if (!(p[2] > cam->znear)) continue;
    // Sigma = R S S^T R^T with R from the normalised quaternion, S = diag(exp(s')).
    double q[4], qn = 0;
    for (int k = 0; k < 4; ++k) { q[k] = quats[4 * (int64_t)g + k]; qn += q[k] * q[k]; }
    qn = std::sqrt(qn);
    for (int k = 0; k < 4; ++k) q[k] /= qn;
    double R[3][3];
    quat_to_rot(q, R);
    double S[3];
    for (int k = 0; k < 3; ++k) S[k] = std::exp(log_scales[3 * (int64_t)g + k]);
    double Sig[3][3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) {
        double acc = 0;
        for (int k = 0; k < 3; ++k) acc += R[i][k] * S[k] * S[k] * R[j][k];
        Sig[i][j] = acc;
      }
    // Jacobian of the perspective map at the mean (guard-band clamped).
    double txz = std::min(limx, std::max(-limx, p[0] / p[2])) * p[2];
    double tyz = std::min(limy, std::max(-limy, p[1] / p[2])) * p[2];
    double J[2][3] = {{cam->fx / p[2], 0.0, -cam->fx * txz / (p[2] * p[2])},
                      {0.0, cam->fy / p[2], -cam->fy * tyz / (p[2] * p[2])}};
    double T[2][3];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 3; ++j) T[i][j] = J[i][0] * Rc[0][j] + J[i][1] * Rc[1][j] + J[i][2] * Rc[2][j];
    double C2[2][2];
    for (int i = 0; i < 2; ++i)
      for (int j = 0; j < 2; ++j) {
        double acc = 0;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) acc += T[i][a] * Sig[a][b] * T[j][b];
        C2[i][j] = acc;
      }
    double a = C2[0][0] + kDilation, b = C2[0][1], c = C2[1][1] + kDilation;
    out->cov2d[3 * (int64_t)g + 0] = a;
    out->cov2d[3 * (int64_t)g + 1] = b;
    out->cov2d[3 * (int64_t)g + 2] = c;
    double det = a * c - b * b;
    if (!(det > 0.0)) continue;
    out->conic[3 * (int64_t)g + 0] = c / det;
    out->conic[3 * (int64_t)g + 1] = -b / det;
    out->conic[3 * (int64_t)g + 2] = a / det;
    double mid = 0.5 * (a + c);
    double lmax = mid + std::sqrt(std::max(0.0, mid * mid - det));
    double r3 = 3.0 * std::sqrt(lmax);
    int radius = (int)std::ceil(r3);
    double u = cam->fx * p[0] / p[2] + cam->cx, v = cam->fy * p[1] / p[2] + cam->cy;
    out->xy[2 * (int64_t)g + 0] = u;
    out->xy[2 * (int64_t)g + 1] = v;
    double mg = frac_margin(r3);
    int x0 = (int)std::floor((u - radius) / tile), x1 = (int)std::floor((u + radius) / tile) + 1;
    int y0 = (int)std::floor((v - radius) / tile), y1 = (int)std::floor((v + radius) / tile) + 1;
    mg = std::min(mg, tile * std::min(frac_margin((u - radius) / tile), frac_margin((u + radius) / tile)));
    mg = std::min(mg, tile * std::min(frac_margin((v - radius) / tile), frac_margin((v + radius) / tile)));
    out->margin[g] = std::min(out->margin[g], mg);
    x0 = std::min(tiles_x, std::max(0, x0)); x1 = std::min(tiles_x, std::max(0, x1));
    y0 = std::min(tiles_y, std::max(0, y0)); y1 = std::min(tiles_y, std::max(0, y1));
    if (x1 <= x0 || y1 <= y0) continue;
    out->radius[g] = radius;
    int32_t* rc = out->rect + 4 * (int64_t)g;
    rc[0] = x0; rc[1] = y0; rc[2] = x1; rc[3] = y1;
    // Colour: SH evaluated along the viewing direction, offset by 0.5, clamped at 0.
    double dir[3], dn = 0;
    for (int k = 0; k < 3; ++k) { dir[k] = X[k] - campos[k]; dn += dir[k] * dir[k]; }
    dn = std::sqrt(dn);
    for (int k = 0; k < 3; ++k) dir[k] /= dn;
    double Y[16];
    sh_basis(s->sh_degree, dir, Y);
    for (int ch = 0; ch < 3; ++ch) {
      double acc = 0.5;
      for (int k = 0; k < K; ++k) acc += Y[k] * (double)s->sh[((int64_t)g * K + k) * 3 + ch];
      out->rgb[3 * (int64_t)g + ch] = std::max(0.0, acc);
    }
  }
}

// One (tile, depth) key per Gaussian and touched tile, emitted in Gaussian order
// and, within a Gaussian, in row-major tile order; then a stable sort on the key
// (so equal keys stay in Gaussian-index order) and per-tile [start, end) ranges.
int64_t orc_bin_sort(int32_t n, const uint32_t* depth_bits, const int32_t* rect, int32_t tiles_x,
                     int32_t tiles_y, int64_t capacity, uint64_t* keys, uint32_t* values, uint32_t* ranges) {
  std::vector<std::pair<uint64_t, uint32_t>> pairs;
  for (int g = 0; g < n; ++g) {
    const int32_t* rc = rect + 4 * (int64_t)g;
    for (int ty = rc[1]; ty < rc[3]; ++ty)
      for (int tx = rc[0]; tx < rc[2]; ++tx) {
        uint64_t tile_id = (uint64_t)ty * tiles_x + tx;
        pairs.push_back({(tile_id << 32) | depth_bits[g], (uint32_t)g});
      }
  }
  std::stable_sort(pairs.begin(), pairs.end(),
                   [](const std::pair<uint64_t, uint32_t>& a, const std::pair<uint64_t, uint32_t>& b) {
                     return a.first < b.first;
                   });
  const int64_t K = (int64_t)pairs.size();
  for (int64_t i = 0; i < std::min(K, capacity); ++i) {
    keys[i] = pairs[i].first;
    values[i] = pairs[i].second;
  }
  if (ranges) {
    std::memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)tiles_x * tiles_y);
    for (int64_t i = 0; i < K; ++i) {
      uint32_t tile_id = (uint32_t)(pairs[i].first >> 32);
      if (i == 0 || (uint32_t)(pairs[i - 1].first >> 32) != tile_id) ranges[2 * tile_id] = (uint32_t)i;
      if (i == K - 1 || (uint32_t)(pairs[i + 1].first >> 32) != tile_id) ranges[2 * tile_id + 1] = (uint32_t)(i + 1);
    }
  }
  return K;
}

// Eq. 4 with Eq. 1: per pixel, front to back over its tile's sorted list,
// C = sum_i c_i a_i prod_{j<i} (1 - a_j), a_i = min(0.99, o_i exp(-d^T conic d / 2)).
// Terms with a_i < 1/255 are skipped; the loop stops before the term that would
// take the transmittance below 1e-4.  Pixel (x, y) is evaluated at its centre
// (x + 0.5, y + 0.5); the background is black.
void orc_composite(int32_t width, int32_t height, int32_t tile, const uint32_t* ranges, const uint32_t* values,
                   const double* xy, const double* conic, const double* opacity, const double* rgb,
                   const double* depth, double* image, double* t_final, int32_t* n_contrib, double* margin) {
  const int tiles_x = (width + tile - 1) / tile;
#pragma omp parallel for schedule(dynamic, 16)
  for (int pix = 0; pix < width * height; ++pix) {
    const int px = pix % width, py = pix / width;
    const int tid = (py / tile) * tiles_x + (px / tile);
    const uint32_t start = ranges[2 * tid], end = ranges[2 * tid + 1];
    double T = 1.0, C[3] = {0, 0, 0}, mg = 1e30, prev_depth = -1.0;
    int last = 0;
    const double cx = px + 0.5, cy = py + 0.5;
    for (uint32_t k = start; k < end; ++k) {
      const uint32_t g = values[k];
      const double dx = xy[2 * g] - cx, dy = xy[2 * g + 1] - cy;
      const double power = -0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) - conic[3 * g + 1] * dx * dy;
      if (power > 0.0) continue;
      const double a_raw = opacity[g] * std::exp(power);
      const double alpha = std::min(kAlphaMax, a_raw);
      mg = std::min(mg, std::fabs(alpha - kAlphaMin) / kAlphaMin);
      if (alpha < kAlphaMin) continue;
      // Two blended terms whose depths tie to within float32 rounding may be
      // ordered differently by a float32 implementation: record the relative gap
      // (weighted x100, so one threshold of 5e-5 flags alpha/T decisions within
      // 5e-5 and depth gaps within 5e-7, ~8 float32 ulps, relative).
      if (prev_depth > 0.0) mg = std::min(mg, 100.0 * std::fabs(depth[g] - prev_depth) / std::fabs(depth[g]));
      prev_depth = depth[g];
      const double Tn = T * (1.0 - alpha);
      mg = std::min(mg, std::fabs(Tn - kTMin) / kTMin);
      if (Tn < kTMin) break;
      for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * g + ch] * alpha * T;
      T = Tn;
      last = (int)(k - start) + 1;
    }
    for (int ch = 0; ch < 3; ++ch) image[3 * (int64_t)pix + ch] = C[ch];
    if (t_final) t_final[pix] = T;
    if (n_contrib) n_contrib[pix] = last;
    if (margin) margin[pix] = mg;
  }
}

// The same blend without tiling: every pixel walks all visible Gaussians in
// (float32 depth, index) order and keeps those whose tile rectangle holds the
// pixel's tile.
void orc_composite_bruteforce(int32_t n, int32_t width, int32_t height, int32_t tile, const int32_t* radius,
                              const int32_t* rect, const double* xy, const double* conic,
                              const double* opacity, const double* rgb, const double* depth,
                              double* image, double* t_final) {
  std::vector<int> order;
  for (int g = 0; g < n; ++g)
    if (radius[g] > 0) order.push_back(g);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return (float)depth[a] < (float)depth[b];
  });
#pragma omp parallel for schedule(dynamic, 16)
  for (int pix = 0; pix < width * height; ++pix) {
    const int px = pix % width, py = pix / width, tx = px / tile, ty = py / tile;
    double T = 1.0, C[3] = {0, 0, 0};
    const double cx = px + 0.5, cy = py + 0.5;
    for (int g : order) {
      const int32_t* rc = rect + 4 * (int64_t)g;
      if (tx < rc[0] || tx >= rc[2] || ty < rc[1] || ty >= rc[3]) continue;
      const double dx = xy[2 * g] - cx, dy = xy[2 * g + 1] - cy;
      const double power = -0.5 * (conic[3 * g] * dx * dx + conic[3 * g + 2] * dy * dy) - conic[3 * g + 1] * dx * dy;
      if (power > 0.0) continue;
      const double alpha = std::min(kAlphaMax, opacity[g] * std::exp(power));
      if (alpha < kAlphaMin) continue;
      const double Tn = T * (1.0 - alpha);
      if (Tn < kTMin) break;
      for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * g + ch] * alpha * T;
      T = Tn;
    }
    for (int ch = 0; ch < 3; ++ch) image[3 * (int64_t)pix + ch] = C[ch];
    if (t_final) t_final[pix] = T;
  }
}

// Full frame: deform (or not, for the static 3D-GS special case), project, bin,
// sort and composite.  Returns the number of (tile, Gaussian) pairs.
int64_t orc_render(const orc_scene* s, const orc_camera* cam, double t, int32_t deform, int32_t tile,
                   double* image, double* t_final, int32_t* n_contrib, double* margin) {
  const int n = s->n;
  std::vector<double> X(3 * (int64_t)n), Q(4 * (int64_t)n), Sc(3 * (int64_t)n);
  if (deform) {
    orc_deform(s, t, X.data(), Q.data(), Sc.data());
  } else {
    for (int64_t i = 0; i < 3 * (int64_t)n; ++i) { X[i] = s->means[i]; Sc[i] = s->log_scales[i]; }
    for (int64_t i = 0; i < 4 * (int64_t)n; ++i) Q[i] = s->quats[i];
  }
  std::vector<double> xy(2 * (int64_t)n), conic(3 * (int64_t)n, 0.0), cov(3 * (int64_t)n, 0.0), op(n),
      rgb(3 * (int64_t)n, 0.0), depth(n), mg(n);
  std::vector<int32_t> radius(n), rect(4 * (int64_t)n);
  orc_projected P{xy.data(), conic.data(), cov.data(), op.data(), rgb.data(), depth.data(), radius.data(),
                  rect.data(), mg.data()};
  orc_project(s, X.data(), Q.data(), Sc.data(), cam, tile, &P);
  const int tiles_x = (cam->width + tile - 1) / tile, tiles_y = (cam->height + tile - 1) / tile;
  std::vector<uint32_t> dbits(n);
  for (int g = 0; g < n; ++g) {
    float f = (float)depth[g];
    std::memcpy(&dbits[g], &f, 4);
  }
  int64_t K = 0;
  for (int g = 0; g < n; ++g) K += (int64_t)(rect[4 * g + 2] - rect[4 * g]) * (rect[4 * g + 3] - rect[4 * g + 1]);
  std::vector<uint64_t> keys(K);
  std::vector<uint32_t> values(K), ranges(2 * (size_t)tiles_x * tiles_y);
  orc_bin_sort(n, dbits.data(), rect.data(), tiles_x, tiles_y, K, keys.data(), values.data(), ranges.data());
  orc_composite(cam->width, cam->height, tile, ranges.data(), values.data(), xy.data(), conic.data(), op.data(),
                rgb.data(), depth.data(), image, t_final, n_contrib, margin);
  return K;
}

}  // extern "C"

extern "C" int32_t orc_render_backward(const orc_scene* s, const orc_camera* cam, double t, int32_t deform,
                                       int32_t tile, const double* dl_dimage, orc_grads* grads) {
  (void)s; (void)cam; (void)t; (void)deform; (void)tile; (void)dl_dimage; (void)grads;
  return 1;
}
